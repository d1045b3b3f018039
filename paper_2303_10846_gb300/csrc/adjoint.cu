// Host side of the adjoint ABI (include/rykov.h, "adjoint of the steady residual
// operator"): the second workspace, the steady residual, the vector-Jacobian product,
// the objectives and the restarted GMRES solve of (dR/dX)^T lam = -dJ/dX.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "adjoint_dev.cuh"
#include "rykov_ctx.h"

namespace rk {

constexpr int ADJ_WPB = 8;

struct AdjState {
    int gen = -1;                  // bind generation of the main workspace it belongs to
    int m = 0;                     // Krylov dimension of a restart cycle
    size_t np = 0, n = 0;          // padded / packed state-vector lengths
    double *f0 = nullptr, *fbar = nullptr, *nbg = nullptr, *tau = nullptr, *fpar = nullptr,
           *iterp = nullptr, *pout = nullptr, *part = nullptr, *hd = nullptr;
    signed char* nbs = nullptr;
    int* slot_mirg = nullptr;
    double* slot_AVn = nullptr;
    // padded state vectors [2 N Kp | 6 N | 6 N]
    double *vzero = nullptr, *jv = nullptr, *lam = nullptr, *rv = nullptr, *tmp = nullptr,
           *tmp2 = nullptr, *V = nullptr;
    double* stage = nullptr;       // packed staging for host inputs / outputs
    // macroscopic part of the preconditioner: a padded phi-block temporary, the
    // (W, q) outputs of the collision-coupling product, the macro adjoint iterate and
    // the inverse macro diagonals
    double *pc1 = nullptr, *pcW = nullptr, *mY = nullptr, *mDinv = nullptr;
    // mixed-precision contexts: FP64 copies of phi and of the frozen limiter values,
    // s_ij per slot (the FP64 view of the context's FP32 per-velocity arrays)
    double *phi64 = nullptr, *lstore64 = nullptr, *slot_s64 = nullptr;
    double* hpin = nullptr;        // pinned host scratch
    int lam_obj = -1;              // objective of the stored lam (-1: none)
    long long lam_ver = -1;        // state version it was solved at
    long long launches = 0;
};

static inline int cdv(long long a, long long b) { return (int)((a + b - 1) / b); }

// out = -out on the phi block (the transposed sweeps' result), out = -in on (W, q)
__global__ void k_adj_precond_finish(const double* in, double* out, size_t n1, size_t np) {
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < np; t += (size_t)gridDim.x * blockDim.x)
        out[t] = t < n1 ? -out[t] : -in[t];
}

}  // namespace rk

using rk::AdjState;

void rk_adj_release(rk_ctx* ctx) {
    if (!ctx || !ctx->adj) return;
    if (ctx->adj->hpin) cudaFreeHost(ctx->adj->hpin);
    delete ctx->adj;
    ctx->adj = nullptr;
}

static size_t adj_carve(rk_ctx* ctx, int m, char* base, AdjState& A) {
    Carver cv{base};
    const size_t N = ctx->N, F = ctx->F, Kp = ctx->Kp, nnz = ctx->nnz, K = ctx->K;
    A.np = 2 * N * Kp + 12 * N;
    A.n = 2 * N * K + 12 * N;
    A.m = m;
    A.f0 = cv.take<double>(2 * F * Kp);
    A.fbar = cv.take<double>(2 * F * Kp);
    A.nbg = cv.take<double>(8 * N * Kp);
    A.nbs = cv.take<signed char>(2 * N * Kp);
    A.slot_mirg = cv.take<int>(nnz);
    A.slot_AVn = cv.take<double>(nnz);
    A.tau = cv.take<double>(N);
    A.fpar = cv.take<double>((size_t)rk::ADJ_FPAR * (ctx->Fb + 1));
    A.iterp = cv.take<double>(4);
    A.pout = cv.take<double>(16);
    A.part = cv.take<double>((size_t)rk::VEC_GRID * rk::GM_MAX);
    A.hd = cv.take<double>(3 * rk::GM_MAX + 8);
    A.vzero = cv.take<double>(A.np);
    A.jv = cv.take<double>(A.np);
    A.lam = cv.take<double>(A.np);
    A.rv = cv.take<double>(A.np);
    A.tmp = cv.take<double>(A.np);
    A.tmp2 = cv.take<double>(A.np);
    A.V = cv.take<double>((size_t)(m + 1) * A.np);
    A.stage = cv.take<double>(A.n);
    A.pc1 = cv.take<double>(2 * N * Kp);
    A.pcW = cv.take<double>(12 * N);
    A.mY = cv.take<double>(6 * N);
    A.mDinv = cv.take<double>(2 * N);
    A.slot_s64 = cv.take<double>(nnz);
    if (ctx->prec == RK_MIXED) {
        A.phi64 = cv.take<double>(2 * N * Kp);
        A.lstore64 = cv.take<double>(2 * N * Kp);
    }
    return cv.off + 256;
}

static int need_adj(rk_ctx* ctx, const char* who) {
    if (!ctx) return RK_EINVAL;
    if (!ctx->bound) return fail(ctx, RK_ESTATE, std::string(who) + ": bind a workspace first");
    if (!ctx->adj || ctx->adj->gen != ctx->bind_gen)
        return fail(ctx, RK_ESTATE, std::string(who) + ": bind an adjoint workspace first");
    if (!ctx->have_state) return fail(ctx, RK_ESTATE, std::string(who) + ": set a state first");
    return RK_OK;
}

extern "C" int rk_state_len(const rk_ctx* ctx, int64_t* n) {
    if (!ctx || !n) return RK_EINVAL;
    *n = 2 * ctx->N * ctx->K + 12 * ctx->N;
    return RK_OK;
}

extern "C" int rk_adjoint_workspace_size(rk_ctx* ctx, int32_t krylov_dim, size_t* bytes) {
    if (!ctx || !bytes) return RK_EINVAL;
    if (krylov_dim < 1 || krylov_dim > rk::GM_MAX)
        return fail(ctx, RK_EINVAL, "rk_adjoint_workspace_size: krylov_dim out of range");
    if (!ctx->mesh_ok || !ctx->dvs_ok) return fail(ctx, RK_ESTATE, "rk_adjoint_workspace_size: upload mesh and DVS first");
    AdjState A;
    *bytes = adj_carve(ctx, krylov_dim, nullptr, A);
    return RK_OK;
}

extern "C" int rk_bind_adjoint_workspace(rk_ctx* ctx, int32_t krylov_dim, void* dev_ptr, size_t bytes) {
    if (!ctx || !dev_ptr) return RK_EINVAL;
    if (!ctx->bound) return fail(ctx, RK_ESTATE, "rk_bind_adjoint_workspace: bind the main workspace first");
    size_t need = 0;
    int rc = rk_adjoint_workspace_size(ctx, krylov_dim, &need);
    if (rc) return rc;
    if (bytes < need)
        return fail(ctx, RK_ENOMEM, "rk_bind_adjoint_workspace: workspace too small (" + std::to_string(bytes) +
                                        " < " + std::to_string(need) + ")");
    if (reinterpret_cast<uintptr_t>(dev_ptr) & 255)
        return fail(ctx, RK_EINVAL, "rk_bind_adjoint_workspace: pointer not 256-byte aligned");
    rk_adj_release(ctx);
    AdjState* A = new (std::nothrow) AdjState();
    if (!A) return fail(ctx, RK_ENOMEM, "rk_bind_adjoint_workspace: host allocation failed");
    if (cudaMallocHost(&A->hpin, (3 * rk::GM_MAX + 16) * sizeof(double)) != cudaSuccess) {
        delete A;
        return fail(ctx, RK_ECUDA, "rk_bind_adjoint_workspace: pinned host buffer");
    }
    ctx->adj = A;
    adj_carve(ctx, krylov_dim, static_cast<char*>(dev_ptr), *A);
    cudaStream_t s = ctx->stream;
    const size_t N = ctx->N, nnz = ctx->nnz;
    // mirror slots (the same face in the neighbour's list) and A_f / V_neighbour
    std::vector<int> mir(nnz, -1);
    std::vector<double> avn(nnz, 0.0);
    for (size_t i = 0; i < N; ++i) {
        for (int m = ctx->slot_off[i]; m < ctx->slot_off[i + 1]; ++m) {
            const int j = ctx->slot_nbr[m];
            if (j < 0) continue;
            for (int mm = ctx->slot_off[j]; mm < ctx->slot_off[j + 1]; ++mm)
                if (ctx->slot_face[mm] == ctx->slot_face[m]) mir[m] = mm;
            avn[m] = ctx->fa[ctx->slot_face[m]] / ctx->cv[j];
        }
    }
    // zero everything once: the K padding of every vector stays 0
    CK(cudaMemsetAsync(dev_ptr, 0, need - 256, s));
    CK(cudaMemcpyAsync(A->slot_mirg, mir.data(), nnz * sizeof(int), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(A->slot_AVn, avn.data(), nnz * sizeof(double), cudaMemcpyHostToDevice, s));
    {
        const rk::DevBase& b = ctx->prec == RK_FP64 ? static_cast<const rk::DevBase&>(ctx->dd)
                                                    : static_cast<const rk::DevBase&>(ctx->df);
        rk::k_adj_slot_s<<<rk::cdv(nnz, 256), 256, 0, s>>>(b, A->slot_s64);
        CK(cudaGetLastError());
    }
    CK(cudaStreamSynchronize(s));
    A->gen = ctx->bind_gen;
    return RK_OK;
}

// The FP64 view of the context: the FP64 context's own arrays, or, for a mixed
// context, its FP64 geometry and state with FP64 copies of the per-velocity arrays
static rk::Dev<double> dview(rk_ctx* ctx, AdjState& A) {
    if (ctx->prec == RK_FP64) return ctx->dd;
    rk::Dev<double> d{};
    static_cast<rk::DevBase&>(d) = static_cast<const rk::DevBase&>(ctx->df);
    const double v[8] = {d.R, d.Z, d.mu_ref, d.T_ref, d.omega_vis, d.omega0, d.omega1, d.delta};
    for (int j = 0; j < 8; ++j) d.tp[j] = v[j];
    d.slot_nT = const_cast<double*>(d.slot_n);
    d.slot_AVT = d.slot_AV;
    d.slot_dT = d.slot_d;
    d.slot_lsqT = d.slot_lsq;
    d.slot_sT = A.slot_s64;
    d.fnT = const_cast<double*>(d.fn);
    d.fsT = d.fs;
    d.uT = d.u;
    d.wT = d.w;
    d.phi = A.phi64;
    d.face = A.fbar;
    d.res = d.dphi = nullptr;
    d.lstore = A.lstore64;
    d.debug = 0;
    return d;
}

// mixed contexts: refresh the FP64 copies of phi and of the frozen limiter values
static cudaError_t adj_sync(rk_ctx* ctx, AdjState& A) {
    if (ctx->prec != RK_MIXED) return cudaSuccess;
    const size_t n = 2 * (size_t)ctx->N * ctx->Kp;
    rk::k_adj_upcast<<<1216, 256, 0, ctx->stream>>>(ctx->df.phi, A.phi64, n);
    rk::k_adj_upcast<<<1216, 256, 0, ctx->stream>>>(ctx->df.lstore, A.lstore64, n);
    A.launches += 2;
    return cudaGetLastError();
}

// Per-velocity arithmetic of the adjoint kernels: FP64 for FP64 contexts; FP32 with
// compensated velocity sums for mixed-precision contexts (the state and the vectors
// stay FP64), unless RYKOV_ADJ_FP64=1 asks for FP64 arithmetic there too
static bool adj_fp32(const rk_ctx* ctx) {
    if (ctx->prec != RK_MIXED) return false;
    const char* v = std::getenv("RYKOV_ADJ_FP64");
    return !(v && std::strcmp(v, "0") != 0);
}

// ---- kernel sequences -------------------------------------------------------------
static rk::AdjBufs adj_bufs(rk_ctx* ctx, AdjState& A, const double* v, double* o) {
    rk::AdjBufs a{};
    const size_t N = ctx->N, n1 = 2 * N * (size_t)ctx->Kp;
    a.f0 = A.f0; a.fbar = A.fbar;
    a.vphi = v; a.vW = v + n1; a.vq = v + n1 + 6 * N;
    a.ophi = o; a.oW = o + n1; a.oq = o + n1 + 6 * N;
    a.nbg = A.nbg; a.nbs = A.nbs; a.slot_mirg = A.slot_mirg; a.slot_AVn = A.slot_AVn;
    a.tau = A.tau; a.fpar = A.fpar; a.iterp = A.iterp;
    a.obj_scale = 0.0; a.objective = 0;
    if (ctx->prec == RK_MIXED) {
        a.uf = ctx->df.uT; a.wf = ctx->df.wT; a.phif = ctx->df.phi;
        a.f0f = ctx->df.face;            // written by adj_prepare's FP32 reconstruction
    }
    a.edrag[0] = 1.0; a.edrag[1] = a.edrag[2] = 0.0;
    for (int b = 0; b < MAX_BC; ++b) {
        if (ctx->bck[b] != RK_FARFIELD) continue;
        const double* U = ctx->bcv + 5 * b + 1;
        const double nrm = std::sqrt(U[0] * U[0] + U[1] * U[1] + U[2] * U[2]);
        if (nrm > 0.0) {
            for (int d = 0; d < 3; ++d) a.edrag[d] = U[d] / nrm;
        }
        break;
    }
    return a;
}

// the limited reconstruction phi(x_f - u s) of the current state into f0, and tau(W)
static cudaError_t adj_prepare(rk_ctx* ctx, AdjState& A) {
    // the steady operator's reconstruction: the limiter of rk_params, with the stored
    // values once the iteration has frozen them
    double mode = (double)ctx->p.limiter;
    if (ctx->p.limiter == 1 && ctx->p.limiter_freeze > 0 && ctx->iter >= ctx->p.limiter_freeze) mode = 3.0;
    const double ip[4] = {0.0, mode, 0.0, 0.0};
    cudaError_t e = cudaMemcpyAsync(A.iterp, ip, sizeof(ip), cudaMemcpyHostToDevice, ctx->stream);
    if (e != cudaSuccess) return e;
    if ((e = adj_sync(ctx, A)) != cudaSuccess) return e;
    rk::Dev<double> d = dview(ctx, A);
    d.iterp = A.iterp;
    if (adj_fp32(ctx)) {
        // FP32 arithmetic: the context's own FP32 reconstruction, written to its face
        // array (scratch of the iteration) and widened into f0
        rk::Dev<float> df = ctx->df;
        df.iterp = A.iterp;
        rk::k_recon<float, 8><<<rk::cdv(ctx->N, 8), 256, 0, ctx->stream>>>(df);
        rk::k_adj_upcast<<<1216, 256, 0, ctx->stream>>>(df.face, A.f0, 2 * (size_t)ctx->F * ctx->Kp);
        A.launches += 2;
    } else {
        d.face = A.f0;
        rk::k_recon<double, 8><<<rk::cdv(ctx->N, 8), 256, 0, ctx->stream>>>(d);
        A.launches++;
    }
    rk::k_adj_tau<<<rk::cdv(ctx->N, 256), 256, 0, ctx->stream>>>(d, A.tau);
    A.launches++;
    return cudaGetLastError();
}

// o = (dR/dX)^T v (padded vectors), pout = (dR/dp)^T v; with obj_scale = 1 and v = 0
// it gives dJ/dX, pout[0-5] = dJ/dp|_X, pout[6] = J, pout[7-9] = force
static cudaError_t adj_apply(rk_ctx* ctx, AdjState& A, const double* v, double* o, double obj_scale,
                             int objective) {
    rk::AdjBufs a = adj_bufs(ctx, A, v, o);
    a.obj_scale = obj_scale;
    a.objective = objective;
    const rk::Dev<double> d = dview(ctx, A);
    cudaStream_t s = ctx->stream;
    const int gc = rk::cdv(ctx->N, rk::ADJ_WPB);
    const bool f32 = adj_fp32(ctx);
    if (f32) {
        // the phi block of v rounded to FP32 once, into the upper half of the gradient
        // adjoint buffer (FP32 arithmetic stores those adjoints in its lower half)
        float* vf = reinterpret_cast<float*>(A.nbg) + 8 * (size_t)ctx->N * ctx->Kp;
        rk::k_adj_downcast<<<1216, 256, 0, s>>>(v, vf, 2 * (size_t)ctx->N * ctx->Kp);
        a.vphif = vf;
        A.launches++;
    }
    if (f32) rk::k_adj_cell<rk::ADJ_WPB, float><<<gc, rk::ADJ_WPB * 32, 0, s>>>(d, a, 3);
    else rk::k_adj_cell<rk::ADJ_WPB, double><<<gc, rk::ADJ_WPB * 32, 0, s>>>(d, a, 3);
    A.launches += 4;
    if (ctx->Fi) {
        const int gf = rk::cdv(ctx->Fi, rk::ADJ_WPB);
        if (f32) rk::k_adj_face_interior<rk::ADJ_WPB, float><<<gf, rk::ADJ_WPB * 32, 0, s>>>(d, a);
        else rk::k_adj_face_interior<rk::ADJ_WPB, double><<<gf, rk::ADJ_WPB * 32, 0, s>>>(d, a);
        A.launches++;
    }
    if (ctx->Fb) {
        rk::k_adj_face_boundary<256><<<ctx->Fb, 256, 0, s>>>(d, a);
        rk::k_adj_params<<<1, 32, 0, s>>>(A.fpar, ctx->Fb, A.pout);
        A.launches += 2;
    } else {
        cudaError_t e = cudaMemsetAsync(A.pout, 0, 16 * sizeof(double), s);
        if (e != cudaSuccess) return e;
    }
    if (f32) rk::k_adj_gather<rk::ADJ_WPB, float><<<gc, rk::ADJ_WPB * 32, 0, s>>>(d, a);
    else rk::k_adj_gather<rk::ADJ_WPB, double><<<gc, rk::ADJ_WPB * 32, 0, s>>>(d, a);
    if (f32) rk::k_adj_gather2<rk::ADJ_WPB, float><<<gc, rk::ADJ_WPB * 32, 0, s>>>(d, a);
    else rk::k_adj_gather2<rk::ADJ_WPB, double><<<gc, rk::ADJ_WPB * 32, 0, s>>>(d, a);
    return cudaGetLastError();
}

// out = P^-1 in: transposed colour sweeps on the phi block (negated), -in on (W, q)
static cudaError_t adj_precond(rk_ctx* ctx, AdjState& A, const double* in, double* out) {
    cudaStream_t s = ctx->stream;
    const size_t n1 = 2 * (size_t)ctx->N * ctx->Kp;
    cudaError_t e = cudaMemsetAsync(out, 0, n1 * sizeof(double), s);
    if (e != cudaSuccess) return e;
    rk::AdjBufs a = adj_bufs(ctx, A, in, out);
    const rk::Dev<double> d = dview(ctx, A);
    const int C = ctx->C;
    for (int sw = 0; sw < ctx->p.n_micro_sgs; ++sw) {
        for (int dir = 0; dir < 2; ++dir) {
            for (int cc = 0; cc < C; ++cc) {
                const int col = dir == 0 ? cc : C - 1 - cc;
                const int lo = ctx->col_off[col], n = ctx->col_off[col + 1] - lo;
                if (n == 0) continue;
                if (adj_fp32(ctx))
                    rk::k_adj_sweep<rk::ADJ_WPB, float><<<rk::cdv(n, rk::ADJ_WPB), rk::ADJ_WPB * 32, 0, s>>>(
                        d, a, ctx->sched.col_cell + lo, n, in, out);
                else
                    rk::k_adj_sweep<rk::ADJ_WPB, double><<<rk::cdv(n, rk::ADJ_WPB), rk::ADJ_WPB * 32, 0, s>>>(
                        d, a, ctx->sched.col_cell + lo, n, in, out);
                A.launches++;
            }
        }
    }
    rk::k_adj_precond_finish<<<1216, 256, 0, s>>>(in, out, n1, A.np);
    A.launches++;
    return cudaGetLastError();
}

// out = P^-T in with the macroscopic coupling of the forward iteration (transposed):
//   t     = S^-T (in_phi + M_Y^T in_Y)              transposed micro sweeps
//   x     = L^-T (B_W^T t)                          transposed macro PR-SGS sweeps
//   out   = -(t + M_W^T x),  -in_Y                  (the sign convention of adj_precond)
static cudaError_t adj_precond_macro(rk_ctx* ctx, AdjState& A, const double* in, double* out) {
    cudaStream_t s = ctx->stream;
    const size_t N = ctx->N, n1 = 2 * N * (size_t)ctx->Kp;
    const rk::Dev<double> d = dview(ctx, A);
    const double* zW = A.vzero + n1;               // zero (W, q) blocks
    rk::k_adj_momT<<<1216, 256, 0, s>>>(d, in, in + n1, in + n1 + 6 * N, 1.0, A.pc1);
    cudaError_t e = cudaMemsetAsync(out, 0, n1 * sizeof(double), s);
    if (e != cudaSuccess) return e;
    rk::AdjBufs a = adj_bufs(ctx, A, in, out);
    const int C = ctx->C;
    const bool f32 = adj_fp32(ctx);
    for (int sw = 0; sw < ctx->p.n_micro_sgs; ++sw) {
        for (int dir = 0; dir < 2; ++dir) {
            for (int cc = 0; cc < C; ++cc) {
                const int col = dir == 0 ? cc : C - 1 - cc;
                const int lo = ctx->col_off[col], n = ctx->col_off[col + 1] - lo;
                if (n == 0) continue;
                if (f32)
                    rk::k_adj_sweep<rk::ADJ_WPB, float><<<rk::cdv(n, rk::ADJ_WPB), rk::ADJ_WPB * 32, 0, s>>>(
                        d, a, ctx->sched.col_cell + lo, n, A.pc1, out);
                else
                    rk::k_adj_sweep<rk::ADJ_WPB, double><<<rk::cdv(n, rk::ADJ_WPB), rk::ADJ_WPB * 32, 0, s>>>(
                        d, a, ctx->sched.col_cell + lo, n, A.pc1, out);
                A.launches++;
            }
        }
    }
    // B_W^T t: the collision coupling's W derivative applied to t (k_adj_cell, mode 2,
    // with zero (W, q) weights)
    rk::AdjBufs b = adj_bufs(ctx, A, out, nullptr);
    b.vW = zW;
    b.vq = zW + 6 * N;
    b.oW = A.pcW;
    b.oq = A.pcW + 6 * N;
    const int gc = rk::cdv(ctx->N, rk::ADJ_WPB);
    if (f32) {
        float* vf = reinterpret_cast<float*>(A.nbg) + 8 * (size_t)ctx->N * ctx->Kp;
        rk::k_adj_downcast<<<1216, 256, 0, s>>>(out, vf, n1);
        b.vphif = vf;
        rk::k_adj_cell<rk::ADJ_WPB, float><<<gc, rk::ADJ_WPB * 32, 0, s>>>(d, b, 2);
        A.launches += 2;
    } else {
        rk::k_adj_cell<rk::ADJ_WPB, double><<<gc, rk::ADJ_WPB * 32, 0, s>>>(d, b, 2);
        A.launches++;
    }
    // L^-T (B_W^T t) by transposed colour sweeps of the macro operator
    rk::k_adj_macro_prep<<<rk::cdv(ctx->N, 128), 128, 0, s>>>(d, A.tau, A.mDinv);
    if ((e = cudaMemsetAsync(A.mY, 0, 6 * N * sizeof(double), s)) != cudaSuccess) return e;
    for (int it = 0; it < ctx->p.n_macro_sgs; ++it) {
        for (int dir = 0; dir < 2; ++dir) {
            for (int cc = 0; cc < C; ++cc) {
                const int col = dir == 0 ? cc : C - 1 - cc;
                const int lo = ctx->col_off[col], n = ctx->col_off[col + 1] - lo;
                if (n == 0) continue;
                rk::k_adj_macro_sweepT<<<rk::cdv(n, 128), 128, 0, s>>>(d, ctx->sched.col_cell + lo, n, A.mDinv,
                                                                      A.pcW, A.mY);
                A.launches++;
            }
        }
    }
    // t + M_W^T x, then the signs
    rk::k_adj_momT<<<1216, 256, 0, s>>>(d, out, A.mY, zW, 1.0, out);
    rk::k_adj_precond_finish<<<1216, 256, 0, s>>>(in, out, n1, A.np);
    A.launches += 4;
    return cudaGetLastError();
}

// the preconditioner of the adjoint solve: with the macroscopic coupling (default), or
// the transposed micro sweeps alone (RYKOV_ADJ_PC=micro)
static cudaError_t adj_pc(rk_ctx* ctx, AdjState& A, const double* in, double* out) {
    const char* v = std::getenv("RYKOV_ADJ_PC");
    if (v && std::strcmp(v, "micro") == 0) return adj_precond(ctx, A, in, out);
    return adj_precond_macro(ctx, A, in, out);
}

// dots of x with V_0..V_{m-1} into dev (device), deterministic
static void adj_mdot(rk_ctx* ctx, AdjState& A, const double* x, const double* V, int m, double* dev) {
    rk::k_vec_mdot<<<rk::VEC_GRID, rk::VEC_BS, 0, ctx->stream>>>(x, V, A.np, m, A.np, A.part);
    rk::k_vec_finish<<<1, 64, 0, ctx->stream>>>(A.part, m, dev);
    A.launches += 2;
}

static int adj_norm(rk_ctx* ctx, AdjState& A, const double* x, double* out) {
    adj_mdot(ctx, A, x, x, 1, A.hd + 3 * rk::GM_MAX);
    CK(cudaMemcpyAsync(A.hpin, A.hd + 3 * rk::GM_MAX, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    *out = std::sqrt(A.hpin[0]);
    return RK_OK;
}

static void vec_axpby(rk_ctx* ctx, AdjState& A, double a, const double* x, double b, double* y) {
    rk::k_vec_axpby<<<1216, 256, 0, ctx->stream>>>(a, x, b, y, A.np);
    A.launches++;
}

// packed <-> padded
static cudaError_t adj_unpack(rk_ctx* ctx, AdjState& A, const double* x, double* vec) {
    const size_t N = ctx->N, n1 = 2 * N * (size_t)ctx->Kp;
    rk::k_adj_unpack<<<rk::cdv((long long)A.n, 256), 256, 0, ctx->stream>>>(x, (int)N, (int)ctx->K, ctx->Kp, vec,
                                                                           vec + n1, vec + n1 + 6 * N);
    A.launches++;
    return cudaGetLastError();
}
static cudaError_t adj_pack(rk_ctx* ctx, AdjState& A, const double* vec, double* x) {
    const size_t N = ctx->N, n1 = 2 * N * (size_t)ctx->Kp;
    rk::k_adj_pack<<<rk::cdv((long long)A.n, 256), 256, 0, ctx->stream>>>(vec, vec + n1, vec + n1 + 6 * N, (int)N,
                                                                         (int)ctx->K, ctx->Kp, x);
    A.launches++;
    return cudaGetLastError();
}

// packed input (host or device) -> padded device vector
static int load_vec(rk_ctx* ctx, AdjState& A, const double* x, int on_device, double* vec) {
    const double* src = x;
    if (!on_device) {
        CK(cudaMemcpyAsync(A.stage, x, A.n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
        src = A.stage;
    }
    CK(adj_unpack(ctx, A, src, vec));
    return RK_OK;
}
// padded device vector -> packed output (host or device); synchronises
static int store_vec(rk_ctx* ctx, AdjState& A, const double* vec, double* x, int on_device) {
    if (on_device) {
        CK(adj_pack(ctx, A, vec, x));
    } else {
        CK(adj_pack(ctx, A, vec, A.stage));
        CK(cudaMemcpyAsync(x, A.stage, A.n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    }
    CK(cudaStreamSynchronize(ctx->stream));
    return RK_OK;
}

// ---- ABI --------------------------------------------------------------------------
extern "C" int rk_get_state(rk_ctx* ctx, double* x, int on_device) {
    int rc = need_adj(ctx, "rk_get_state");
    if (rc) return rc;
    if (!x) return fail(ctx, RK_EINVAL, "rk_get_state: null pointer");
    AdjState& A = *ctx->adj;
    CK(adj_sync(ctx, A));
    const rk::Dev<double> d = dview(ctx, A);
    const size_t N = ctx->N, n1 = 2 * N * (size_t)ctx->Kp;
    // assemble the padded vector [phi | W | q] in tmp, then pack
    CK(cudaMemcpyAsync(A.tmp, d.phi, n1 * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
    CK(cudaMemcpyAsync(A.tmp + n1, d.W, 6 * N * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
    CK(cudaMemcpyAsync(A.tmp + n1 + 6 * N, d.q, 6 * N * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
    return store_vec(ctx, A, A.tmp, x, on_device);
}

extern "C" int rk_put_state(rk_ctx* ctx, const double* x, int on_device) {
    if (!ctx) return RK_EINVAL;
    if (!ctx->adj || ctx->adj->gen != ctx->bind_gen || !ctx->bound)
        return fail(ctx, RK_ESTATE, "rk_put_state: bind the workspaces first");
    if (!x) return fail(ctx, RK_EINVAL, "rk_put_state: null pointer");
    AdjState& A = *ctx->adj;
    const size_t N = ctx->N, n1 = 2 * N * (size_t)ctx->Kp;
    const double* src = x;
    if (!on_device) {
        CK(cudaMemcpyAsync(A.stage, x, A.n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
        src = A.stage;
    }
    const rk::Dev<double> d = dview(ctx, A);
    rk::k_adj_unpack<<<rk::cdv((long long)A.n, 256), 256, 0, ctx->stream>>>(src, (int)N, (int)ctx->K, ctx->Kp,
                                                                           d.phi, d.W, d.q);
    CK(cudaGetLastError());
    if (ctx->prec == RK_MIXED) {
        // a mixed context stores phi in FP32 (rounded)
        rk::k_adj_downcast<<<1216, 256, 0, ctx->stream>>>(A.phi64, ctx->df.phi, n1);
        CK(cudaGetLastError());
    }
    CK(cudaMemsetAsync(d.iterp, 0, 4 * sizeof(double), ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->iter = 0;
    ctx->have_state = true;
    ctx->state_ver++;
    return RK_OK;
}

extern "C" int rk_steady_residual(rk_ctx* ctx, double* r, int on_device) {
    int rc = need_adj(ctx, "rk_steady_residual");
    if (rc) return rc;
    if (!r) return fail(ctx, RK_EINVAL, "rk_steady_residual: null pointer");
    AdjState& A = *ctx->adj;
    CK(adj_prepare(ctx, A));
    // forward face pass of the steady operator into the fbar scratch (FP64)
    rk::Dev<double> d = dview(ctx, A);
    d.iterp = A.iterp;
    d.face = A.fbar;
    d.debug = 0;
    cudaStream_t s = ctx->stream;
    rk::k_recon<double, 8><<<rk::cdv(ctx->N, 8), 256, 0, s>>>(d);
    if (ctx->Fi) rk::k_face_interior<double, 8, 1><<<rk::cdv(ctx->Fi, 8), 256, 0, s>>>(d);
    if (ctx->Fb) rk::k_face_boundary<double, 256><<<ctx->Fb, 256, 0, s>>>(d);
    rk::AdjBufs a = adj_bufs(ctx, A, A.vzero, A.tmp);
    rk::k_adj_residual<rk::ADJ_WPB><<<rk::cdv(ctx->N, rk::ADJ_WPB), rk::ADJ_WPB * 32, 0, s>>>(d, a);
    A.launches += 4;
    CK(cudaGetLastError());
    return store_vec(ctx, A, A.tmp, r, on_device);
}

extern "C" int rk_vjp(rk_ctx* ctx, const double* v, double* out, double* out_params, int on_device) {
    int rc = need_adj(ctx, "rk_vjp");
    if (rc) return rc;
    if (!v || !out) return fail(ctx, RK_EINVAL, "rk_vjp: null pointer");
    AdjState& A = *ctx->adj;
    if ((rc = load_vec(ctx, A, v, on_device, A.rv))) return rc;
    CK(adj_prepare(ctx, A));
    CK(adj_apply(ctx, A, A.rv, A.tmp, 0.0, 0));
    if (out_params) {
        CK(cudaMemcpyAsync(A.hpin, A.pout, 6 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    }
    if ((rc = store_vec(ctx, A, A.tmp, out, on_device))) return rc;
    if (out_params) std::memcpy(out_params, A.hpin, 6 * sizeof(double));
    return RK_OK;
}

// J, force and dJ/dp|_X (host), dJ/dX into A.jv; drag adds the explicit dependence of
// e = U_inf / |U_inf| on the farfield velocity
static int objective_impl(rk_ctx* ctx, AdjState& A, int objective, double* J, double dJdp[6]) {
    CK(adj_prepare(ctx, A));
    CK(adj_apply(ctx, A, A.vzero, A.jv, 1.0, objective));
    CK(cudaMemcpyAsync(A.hpin, A.pout, 10 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (int j = 0; j < 6; ++j) dJdp[j] = A.hpin[j];
    *J = A.hpin[6];
    if (objective == RK_OBJ_DRAG) {
        for (int b = 0; b < MAX_BC; ++b) {
            if (ctx->bck[b] != RK_FARFIELD) continue;
            const double* U = ctx->bcv + 5 * b + 1;
            const double nrm = std::sqrt(U[0] * U[0] + U[1] * U[1] + U[2] * U[2]);
            if (nrm > 0.0) {
                const double* Fo = A.hpin + 7;
                const double Fe = (Fo[0] * U[0] + Fo[1] * U[1] + Fo[2] * U[2]) / nrm;
                for (int d = 0; d < 3; ++d) dJdp[2 + d] += (Fo[d] - Fe * U[d] / nrm) / nrm;
            }
            break;
        }
    }
    return RK_OK;
}

extern "C" int rk_objective(rk_ctx* ctx, int objective, double* J, double* dJdX, double* dJdp, int on_device) {
    int rc = need_adj(ctx, "rk_objective");
    if (rc) return rc;
    if (objective != RK_OBJ_HEAT && objective != RK_OBJ_DRAG) return fail(ctx, RK_EINVAL, "rk_objective: unknown objective");
    AdjState& A = *ctx->adj;
    double Jv = 0.0, dp[6];
    if ((rc = objective_impl(ctx, A, objective, &Jv, dp))) return rc;
    if (J) *J = Jv;
    if (dJdp) std::memcpy(dJdp, dp, sizeof(dp));
    if (dJdX) return store_vec(ctx, A, A.jv, dJdX, on_device);
    return RK_OK;
}

// restarted GMRES(m), right preconditioned, classical Gram-Schmidt with one
// re-orthogonalisation; Givens rotations and the small least-squares problem on the host
extern "C" int rk_adjoint_solve(rk_ctx* ctx, int objective, int32_t max_iter, double tol, int32_t* iters_done,
                                double* rel_res, double* J, double* dJdp) {
    int rc = need_adj(ctx, "rk_adjoint_solve");
    if (rc) return rc;
    if (objective != RK_OBJ_HEAT && objective != RK_OBJ_DRAG) return fail(ctx, RK_EINVAL, "rk_adjoint_solve: unknown objective");
    if (max_iter < 0 || !(tol >= 0.0)) return fail(ctx, RK_EINVAL, "rk_adjoint_solve: bad max_iter or tol");
    AdjState& A = *ctx->adj;
    cudaStream_t s = ctx->stream;
    double Jv = 0.0, dpx[6];
    if ((rc = objective_impl(ctx, A, objective, &Jv, dpx))) return rc;
    double jn = 0.0;
    if ((rc = adj_norm(ctx, A, A.jv, &jn))) return rc;
    const bool warm = A.lam_obj == objective && A.lam_ver == ctx->state_ver;
    if (!warm) CK(cudaMemsetAsync(A.lam, 0, A.np * sizeof(double), s));
    // rv = -(A^T lam + j)
    auto residual = [&](double* beta) -> int {
        CK(adj_apply(ctx, A, A.lam, A.rv, 0.0, 0));
        vec_axpby(ctx, A, -1.0, A.jv, -1.0, A.rv);
        return adj_norm(ctx, A, A.rv, beta);
    };
    double beta = 0.0;
    if ((rc = residual(&beta))) return rc;
    const int m = A.m;
    int total = 0;
    std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m);
    auto Hx = [&](int i, int j) -> double& { return H[(size_t)i * m + j]; };
    while (jn > 0.0 && beta / jn > tol && total < max_iter) {
        if (!std::isfinite(beta)) return fail(ctx, RK_EDIVERGED, "rk_adjoint_solve: non-finite residual");
        vec_axpby(ctx, A, 1.0 / beta, A.rv, 0.0, A.V);
        std::fill(g.begin(), g.end(), 0.0);
        g[0] = beta;
        int jj = 0;
        for (int j = 0; j < m && total < max_iter; ++j) {
            double* Vj = A.V + (size_t)j * A.np;
            double* w = A.V + (size_t)(j + 1) * A.np;
            CK(adj_pc(ctx, A, Vj, A.tmp));
            CK(adj_apply(ctx, A, A.tmp, w, 0.0, 0));
            // two passes of classical Gram-Schmidt
            adj_mdot(ctx, A, w, A.V, j + 1, A.hd);
            rk::k_vec_msub<<<1216, 256, 0, s>>>(w, A.V, A.np, j + 1, A.hd, A.np);
            adj_mdot(ctx, A, w, A.V, j + 1, A.hd + rk::GM_MAX);
            rk::k_vec_msub<<<1216, 256, 0, s>>>(w, A.V, A.np, j + 1, A.hd + rk::GM_MAX, A.np);
            adj_mdot(ctx, A, w, w, 1, A.hd + 2 * rk::GM_MAX);
            A.launches += 2;
            CK(cudaMemcpyAsync(A.hpin, A.hd, (2 * rk::GM_MAX + 1) * sizeof(double), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            for (int i = 0; i <= j; ++i) Hx(i, j) = A.hpin[i] + A.hpin[rk::GM_MAX + i];
            const double hn = std::sqrt(A.hpin[2 * rk::GM_MAX]);
            Hx(j + 1, j) = hn;
            if (!std::isfinite(hn)) return fail(ctx, RK_EDIVERGED, "rk_adjoint_solve: non-finite Krylov vector");
            if (hn > 0.0) vec_axpby(ctx, A, 0.0, w, 1.0 / hn, w);
            for (int i = 0; i < j; ++i) {
                const double t = cs[i] * Hx(i, j) + sn[i] * Hx(i + 1, j);
                Hx(i + 1, j) = -sn[i] * Hx(i, j) + cs[i] * Hx(i + 1, j);
                Hx(i, j) = t;
            }
            const double r = std::hypot(Hx(j, j), Hx(j + 1, j));
            cs[j] = r > 0.0 ? Hx(j, j) / r : 1.0;
            sn[j] = r > 0.0 ? Hx(j + 1, j) / r : 0.0;
            Hx(j, j) = r;
            Hx(j + 1, j) = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            ++total;
            jj = j + 1;
            if (std::fabs(g[j + 1]) <= tol * jn || hn == 0.0) break;
        }
        // y = H^-1 g (upper triangular), lam += P^-1 (V y)
        for (int i = jj - 1; i >= 0; --i) {
            double t = g[i];
            for (int k = i + 1; k < jj; ++k) t -= Hx(i, k) * y[k];
            y[i] = Hx(i, i) != 0.0 ? t / Hx(i, i) : 0.0;
        }
        CK(cudaMemcpyAsync(A.hd, y.data(), jj * sizeof(double), cudaMemcpyHostToDevice, s));
        CK(cudaMemsetAsync(A.tmp2, 0, A.np * sizeof(double), s));
        rk::k_vec_madd<<<1216, 256, 0, s>>>(A.tmp2, A.V, A.np, jj, A.hd, A.np);
        A.launches++;
        CK(adj_pc(ctx, A, A.tmp2, A.tmp));
        vec_axpby(ctx, A, 1.0, A.tmp, 1.0, A.lam);
        if ((rc = residual(&beta))) return rc;
    }
    if (!std::isfinite(beta)) return fail(ctx, RK_EDIVERGED, "rk_adjoint_solve: non-finite residual");
    A.lam_obj = objective;
    A.lam_ver = ctx->state_ver;
    // total derivative: dJ/dp|_X + lam^T dR/dp
    CK(adj_apply(ctx, A, A.lam, A.tmp, 0.0, 0));
    CK(cudaMemcpyAsync(A.hpin, A.pout, 6 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (dJdp)
        for (int j = 0; j < 6; ++j) dJdp[j] = dpx[j] + A.hpin[j];
    if (J) *J = Jv;
    if (iters_done) *iters_done = total;
    if (rel_res) *rel_res = jn > 0.0 ? beta / jn : 0.0;
    return RK_OK;
}

extern "C" int rk_adjoint_get(rk_ctx* ctx, double* lam, int on_device) {
    int rc = need_adj(ctx, "rk_adjoint_get");
    if (rc) return rc;
    if (!lam) return fail(ctx, RK_EINVAL, "rk_adjoint_get: null pointer");
    return store_vec(ctx, *ctx->adj, ctx->adj->lam, lam, on_device);
}
