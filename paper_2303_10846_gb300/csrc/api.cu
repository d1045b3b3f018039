// Host side of librykov: the C ABI declared in include/rykov.h.  Validates and
// stages the mesh and velocity space, builds the cell->face incidence lists and the
// colour schedule, carves every device array out of the caller's workspace, and
// enqueues the kernel sequence of one implicit iteration on the caller's stream.
#include <cmath>
#include <type_traits>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "rykov_ctx.h"

static double implicit_cfl(const rk_params& p, int64_t n) {
    if (p.cfl_imp0 <= 0.0 || p.cfl_ramp <= 1.0) return p.cfl_imp;
    double c = p.cfl_imp0 * std::pow(p.cfl_ramp, (double)n);
    return c < p.cfl_imp ? c : p.cfl_imp;
}

extern "C" int rk_version(void) { return RK_VERSION; }

extern "C" int rk_create(rk_ctx** out, int precision, uintptr_t cuda_stream) {
    if (!out) return RK_EINVAL;
    int base = precision & 0xff;
    if (base != RK_FP64 && base != RK_MIXED) return RK_EINVAL;
    rk_ctx* ctx = new (std::nothrow) rk_ctx();
    if (!ctx) return RK_ENOMEM;
    ctx->prec = base;
    ctx->debug = (precision & RK_DEBUG_FLAG) != 0;
    // RYKOV_GRAPH=0 switches off the CUDA graph of an iteration, RYKOV_COOP=1 switches
    // on the cooperative macro solve (same results; used to compare launch schemes)
    if (const char* v = std::getenv("RYKOV_GRAPH")) ctx->use_graph = std::strcmp(v, "0") != 0;
    if (const char* v = std::getenv("RYKOV_COOP")) ctx->use_coop = std::strcmp(v, "0") != 0;
    // RYKOV_STAGED: which micro sweeps stage their row loads (bits 0/1/2: first,
    // middle, last sweep); the results are the same either way
    if (const char* v = std::getenv("RYKOV_STAGED")) ctx->use_staged = std::atoi(v) & 15;
    if (const char* v = std::getenv("RYKOV_PRIO")) ctx->use_prio = std::strcmp(v, "0") != 0;
    // RK_MACRO_FP32 flag: mixed contexts solve the macro PR-SGS in FP32 in delta form
    // instead of FP64 (FP64 contexts ignore it)
    ctx->use_macro32 = (precision & RK_MACRO_FP32) != 0;
    // RYKOV_PDL=1: the macro phases with programmatic stream serialisation (same
    // results; off by default: in the graph the plain launches leave the micro-flux
    // branch beside them more room)
    if (const char* v = std::getenv("RYKOV_PDL")) ctx->use_pdl = std::strcmp(v, "0") != 0;
    // RYKOV_PACKED=0: the mixed-precision kernels with scalar FP32 arithmetic instead of
    // the packed pairs (same steps, rounding-level differences)
    if (const char* v = std::getenv("RYKOV_PACKED")) ctx->use_packed = std::strcmp(v, "0") != 0;
    ctx->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    for (int b = 0; b < MAX_BC; ++b) ctx->bck[b] = -1;
    std::memset(ctx->bcv, 0, sizeof(ctx->bcv));
    if (cudaMallocHost(&ctx->pin, 16 * sizeof(double)) != cudaSuccess) {
        delete ctx;
        return RK_ECUDA;
    }
    rk_params d{};
    d.R = 0.5; d.Z_rot = 3.5; d.omega_vis = 0.74; d.mu_ref = 0.05; d.T_ref = 1.0;
    d.omega0 = 0.2354; d.omega1 = 0.3049; d.delta = 1.0 / 1.55; d.cfl_s = 0.8;
    d.cfl_imp = 1e3; d.cfl_imp0 = 0.0; d.cfl_ramp = 1.0; d.lim_k = 0.1;
    d.n_micro_sgs = 2; d.n_macro_sgs = 40; d.limiter = 1; d.first_order_iters = 0;
    d.limiter_freeze = 0; d.viscosity_law = 0; d.sutherland_c = 111.0 / 273.0;
    ctx->p = d;
    *out = ctx;
    return RK_OK;
}

extern "C" int rk_destroy(rk_ctx* ctx) {
    if (!ctx) return RK_EINVAL;
    rk_adj_release(ctx);
    if (ctx->pin) cudaFreeHost(ctx->pin);
    for (cudaEvent_t e : ctx->prof.ev) cudaEventDestroy(e);
    if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
    if (ctx->cap) cudaStreamDestroy(ctx->cap);
    if (ctx->cap2) cudaStreamDestroy(ctx->cap2);
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
    if (ctx->ev_bnd) cudaEventDestroy(ctx->ev_bnd);
    if (ctx->ev_int) cudaEventDestroy(ctx->ev_int);
    delete ctx;
    return RK_OK;
}

extern "C" const char* rk_last_error(const rk_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

extern "C" int rk_set_params(rk_ctx* ctx, const rk_params* p) {
    if (!ctx || !p) return RK_EINVAL;
    if (!(p->R > 0) || !(p->Z_rot >= 1.0) || !(p->mu_ref > 0) || !(p->T_ref > 0) ||
        !(p->cfl_s > 0) || !(p->cfl_imp > 0) || p->n_micro_sgs < 1 || p->n_macro_sgs < 0 ||
        p->limiter < 0 || p->limiter > 2 || !(p->lim_k >= 0) || p->limiter_freeze < 0 ||
        (p->limiter_freeze > 0 && p->limiter_freeze <= p->first_order_iters) ||
        (p->viscosity_law != 0 && p->viscosity_law != 1) || !(p->sutherland_c >= 0))
        return fail(ctx, RK_EINVAL, "rk_set_params: parameter out of range");
    bool geo_change = ctx->p.cfl_s != p->cfl_s || ctx->p.lim_k != p->lim_k;
    ctx->p = *p;
    ctx->have_params = true;
    if (ctx->gexec) {
        cudaGraphExecDestroy(ctx->gexec);
        ctx->gexec = nullptr;
    }
    if (ctx->bound && geo_change) {
        ctx->dd.cfl_s = ctx->df.cfl_s = p->cfl_s;
        ctx->dd.lim_k = ctx->df.lim_k = p->lim_k;
    }
    auto fill = [&](auto& d) {
        d.R = p->R; d.Z = p->Z_rot; d.omega_vis = p->omega_vis; d.mu_ref = p->mu_ref;
        d.T_ref = p->T_ref; d.omega0 = p->omega0; d.omega1 = p->omega1; d.delta = p->delta;
        d.cfl_s = p->cfl_s; d.lim_k = p->lim_k;
        d.cfl_imp = p->cfl_imp; d.cfl_imp0 = p->cfl_imp0; d.cfl_ramp = p->cfl_ramp;
        d.first_order_iters = p->first_order_iters; d.limiter = p->limiter;
        d.limiter_freeze = p->limiter_freeze;
        d.viscosity_law = p->viscosity_law; d.sutherland_c = p->sutherland_c;
        using TT = std::remove_reference_t<decltype(d.tp[0])>;
        const double v[8] = {p->R, p->Z_rot, p->mu_ref, p->T_ref, p->omega_vis, p->omega0, p->omega1, p->delta};
        for (int j = 0; j < 8; ++j) d.tp[j] = (TT)v[j];
    };
    fill(ctx->dd);
    fill(ctx->df);
    if (ctx->bound && geo_change) {
        cudaError_t e = ctx->prec == RK_FP64 ? rk::Launch<double>::setup(ctx->dd, ctx->stream)
                                             : rk::Launch<float>::setup(ctx->df, ctx->stream);
        if (e != cudaSuccess) return fail(ctx, RK_ECUDA, cudaGetErrorString(e));
        CK(cudaStreamSynchronize(ctx->stream));
    }
    return RK_OK;
}

extern "C" int rk_set_bc(rk_ctx* ctx, int32_t bc_id, int32_t kind, double rho, const double* U, double T) {
    if (!ctx || !U) return RK_EINVAL;
    if (bc_id < 0 || bc_id >= MAX_BC) return fail(ctx, RK_EINVAL, "rk_set_bc: bc id out of range");
    if (kind != RK_WALL && kind != RK_FARFIELD) return fail(ctx, RK_EINVAL, "rk_set_bc: bad kind");
    if (!(T > 0) || (kind == RK_FARFIELD && !(rho > 0)))
        return fail(ctx, RK_EINVAL, "rk_set_bc: non-positive temperature or density");
    ctx->bck[bc_id] = kind;
    double* v = ctx->bcv + 5 * bc_id;
    v[0] = rho; v[1] = U[0]; v[2] = U[1]; v[3] = U[2]; v[4] = T;
    if (ctx->bound) {
        double* bcv = const_cast<double*>(ctx->prec == RK_FP64 ? ctx->dd.bcv : ctx->df.bcv);
        int* bck = const_cast<int*>(ctx->prec == RK_FP64 ? ctx->dd.bck : ctx->df.bck);
        CK(cudaMemcpyAsync(bcv, ctx->bcv, sizeof(ctx->bcv), cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaMemcpyAsync(bck, ctx->bck, sizeof(ctx->bck), cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    }
    return RK_OK;
}

extern "C" int rk_upload_mesh(rk_ctx* ctx, int64_t n_cell, int64_t n_face, const int64_t* face_cell,
                              const double* face_normal, const double* face_area,
                              const double* face_center, const double* cell_center,
                              const double* cell_volume, const int32_t* cell_colour) {
    if (!ctx) return RK_EINVAL;
    if (n_cell <= 0 || n_face <= 0 || n_cell > (1LL << 30) || n_face > (1LL << 30) || !face_cell ||
        !face_normal || !face_area || !face_center || !cell_center || !cell_volume || !cell_colour)
        return fail(ctx, RK_EINVAL, "rk_upload_mesh: bad sizes or null pointer");
    ctx->bound = false;
    ctx->mesh_ok = false;
    ctx->have_state = false;
    const int64_t N = n_cell, F = n_face;
    std::vector<int> nfaces(N, 0);
    std::vector<double> clo(3 * N, 0.0), asum(N, 0.0);
    for (int64_t f = 0; f < F; ++f) {
        int64_t a = face_cell[2 * f], b = face_cell[2 * f + 1];
        if (a < 0 || a >= N || b >= N || b < -MAX_BC || a == b)
            return fail(ctx, RK_EINVAL, "rk_upload_mesh: face " + std::to_string(f) + " has a bad cell index");
        if (!(face_area[f] > 0))
            return fail(ctx, RK_EINVAL, "rk_upload_mesh: non-positive face area");
        const double* n = face_normal + 3 * f;
        if (std::fabs(n[0] * n[0] + n[1] * n[1] + n[2] * n[2] - 1.0) > 1e-8)
            return fail(ctx, RK_EINVAL, "rk_upload_mesh: face normal not unit");
        nfaces[a]++;
        for (int d = 0; d < 3; ++d) clo[3 * a + d] += face_area[f] * n[d];
        asum[a] += face_area[f];
        if (b >= 0) {
            nfaces[b]++;
            for (int d = 0; d < 3; ++d) clo[3 * b + d] -= face_area[f] * n[d];
            asum[b] += face_area[f];
            if (cell_colour[a] == cell_colour[b])
                return fail(ctx, RK_EINVAL, "rk_upload_mesh: colouring not proper at face " + std::to_string(f));
        }
    }
    int C = 0;
    for (int64_t i = 0; i < N; ++i) {
        if (!(cell_volume[i] > 0)) return fail(ctx, RK_EINVAL, "rk_upload_mesh: non-positive volume");
        if (nfaces[i] < 1 || nfaces[i] > rk::MAXF)
            return fail(ctx, RK_EINVAL, "rk_upload_mesh: cell with 0 or more than 8 faces");
        if (cell_colour[i] < 0 || cell_colour[i] > 255) return fail(ctx, RK_EINVAL, "rk_upload_mesh: bad colour");
        C = std::max(C, cell_colour[i] + 1);
        double cl = std::sqrt(clo[3 * i] * clo[3 * i] + clo[3 * i + 1] * clo[3 * i + 1] + clo[3 * i + 2] * clo[3 * i + 2]);
        if (cl > 1e-8 * asum[i])
            return fail(ctx, RK_EINVAL, "rk_upload_mesh: cell " + std::to_string(i) + " is not closed");
    }
    ctx->N = N; ctx->F = F; ctx->C = C;
    ctx->fc.assign(face_cell, face_cell + 2 * F);
    ctx->fn.assign(face_normal, face_normal + 3 * F);
    ctx->fa.assign(face_area, face_area + F);
    ctx->fx.assign(face_center, face_center + 3 * F);
    ctx->cx.assign(cell_center, cell_center + 3 * N);
    ctx->cv.assign(cell_volume, cell_volume + N);
    ctx->col.assign(cell_colour, cell_colour + N);
    // cell -> face incidences in increasing face order
    ctx->slot_off.assign(N + 1, 0);
    for (int64_t i = 0; i < N; ++i) ctx->slot_off[i + 1] = ctx->slot_off[i] + nfaces[i];
    ctx->nnz = ctx->slot_off[N];
    ctx->slot_face.assign(ctx->nnz, 0); ctx->slot_nbr.assign(ctx->nnz, 0);
    ctx->slot_left.assign(ctx->nnz, 0); ctx->slot_ncol.assign(ctx->nnz, -1);
    ctx->slot_n.assign(3 * (size_t)ctx->nnz, 0.0);
    std::vector<int> fill(N, 0);
    ctx->face_int.clear(); ctx->face_bnd.clear();
    ctx->fc32.assign(2 * F, 0);
    for (int64_t f = 0; f < F; ++f) {
        int64_t a = face_cell[2 * f], b = face_cell[2 * f + 1];
        ctx->fc32[2 * f] = (int)a; ctx->fc32[2 * f + 1] = (int)b;
        int64_t cells[2] = {a, b};
        for (int side = 0; side < 2; ++side) {
            int64_t i = cells[side];
            if (i < 0) continue;
            int m = ctx->slot_off[i] + fill[i]++;
            ctx->slot_face[m] = (int)f;
            ctx->slot_left[m] = side == 0;
            ctx->slot_nbr[m] = (int)(side == 0 ? b : a);
            ctx->slot_ncol[m] = (side == 0 ? (b >= 0 ? cell_colour[b] : -1) : cell_colour[a]);
            for (int d = 0; d < 3; ++d) ctx->slot_n[(size_t)d * ctx->nnz + m] = face_normal[3 * f + d];
        }
        if (b >= 0) ctx->face_int.push_back((int)f);
        else ctx->face_bnd.push_back((int)f);
    }
    ctx->Fi = (int)ctx->face_int.size();
    ctx->Fb = (int)ctx->face_bnd.size();
    ctx->col_off.assign(C + 1, 0);
    for (int64_t i = 0; i < N; ++i) ctx->col_off[cell_colour[i] + 1]++;
    for (int c = 0; c < C; ++c) ctx->col_off[c + 1] += ctx->col_off[c];
    ctx->col_cell.assign(N, 0);
    std::vector<int> cf(C, 0);
    for (int64_t i = 0; i < N; ++i) ctx->col_cell[ctx->col_off[cell_colour[i]] + cf[cell_colour[i]]++] = (int)i;
    ctx->mesh_ok = true;
    return RK_OK;
}

extern "C" int rk_upload_dvs(rk_ctx* ctx, int64_t K, const double* u, const double* w) {
    if (!ctx) return RK_EINVAL;
    if (K <= 0 || K > (1 << 20) || !u || !w) return fail(ctx, RK_EINVAL, "rk_upload_dvs: bad size or null pointer");
    for (int64_t k = 0; k < K; ++k)
        if (!(w[k] > 0) || !std::isfinite(u[3 * k]) || !std::isfinite(u[3 * k + 1]) || !std::isfinite(u[3 * k + 2]))
            return fail(ctx, RK_EINVAL, "rk_upload_dvs: non-positive weight or non-finite velocity");
    ctx->bound = false;
    ctx->have_state = false;
    ctx->K = K;
    ctx->Kp = (int)((K + 31) / 32 * 32);
    ctx->u.assign(u, u + 3 * K);
    ctx->w.assign(w, w + K);
    ctx->dvs_ok = true;
    return RK_OK;
}

extern "C" int rk_dims(const rk_ctx* ctx, int64_t out[6]) {
    if (!ctx || !out) return RK_EINVAL;
    int nw = 0;
    for (int f : ctx->face_bnd) {
        int bc = -1 - (int)ctx->fc[2 * (size_t)f + 1];
        if (ctx->bck[bc] == RK_WALL) ++nw;
    }
    out[0] = ctx->N; out[1] = ctx->F; out[2] = ctx->K; out[3] = ctx->Kp; out[4] = ctx->C; out[5] = nw;
    return RK_OK;
}

// Carve every device array; with base == nullptr only count bytes.
template <typename T>
static size_t carve(rk_ctx* ctx, char* base, rk::Dev<T>& d) {
    Carver cv{base};
    const size_t N = ctx->N, F = ctx->F, Kp = ctx->Kp, nnz = ctx->nnz;
    d.N = (int)N; d.F = (int)F; d.K = (int)ctx->K; d.Kp = (int)Kp; d.C = ctx->C;
    d.Fi = ctx->Fi; d.Fb = ctx->Fb; d.nnz = (int)nnz;
    d.vol = cv.take<double>(N); d.cx = cv.take<double>(3 * N);
    d.dt = cv.take<double>(N); d.eps2 = cv.take<double>(N);
    d.colour = cv.take<int>(N); d.slot_off = cv.take<int>(N + 1);
    d.slot_face = cv.take<int>(nnz); d.slot_nbr = cv.take<int>(nnz);
    d.slot_left = cv.take<int>(nnz); d.slot_ncol = cv.take<int>(nnz);
    d.slot_n = cv.take<double>(3 * nnz); d.slot_AV = cv.take<double>(nnz);
    d.slot_d = cv.take<double>(3 * nnz); d.slot_lsq = cv.take<double>(3 * nnz);
    d.slot_nT = cv.take<T>(3 * nnz); d.slot_AVT = cv.take<T>(nnz); d.slot_dT = cv.take<T>(3 * nnz);
    d.slot_lsqT = cv.take<T>(3 * nnz); d.slot_sT = cv.take<T>(nnz);
    d.fc = cv.take<int>(2 * F); d.fn = cv.take<double>(3 * F); d.fa = cv.take<double>(F);
    d.fxc = cv.take<double>(3 * F); d.fs = cv.take<double>(F); d.fdl = cv.take<double>(F);
    d.rf = cv.take<double>(F);
    d.fnT = cv.take<T>(3 * F); d.fsT = cv.take<T>(F);
    d.iterp = cv.take<double>(4);
    d.debug = ctx->debug ? 1 : 0;
    d.packed = ctx->use_packed ? 1 : 0;
    d.face_int = cv.take<int>(ctx->Fi + 1); d.face_bnd = cv.take<int>(ctx->Fb + 1);
    d.bcv = cv.take<double>(MAX_BC * 5); d.bck = cv.take<int>(MAX_BC);
    d.u = cv.take<double>(3 * Kp); d.w = cv.take<double>(Kp);
    d.uT = cv.take<T>(3 * Kp); d.wT = cv.take<T>(Kp);
    d.phi = cv.take<T>(2 * N * Kp); d.face = cv.take<T>(2 * F * Kp);
    d.lstore = cv.take<T>(2 * N * Kp);
    d.res = cv.take<T>(2 * N * Kp); d.dphi = cv.take<T>(2 * N * Kp);
    d.W = cv.take<double>(6 * N); d.q = cv.take<double>(6 * N); d.Wold = cv.take<double>(6 * N);
    d.fstate = cv.take<double>(rk::FST * F); d.mface = cv.take<double>(6 * F);
    d.wallq = cv.take<double>(8 * (size_t)(ctx->Fb + 1));
    d.macroF = cv.take<double>(6 * N); d.dW = cv.take<double>(6 * N); d.Wt = cv.take<double>(6 * N);
    d.ceq = cv.take<double>(rk::CEQ * N); d.taut = cv.take<double>(N); d.S = cv.take<double>(12 * N);
    d.cellres = cv.take<double>(12 * N); d.res12 = cv.take<double>(16);
    d.mPc = cv.take<double>(8 * N); d.mDb = cv.take<double>(4 * N); d.mB = cv.take<double>(12 * N);
    d.sG0 = cv.take<double>(6 * nnz); d.sC = cv.take<double>(2 * nnz);
    d.pos_off = cv.take<int>(N + 1); d.cell_pos = cv.take<int>(N);
    d.pslot_nbr = cv.take<int>(nnz); d.pslot_ncol = cv.take<int>(nnz);
    d.pslot_n = cv.take<double>(3 * nnz);
    d.bar = cv.take<unsigned int>(4);
    d.col_off_d = cv.take<int>(ctx->C + 1);
    d.status = cv.take<int>(4);
    int* col_cell = cv.take<int>(N);
    ctx->sched.col_cell = col_cell;
    ctx->stage_a = cv.take<double>(6 * N);
    ctx->stage_b = cv.take<double>(6 * N);
    ctx->surf_out = cv.take<double>(8 * (size_t)(ctx->Fb + 1));
    ctx->surf_contrib = cv.take<double>(4 * (size_t)(ctx->Fb + 1));
    ctx->surf_tot = cv.take<double>(4);
    ctx->aero_contrib = cv.take<double>(6 * (size_t)(ctx->Fb + 1));
    ctx->aero_tot = cv.take<double>(6);
    ctx->wall_b_dev = cv.take<int>(ctx->Fb + 1);
    ctx->dbg = ctx->debug ? (void*)cv.take<T>(2 * N * Kp) : nullptr;
    return cv.off + 256;
}

extern "C" int rk_workspace_size(rk_ctx* ctx, size_t* bytes) {
    if (!ctx || !bytes) return RK_EINVAL;
    if (!ctx->mesh_ok || !ctx->dvs_ok) return fail(ctx, RK_ESTATE, "rk_workspace_size: upload mesh and DVS first");
    *bytes = ctx->prec == RK_FP64 ? carve(ctx, nullptr, ctx->dd) : carve(ctx, nullptr, ctx->df);
    return RK_OK;
}

template <typename T>
static int bind_impl(rk_ctx* ctx, rk::Dev<T>& d) {
    carve(ctx, ctx->ws, d);
    const size_t N = ctx->N, F = ctx->F, Kp = ctx->Kp, nnz = ctx->nnz, K = ctx->K;
    cudaStream_t s = ctx->stream;
    auto h2d = [&](const void* dst, const void* src, size_t bytes) {
        return cudaMemcpyAsync(const_cast<void*>(dst), src, bytes, cudaMemcpyHostToDevice, s);
    };
    // host-side staging in device layouts (kept alive until the stream syncs)
    std::vector<double> cxs(3 * N), fns(3 * F), fxs(3 * F);
    for (size_t i = 0; i < N; ++i)
        for (int r = 0; r < 3; ++r) cxs[r * N + i] = ctx->cx[3 * i + r];
    for (size_t f = 0; f < F; ++f)
        for (int r = 0; r < 3; ++r) { fns[r * F + f] = ctx->fn[3 * f + r]; fxs[r * F + f] = ctx->fx[3 * f + r]; }
    std::vector<double> us(3 * Kp, 0.0), ws(Kp, 0.0);
    std::vector<T> uTs(3 * Kp, T(0)), wTs(Kp, T(0));
    for (size_t k = 0; k < K; ++k) {
        for (int r = 0; r < 3; ++r) { us[r * Kp + k] = ctx->u[3 * k + r]; uTs[r * Kp + k] = (T)ctx->u[3 * k + r]; }
        ws[k] = ctx->w[k];
        wTs[k] = (T)ctx->w[k];
    }
    ctx->wall_b.clear();
    for (int b = 0; b < ctx->Fb; ++b) {
        int bc = -1 - ctx->fc32[2 * (size_t)ctx->face_bnd[b] + 1];
        if (ctx->bck[bc] < 0) return fail(ctx, RK_EINVAL, "rk_bind_workspace: boundary id " + std::to_string(bc) + " has no condition");
        if (ctx->bck[bc] == RK_WALL) ctx->wall_b.push_back(b);
    }
    ctx->nwall = (int)ctx->wall_b.size();
    CK(h2d(d.vol, ctx->cv.data(), N * 8));
    CK(h2d(d.cx, cxs.data(), 3 * N * 8));
    CK(h2d(d.colour, ctx->col.data(), N * 4));
    CK(h2d(d.slot_off, ctx->slot_off.data(), (N + 1) * 4));
    CK(h2d(d.slot_face, ctx->slot_face.data(), nnz * 4));
    CK(h2d(d.slot_nbr, ctx->slot_nbr.data(), nnz * 4));
    CK(h2d(d.slot_left, ctx->slot_left.data(), nnz * 4));
    CK(h2d(d.slot_ncol, ctx->slot_ncol.data(), nnz * 4));
    CK(h2d(d.slot_n, ctx->slot_n.data(), 3 * nnz * 8));
    CK(h2d(d.fc, ctx->fc32.data(), 2 * F * 4));
    CK(h2d(d.fn, fns.data(), 3 * F * 8));
    CK(h2d(d.fa, ctx->fa.data(), F * 8));
    CK(h2d(d.fxc, fxs.data(), 3 * F * 8));
    if (ctx->Fi) CK(h2d(d.face_int, ctx->face_int.data(), ctx->Fi * 4));
    if (ctx->Fb) CK(h2d(d.face_bnd, ctx->face_bnd.data(), ctx->Fb * 4));
    if (ctx->nwall) CK(h2d(ctx->wall_b_dev, ctx->wall_b.data(), ctx->nwall * 4));
    CK(h2d(d.bcv, ctx->bcv, sizeof(ctx->bcv)));
    CK(h2d(d.bck, ctx->bck, sizeof(ctx->bck)));
    CK(h2d(d.u, us.data(), 3 * Kp * 8));
    CK(h2d(d.w, ws.data(), Kp * 8));
    CK(h2d(d.uT, uTs.data(), 3 * Kp * sizeof(T)));
    CK(h2d(d.wT, wTs.data(), Kp * sizeof(T)));
    CK(h2d(ctx->sched.col_cell, ctx->col_cell.data(), N * 4));
    {
        // slots in colour-position order for the macro PR-SGS
        std::vector<int> pos_off(N + 1, 0), cell_pos(N), pnbr(nnz), pncol(nnz);
        std::vector<double> pn(3 * nnz);
        int mp = 0;
        for (size_t p = 0; p < N; ++p) {
            const int i = ctx->col_cell[p];
            cell_pos[i] = (int)p;
            pos_off[p] = mp;
            for (int m = ctx->slot_off[i]; m < ctx->slot_off[i + 1]; ++m, ++mp) {
                pnbr[mp] = ctx->slot_nbr[m];
                pncol[mp] = ctx->slot_ncol[m];
                // outward normal scaled by A_f / (2 V_i): the macro point update's flux
                // coefficient folded into the normal
                const double sg = ctx->slot_left[m] ? 1.0 : -1.0;
                const double c1 = 0.5 * ctx->fa[ctx->slot_face[m]] / ctx->cv[i];
                for (int r = 0; r < 3; ++r) pn[(size_t)r * nnz + mp] = sg * c1 * ctx->slot_n[(size_t)r * nnz + m];
            }
        }
        pos_off[N] = mp;
        CK(h2d(d.pos_off, pos_off.data(), (N + 1) * 4));
        CK(h2d(d.cell_pos, cell_pos.data(), N * 4));
        CK(h2d(d.pslot_nbr, pnbr.data(), nnz * 4));
        CK(h2d(d.pslot_ncol, pncol.data(), nnz * 4));
        CK(h2d(d.pslot_n, pn.data(), 3 * nnz * 8));
        CK(cudaStreamSynchronize(s));
    }
    CK(h2d(d.col_off_d, ctx->col_off.data(), (ctx->C + 1) * 4));
    CK(cudaMemsetAsync(d.bar, 0, 4 * sizeof(unsigned int), s));
    ctx->sched.col_off = ctx->col_off;
    {
        // cooperative macro solve: one co-resident grid of up to 2 blocks per SM
        int dev = 0, sms = 0, coop = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
        const int per = std::min(2, rk::Launch<T>::coop_blocks_per_sm());
        ctx->sched.coop_grid = (coop && per > 0 && ctx->use_coop) ? sms * per : 0;
        // RYKOV_COOP_UNREACHABLE=1 (tests of the bounded wait only): the barriers of the
        // cooperative solve wait for one arrival more than the grid makes, bounded by
        // 50 ms, so the solve returns RK_ETIMEOUT
        const char* ur = std::getenv("RYKOV_COOP_UNREACHABLE");
        const bool unreachable = ur && std::strcmp(ur, "1") == 0;
        ctx->sched.coop_extra = unreachable ? 1u : 0u;
        ctx->sched.coop_limit_ns = unreachable ? 50000000ull : 1000000000ull;
    }
    {
        // staged micro sweeps where their shared memory fits (same results either way)
        int maxs = 0;
        for (int64_t i = 0; i < N; ++i) maxs = std::max(maxs, ctx->slot_off[i + 1] - ctx->slot_off[i]);
        ctx->sched.maxs = maxs;
        ctx->sched.staged = (ctx->use_staged && rk::Launch<T>::micro_staged_smem(maxs) > 0) ? ctx->use_staged : 0;
        ctx->sched.macro32 = (ctx->prec == RK_MIXED && ctx->use_macro32) ? 1 : 0;
        ctx->sched.pdl = ctx->use_pdl ? 1 : 0;
        // RYKOV_MACRO_LANES=1|2|4: threads per cell of the FP32 macro phases, each taking
        // every L-th face (default 4: one face each on tetrahedra)
        if (const char* v = std::getenv("RYKOV_MACRO_LANES")) {
            const int l = std::atoi(v);
            ctx->sched.macro_lanes = (l == 1 || l == 2) ? l : 4;
        }
        cudaGetLastError();
    }
    // zero the distribution-sized arrays once so that the K padding stays 0
    CK(cudaMemsetAsync(d.phi, 0, 2 * N * Kp * sizeof(T), s));
    CK(cudaMemsetAsync(d.face, 0, 2 * F * Kp * sizeof(T), s));
    CK(cudaMemsetAsync(d.res, 0, 2 * N * Kp * sizeof(T), s));
    CK(cudaMemsetAsync(d.dphi, 0, 2 * N * Kp * sizeof(T), s));
    CK(cudaMemsetAsync(d.status, 0, 4 * sizeof(int), s));
    CK(cudaMemsetAsync(d.iterp, 0, 4 * sizeof(double), s));
    if (ctx->gexec) {
        cudaGraphExecDestroy(ctx->gexec);
        ctx->gexec = nullptr;
    }
    CK(cudaMemsetAsync(d.wallq, 0, 8 * (size_t)(ctx->Fb + 1) * 8, s));
    CK(cudaMemsetAsync(d.fstate, 0, rk::FST * F * 8, s));
    cudaError_t e = rk::Launch<T>::setup(d, s);
    if (e != cudaSuccess) return fail(ctx, RK_ECUDA, std::string("setup kernels: ") + cudaGetErrorString(e));
    CK(cudaStreamSynchronize(s));
    ctx->bound = true;
    ctx->have_state = false;
    ctx->bind_gen++;
    return RK_OK;
}

extern "C" int rk_bind_workspace(rk_ctx* ctx, void* dev_ptr, size_t bytes) {
    if (!ctx || !dev_ptr) return RK_EINVAL;
    if (!ctx->mesh_ok || !ctx->dvs_ok) return fail(ctx, RK_ESTATE, "rk_bind_workspace: upload mesh and DVS first");
    size_t need = 0;
    rk_workspace_size(ctx, &need);
    if (bytes < need) return fail(ctx, RK_ENOMEM, "rk_bind_workspace: workspace too small (" + std::to_string(bytes) + " < " + std::to_string(need) + ")");
    if (reinterpret_cast<uintptr_t>(dev_ptr) & 255) return fail(ctx, RK_EINVAL, "rk_bind_workspace: pointer not 256-byte aligned");
    ctx->ws = static_cast<char*>(dev_ptr);
    ctx->ws_bytes = bytes;
    rk_set_params(ctx, &ctx->p);
    return ctx->prec == RK_FP64 ? bind_impl(ctx, ctx->dd) : bind_impl(ctx, ctx->df);
}

static int need_bound(rk_ctx* ctx, const char* who) {
    if (!ctx) return RK_EINVAL;
    if (!ctx->bound) return fail(ctx, RK_ESTATE, std::string(who) + ": bind a workspace first");
    return RK_OK;
}

template <typename T>
static int set_state_prim_impl(rk_ctx* ctx, rk::Dev<T>& d, const double* prim, const double* q, int on_device) {
    const size_t N = ctx->N;
    const double* pd = prim;
    const double* qd = q;
    if (!on_device) {
        CK(cudaMemcpyAsync(ctx->stage_a, prim, 6 * N * 8, cudaMemcpyHostToDevice, ctx->stream));
        pd = ctx->stage_a;
        if (q) {
            CK(cudaMemcpyAsync(ctx->stage_b, q, 6 * N * 8, cudaMemcpyHostToDevice, ctx->stream));
            qd = ctx->stage_b;
        }
    }
    cudaError_t e = rk::Launch<T>::set_state(d, ctx->stream, pd, qd);
    if (e != cudaSuccess) return fail(ctx, RK_ECUDA, cudaGetErrorString(e));
    CK(cudaMemsetAsync(d.iterp, 0, 4 * sizeof(double), ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->iter = 0;
    ctx->have_state = true;
    ctx->state_ver++;
    return RK_OK;
}

extern "C" int rk_set_state_prim(rk_ctx* ctx, const double* prim, const double* q, int on_device) {
    int rc = need_bound(ctx, "rk_set_state_prim");
    if (rc) return rc;
    if (!prim) return fail(ctx, RK_EINVAL, "rk_set_state_prim: null prim");
    if (!on_device) {
        for (int64_t i = 0; i < ctx->N; ++i)
            if (!(prim[6 * i] > 0) || !(prim[6 * i + 4] > 0) || !(prim[6 * i + 5] > 0))
                return fail(ctx, RK_EINVAL, "rk_set_state_prim: non-positive density or temperature");
    }
    return ctx->prec == RK_FP64 ? set_state_prim_impl(ctx, ctx->dd, prim, q, on_device)
                                : set_state_prim_impl(ctx, ctx->df, prim, q, on_device);
}

extern "C" int rk_set_state(rk_ctx* ctx, const double* W, const double* q, const void* dist, int on_device) {
    int rc = need_bound(ctx, "rk_set_state");
    if (rc) return rc;
    if (!W || !dist) return fail(ctx, RK_EINVAL, "rk_set_state: null pointer");
    cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const size_t N = ctx->N, Kp = ctx->Kp;
    double* dW = ctx->prec == RK_FP64 ? ctx->dd.W : ctx->df.W;
    double* dq = ctx->prec == RK_FP64 ? ctx->dd.q : ctx->df.q;
    void* dphi = ctx->prec == RK_FP64 ? (void*)ctx->dd.phi : (void*)ctx->df.phi;
    size_t tsz = ctx->prec == RK_FP64 ? 8 : 4;
    CK(cudaMemcpyAsync(dW, W, 6 * N * 8, kind, ctx->stream));
    if (q) CK(cudaMemcpyAsync(dq, q, 6 * N * 8, kind, ctx->stream));
    else CK(cudaMemsetAsync(dq, 0, 6 * N * 8, ctx->stream));
    CK(cudaMemcpyAsync(dphi, dist, 2 * N * Kp * tsz, kind, ctx->stream));
    CK(cudaMemsetAsync(ctx->prec == RK_FP64 ? (void*)ctx->dd.iterp : (void*)ctx->df.iterp, 0,
                       4 * sizeof(double), ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->iter = 0;
    ctx->have_state = true;
    ctx->state_ver++;
    return RK_OK;
}

extern "C" int rk_get_distribution(rk_ctx* ctx, void* dist, int on_device) {
    int rc = need_bound(ctx, "rk_get_distribution");
    if (rc) return rc;
    const size_t N = ctx->N, Kp = ctx->Kp;
    const void* src = ctx->prec == RK_FP64 ? (const void*)ctx->dd.phi : (const void*)ctx->df.phi;
    size_t tsz = ctx->prec == RK_FP64 ? 8 : 4;
    CK(cudaMemcpyAsync(dist, src, 2 * N * Kp * tsz, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return RK_OK;
}

// one step of the iteration (see RK_STEP_*), launched on stream s
template <typename T>
static cudaError_t launch_step(rk_ctx* ctx, rk::Dev<T>& d, int step, cudaStream_t s) {
    switch (step) {
        case RK_STEP_RECON: return rk::Launch<T>::recon(d, s, ctx->prof);
        case RK_STEP_FACES: return rk::Launch<T>::faces(d, s, ctx->prof);
        case RK_STEP_FLUXES: {
            cudaError_t e = rk::Launch<T>::fluxes(d, s, ctx->prof);
            return e != cudaSuccess ? e : rk::Launch<T>::micro_flux(d, s, ctx->prof);
        }
        case RK_STEP_MACRO: return rk::Launch<T>::macro(d, s, ctx->sched, ctx->p.n_macro_sgs, ctx->prof);
        case RK_STEP_MICRO: return rk::Launch<T>::micro(d, s, ctx->sched, ctx->p.n_micro_sgs, ctx->prof);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T>
static int step_impl(rk_ctx* ctx, rk::Dev<T>& d, int step) {
    if (step < RK_STEP_RECON || step > RK_STEP_MICRO) return fail(ctx, RK_EINVAL, "rk_step: unknown step");
    cudaError_t e = launch_step(ctx, d, step, ctx->stream);
    if (e != cudaSuccess) return fail(ctx, RK_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    if (step == RK_STEP_MICRO) ctx->iter++;
    ctx->state_ver++;
    return RK_OK;
}

// capture one whole iteration into a CUDA graph (on a private stream)
template <typename T>
static int build_graph(rk_ctx* ctx, rk::Dev<T>& d) {
    // the main branch (macro solve, the critical path) is captured on a high-priority
    // stream and the side branch (micro flux, boundary faces) on a low-priority one, and
    // the graph runs with these per-node priorities (RYKOV_PRIO=0: no priorities)
    int plo = 0, phi = 0;
    if (ctx->use_prio) CK(cudaDeviceGetStreamPriorityRange(&plo, &phi));
    if (!ctx->cap) CK(cudaStreamCreateWithPriority(&ctx->cap, cudaStreamNonBlocking, ctx->use_prio ? phi : 0));
    const bool pon = ctx->prof.on;
    const long long l0 = ctx->prof.launches;
    ctx->prof.on = false;
    cudaGraph_t g = nullptr;
    if (!ctx->cap2) CK(cudaStreamCreateWithPriority(&ctx->cap2, cudaStreamNonBlocking, ctx->use_prio ? plo : 0));
    if (!ctx->ev_fork) CK(cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming));
    if (!ctx->ev_join) CK(cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming));
    if (!ctx->ev_bnd) CK(cudaEventCreateWithFlags(&ctx->ev_bnd, cudaEventDisableTiming));
    if (!ctx->ev_int) CK(cudaEventCreateWithFlags(&ctx->ev_int, cudaEventDisableTiming));
    CK(cudaStreamBeginCapture(ctx->cap, cudaStreamCaptureModeThreadLocal));
    // reconstruction and faces; then two branches: the micro flux gather on a second
    // stream while the macro fluxes and the macro PR-SGS (latency-bound, few SMs busy)
    // run on the first; joined before the micro sweeps
    // the boundary faces run beside the interior faces (both only read phi(x_f - u s)
    // of their own faces)
    cudaError_t e = launch_step(ctx, d, RK_STEP_RECON, ctx->cap);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_fork, ctx->cap);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->cap2, ctx->ev_fork, 0);
    if (e == cudaSuccess) e = rk::Launch<T>::faces_boundary(d, ctx->cap2, ctx->prof);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_bnd, ctx->cap2);
    if (e == cudaSuccess) e = rk::Launch<T>::faces_interior(d, ctx->cap, ctx->prof);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_int, ctx->cap);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->cap2, ctx->ev_int, 0);
    if (e == cudaSuccess) e = rk::Launch<T>::micro_flux(d, ctx->cap2, ctx->prof);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_join, ctx->cap2);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->cap, ctx->ev_bnd, 0);
    if (e == cudaSuccess) e = rk::Launch<T>::fluxes(d, ctx->cap, ctx->prof);
    if (e == cudaSuccess) e = launch_step(ctx, d, RK_STEP_MACRO, ctx->cap);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->cap, ctx->ev_join, 0);
    if (e == cudaSuccess) e = launch_step(ctx, d, RK_STEP_MICRO, ctx->cap);
    cudaError_t e2 = cudaStreamEndCapture(ctx->cap, &g);
    ctx->graph_kernels = ctx->prof.launches - l0;
    ctx->prof.launches = l0;
    ctx->prof.on = pon;
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return fail(ctx, RK_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    cudaError_t e3 = cudaGraphInstantiateWithFlags(&ctx->gexec, g,
                                                   ctx->use_prio ? cudaGraphInstantiateFlagUseNodePriority : 0);
    cudaGraphDestroy(g);
    if (e3 != cudaSuccess) {
        ctx->gexec = nullptr;
        return fail(ctx, RK_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e3));
    }
    return RK_OK;
}

// one whole iteration: the captured graph, or direct launches while profiling
template <typename T>
static int iteration(rk_ctx* ctx, rk::Dev<T>& d) {
    if (ctx->use_graph && !ctx->prof.on) {
        if (!ctx->gexec && build_graph(ctx, d) != RK_OK) {
            // capture not available for this sequence: direct launches from now on
            ctx->use_graph = false;
            (void)cudaGetLastError();
        } else {
            CK(cudaGraphLaunch(ctx->gexec, ctx->stream));
            ctx->prof.launches += ctx->graph_kernels;
            ctx->iter++;
            ctx->state_ver++;
            return RK_OK;
        }
    }
    for (int st = RK_STEP_RECON; st <= RK_STEP_MICRO; ++st) {
        int rc = step_impl(ctx, d, st);
        if (rc) return rc;
    }
    return RK_OK;
}

template <typename T>
static int read_residual(rk_ctx* ctx, rk::Dev<T>& d) {
    CK(cudaMemcpyAsync(ctx->pin, d.res12, 6 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(ctx->pin + 8, d.status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (int m = 0; m < 6; ++m) ctx->last_res[m] = ctx->pin[m];
    int status = 0;
    std::memcpy(&status, ctx->pin + 8, sizeof(int));
    if (status & 4) {
        // reported once: the flag is cleared so that the context stays usable
        CK(cudaMemsetAsync(d.status, 0, sizeof(int), ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        return fail(ctx, RK_ETIMEOUT, "macro PR-SGS: a grid barrier wait gave up");
    }
    return RK_OK;
}

template <typename T>
static int iterate_impl(rk_ctx* ctx, rk::Dev<T>& d, int32_t n_iter, double tol, int32_t* done, double* res_out) {
    int32_t it = 0;
    int rc = RK_OK;
    for (; it < n_iter; ++it) {
        if ((rc = iteration(ctx, d))) return rc;
        if (tol > 0.0 || it == n_iter - 1) {
            if ((rc = read_residual(ctx, d))) return rc;
            bool bad = false;
            double mx = 0.0;
            for (int m = 0; m < 6; ++m) {
                if (!std::isfinite(ctx->last_res[m])) bad = true;
                mx = std::max(mx, ctx->last_res[m]);
            }
            if (bad) {
                if (done) *done = it + 1;
                if (res_out) std::memcpy(res_out, ctx->last_res, sizeof(ctx->last_res));
                return fail(ctx, RK_EDIVERGED, "rk_implicit_iterate: non-finite residual");
            }
            if (tol > 0.0 && mx < tol) { ++it; break; }
        }
    }
    if (done) *done = it;
    if (res_out) std::memcpy(res_out, ctx->last_res, sizeof(ctx->last_res));
    return RK_OK;
}

extern "C" int rk_implicit_iterate(rk_ctx* ctx, int32_t n_iter, double tol, int32_t* iters_done, double res_out[6]) {
    int rc = need_bound(ctx, "rk_implicit_iterate");
    if (rc) return rc;
    if (!ctx->have_state) return fail(ctx, RK_ESTATE, "rk_implicit_iterate: set a state first");
    if (n_iter < 0) return fail(ctx, RK_EINVAL, "rk_implicit_iterate: negative count");
    if (n_iter == 0) {
        if (iters_done) *iters_done = 0;
        if (res_out) std::memcpy(res_out, ctx->last_res, sizeof(ctx->last_res));
        return RK_OK;
    }
    return ctx->prec == RK_FP64 ? iterate_impl(ctx, ctx->dd, n_iter, tol, iters_done, res_out)
                                : iterate_impl(ctx, ctx->df, n_iter, tol, iters_done, res_out);
}

extern "C" int rk_step(rk_ctx* ctx, int step) {
    int rc = need_bound(ctx, "rk_step");
    if (rc) return rc;
    if (!ctx->have_state) return fail(ctx, RK_ESTATE, "rk_step: set a state first");
    rc = ctx->prec == RK_FP64 ? step_impl(ctx, ctx->dd, step) : step_impl(ctx, ctx->df, step);
    if (rc) return rc;
    if (step == RK_STEP_MICRO)
        rc = ctx->prec == RK_FP64 ? read_residual(ctx, ctx->dd) : read_residual(ctx, ctx->df);
    else
        CK(cudaStreamSynchronize(ctx->stream));
    return rc;
}

extern "C" int rk_residual(rk_ctx* ctx, double res_out[6]) {
    if (!ctx || !res_out) return RK_EINVAL;
    std::memcpy(res_out, ctx->last_res, sizeof(ctx->last_res));
    return RK_OK;
}

extern "C" int rk_moments(rk_ctx* ctx, double* W, double* q, double* T3, int on_device) {
    int rc = need_bound(ctx, "rk_moments");
    if (rc) return rc;
    const size_t N = ctx->N;
    cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    const double* dW = ctx->prec == RK_FP64 ? ctx->dd.W : ctx->df.W;
    const double* dq = ctx->prec == RK_FP64 ? ctx->dd.q : ctx->df.q;
    if (W) CK(cudaMemcpyAsync(W, dW, 6 * N * 8, kind, ctx->stream));
    if (q) CK(cudaMemcpyAsync(q, dq, 6 * N * 8, kind, ctx->stream));
    if (T3) {
        cudaError_t e = ctx->prec == RK_FP64 ? rk::Launch<double>::temps(ctx->dd, ctx->stream, ctx->stage_a)
                                             : rk::Launch<float>::temps(ctx->df, ctx->stream, ctx->stage_a);
        if (e != cudaSuccess) return fail(ctx, RK_ECUDA, cudaGetErrorString(e));
        CK(cudaMemcpyAsync(T3, ctx->stage_a, 3 * N * 8, kind, ctx->stream));
    }
    CK(cudaStreamSynchronize(ctx->stream));
    return RK_OK;
}

template <typename T>
static int surface_impl(rk_ctx* ctx, rk::Dev<T>& d, double rho_inf, const double* U_inf, double T_inf,
                        double* per, double force[3], double* heat) {
    cudaError_t e = rk::Launch<T>::recon(d, ctx->stream, ctx->prof);
    if (e == cudaSuccess) e = rk::Launch<T>::faces(d, ctx->stream, ctx->prof);
    const double U2 = U_inf[0] * U_inf[0] + U_inf[1] * U_inf[1] + U_inf[2] * U_inf[2];
    const double qd = 0.5 * rho_inf * U2;
    if (e == cudaSuccess)
        e = rk::Launch<T>::surface(d, ctx->stream, ctx->wall_b_dev, ctx->nwall, rho_inf * ctx->p.R * T_inf, qd,
                                   std::sqrt(U2), ctx->surf_out, ctx->surf_contrib, ctx->surf_tot);
    if (e != cudaSuccess) return fail(ctx, RK_ECUDA, cudaGetErrorString(e));
    if (per && ctx->nwall) CK(cudaMemcpyAsync(per, ctx->surf_out, 8 * (size_t)ctx->nwall * 8, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(ctx->pin, ctx->surf_tot, 4 * 8, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (force) { force[0] = ctx->pin[0]; force[1] = ctx->pin[1]; force[2] = ctx->pin[2]; }
    if (heat) *heat = ctx->pin[3];
    return RK_OK;
}

extern "C" int rk_surface(rk_ctx* ctx, double rho_inf, const double* U_inf, double T_inf,
                          double* per_wall_face, double force[3], double* heat) {
    int rc = need_bound(ctx, "rk_surface");
    if (rc) return rc;
    if (!ctx->have_state) return fail(ctx, RK_ESTATE, "rk_surface: set a state first");
    if (!U_inf || !(rho_inf > 0) || !(T_inf > 0)) return fail(ctx, RK_EINVAL, "rk_surface: bad freestream");
    return ctx->prec == RK_FP64 ? surface_impl(ctx, ctx->dd, rho_inf, U_inf, T_inf, per_wall_face, force, heat)
                                : surface_impl(ctx, ctx->df, rho_inf, U_inf, T_inf, per_wall_face, force, heat);
}

template <typename T>
static int aero_impl(rk_ctx* ctx, rk::Dev<T>& d, const double* x_ref, double FM[6]) {
    cudaError_t e = rk::Launch<T>::recon(d, ctx->stream, ctx->prof);
    if (e == cudaSuccess) e = rk::Launch<T>::faces(d, ctx->stream, ctx->prof);
    if (e == cudaSuccess)
        e = rk::Launch<T>::aero(d, ctx->stream, ctx->wall_b_dev, ctx->nwall, x_ref, ctx->aero_contrib, ctx->aero_tot);
    if (e != cudaSuccess) return fail(ctx, RK_ECUDA, cudaGetErrorString(e));
    CK(cudaMemcpyAsync(ctx->pin, ctx->aero_tot, 6 * 8, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (int j = 0; j < 6; ++j) FM[j] = ctx->pin[j];
    return RK_OK;
}

extern "C" int rk_aero(rk_ctx* ctx, double rho_inf, const double* U_inf, const double* x_ref, double S_ref,
                       double L_ref, const double* lift_dir, double out[10]) {
    int rc = need_bound(ctx, "rk_aero");
    if (rc) return rc;
    if (!ctx->have_state) return fail(ctx, RK_ESTATE, "rk_aero: set a state first");
    if (!U_inf || !x_ref || !lift_dir || !out) return fail(ctx, RK_EINVAL, "rk_aero: null pointer");
    const double U2 = U_inf[0] * U_inf[0] + U_inf[1] * U_inf[1] + U_inf[2] * U_inf[2];
    const double q = 0.5 * rho_inf * U2;
    if (!(q > 0) || !(S_ref > 0) || !(L_ref > 0))
        return fail(ctx, RK_EINVAL, "rk_aero: rho_inf, |U_inf|, S_ref and L_ref must be positive");
    const double Um = std::sqrt(U2);
    const double eD[3] = {U_inf[0] / Um, U_inf[1] / Um, U_inf[2] / Um};
    const double a = lift_dir[0] * eD[0] + lift_dir[1] * eD[1] + lift_dir[2] * eD[2];
    double eL[3] = {lift_dir[0] - a * eD[0], lift_dir[1] - a * eD[1], lift_dir[2] - a * eD[2]};
    const double nl = std::sqrt(eL[0] * eL[0] + eL[1] * eL[1] + eL[2] * eL[2]);
    const double n0 = std::sqrt(lift_dir[0] * lift_dir[0] + lift_dir[1] * lift_dir[1] + lift_dir[2] * lift_dir[2]);
    if (!(nl > 1e-12 * n0)) return fail(ctx, RK_EINVAL, "rk_aero: lift direction parallel to U_inf");
    for (int j = 0; j < 3; ++j) eL[j] /= nl;
    const double eP[3] = {eL[1] * eD[2] - eL[2] * eD[1], eL[2] * eD[0] - eL[0] * eD[2],
                          eL[0] * eD[1] - eL[1] * eD[0]};
    double FM[6];
    rc = ctx->prec == RK_FP64 ? aero_impl(ctx, ctx->dd, x_ref, FM) : aero_impl(ctx, ctx->df, x_ref, FM);
    if (rc) return rc;
    for (int j = 0; j < 6; ++j) out[j] = FM[j];
    auto dot = [](const double* x, const double* y) { return x[0] * y[0] + x[1] * y[1] + x[2] * y[2]; };
    out[6] = dot(FM, eD) / (q * S_ref);
    out[7] = dot(FM, eL) / (q * S_ref);
    out[8] = dot(FM + 3, eP) / (q * S_ref * L_ref);
    out[9] = out[7] / out[6];
    return RK_OK;
}

// ---- verification access --------------------------------------------------------
template <typename T>
static int copy_dist(rk_ctx* ctx, const T* src, size_t rows, double* out) {
    const size_t Kp = ctx->Kp, K = ctx->K;
    std::vector<T> tmp(rows * Kp);
    CK(cudaMemcpyAsync(tmp.data(), src, rows * Kp * sizeof(T), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (size_t r = 0; r < rows; ++r)
        for (size_t k = 0; k < K; ++k) out[r * K + k] = (double)tmp[r * Kp + k];
    return RK_OK;
}

template <typename T>
static int debug_impl(rk_ctx* ctx, rk::Dev<T>& d, int which, double* out, int64_t count) {
    const size_t N = ctx->N, F = ctx->F, K = ctx->K;
    auto need = [&](size_t n) { return (int64_t)n <= count; };
    auto d2h = [&](const double* src, size_t n) -> int {
        if (!need(n)) return fail(ctx, RK_EINVAL, "rk_debug_get: output too small");
        CK(cudaMemcpyAsync(out, src, n * 8, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        return RK_OK;
    };
    switch (which) {
        case RK_BUF_PHI: return need(2 * N * K) ? copy_dist(ctx, d.phi, 2 * N, out) : RK_EINVAL;
        case RK_BUF_RES: return need(2 * N * K) ? copy_dist(ctx, d.res, 2 * N, out) : RK_EINVAL;
        case RK_BUF_DPHI: return need(2 * N * K) ? copy_dist(ctx, d.dphi, 2 * N, out) : RK_EINVAL;
        case RK_BUF_FACE: return need(2 * F * K) ? copy_dist(ctx, d.face, 2 * F, out) : RK_EINVAL;
        case RK_BUF_MICRO_F: {
            if (!ctx->dbg) return fail(ctx, RK_ESTATE, "rk_debug_get: context not created with the debug flag");
            if (!need(2 * N * K)) return RK_EINVAL;
            cudaError_t e = rk::Launch<T>::debug_micro_flux(d, ctx->stream, (T*)ctx->dbg);
            if (e != cudaSuccess) return fail(ctx, RK_ECUDA, cudaGetErrorString(e));
            return copy_dist(ctx, (const T*)ctx->dbg, 2 * N, out);
        }
        case RK_BUF_W: return d2h(d.W, 6 * N);
        case RK_BUF_Q: return d2h(d.q, 6 * N);
        case RK_BUF_MACRO_F: return d2h(d.macroF, 6 * N);
        case RK_BUF_WT: return d2h(d.Wt, 6 * N);
        case RK_BUF_FSTATE: return d2h(d.fstate, rk::FST * F);
        case RK_BUF_S: return d2h(d.fs, F);
        case RK_BUF_TAUT: return d2h(d.taut, N);
        case RK_BUF_DT: {
            if (!need(3 * N)) return RK_EINVAL;
            std::vector<double> dt(N), e2(N);
            CK(cudaMemcpyAsync(dt.data(), d.dt, N * 8, cudaMemcpyDeviceToHost, ctx->stream));
            CK(cudaMemcpyAsync(e2.data(), d.eps2, N * 8, cudaMemcpyDeviceToHost, ctx->stream));
            CK(cudaStreamSynchronize(ctx->stream));
            const double cfl = implicit_cfl(ctx->p, ctx->iter);
            for (size_t i = 0; i < N; ++i) { out[3 * i] = dt[i]; out[3 * i + 1] = cfl * dt[i]; out[3 * i + 2] = e2[i]; }
            return RK_OK;
        }
        default: return fail(ctx, RK_EINVAL, "rk_debug_get: unknown buffer");
    }
}

template <typename T>
static int debug_rows_impl(rk_ctx* ctx, rk::Dev<T>& d, int which, const int64_t* rows, int64_t n, double* out) {
    const size_t N = ctx->N, F = ctx->F, K = ctx->K, Kp = ctx->Kp;
    const T* src = nullptr;
    size_t nrows = N;
    switch (which) {
        case RK_BUF_PHI: src = d.phi; break;
        case RK_BUF_RES: src = d.res; break;
        case RK_BUF_DPHI: src = d.dphi; break;
        case RK_BUF_FACE: src = d.face; nrows = F; break;
        case RK_BUF_MICRO_F: {
            if (!ctx->dbg) return fail(ctx, RK_ESTATE, "rk_debug_rows: context not created with the debug flag");
            cudaError_t e = rk::Launch<T>::debug_micro_flux(d, ctx->stream, (T*)ctx->dbg);
            if (e != cudaSuccess) return fail(ctx, RK_ECUDA, cudaGetErrorString(e));
            src = (const T*)ctx->dbg;
            break;
        }
        default: return fail(ctx, RK_EINVAL, "rk_debug_rows: unsupported buffer");
    }
    for (int64_t r = 0; r < n; ++r)
        if (rows[r] < 0 || (size_t)rows[r] >= nrows) return fail(ctx, RK_EINVAL, "rk_debug_rows: row out of range");
    std::vector<T> tmp(2 * (size_t)n * Kp);
    for (int fd = 0; fd < 2; ++fd)
        for (int64_t r = 0; r < n; ++r)
            CK(cudaMemcpyAsync(tmp.data() + ((size_t)fd * n + r) * Kp, src + ((size_t)fd * nrows + rows[r]) * Kp,
                               Kp * sizeof(T), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (size_t q = 0; q < 2 * (size_t)n; ++q)
        for (size_t k = 0; k < K; ++k) out[q * K + k] = (double)tmp[q * Kp + k];
    return RK_OK;
}

extern "C" int rk_debug_rows(rk_ctx* ctx, int which, const int64_t* rows, int64_t n_rows, double* host_out) {
    int rc = need_bound(ctx, "rk_debug_rows");
    if (rc) return rc;
    if (!host_out || !rows || n_rows < 0) return fail(ctx, RK_EINVAL, "rk_debug_rows: bad arguments");
    return ctx->prec == RK_FP64 ? debug_rows_impl(ctx, ctx->dd, which, rows, n_rows, host_out)
                                : debug_rows_impl(ctx, ctx->df, which, rows, n_rows, host_out);
}

extern "C" int rk_debug_get(rk_ctx* ctx, int which, double* host_out, int64_t count) {
    int rc = need_bound(ctx, "rk_debug_get");
    if (rc) return rc;
    if (!host_out) return fail(ctx, RK_EINVAL, "rk_debug_get: null output");
    return ctx->prec == RK_FP64 ? debug_impl(ctx, ctx->dd, which, host_out, count)
                                : debug_impl(ctx, ctx->df, which, host_out, count);
}

extern "C" int rk_profile(rk_ctx* ctx, int enable) {
    if (!ctx) return RK_EINVAL;
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->prof.on = enable != 0;
    ctx->prof.used = 0;
    ctx->prof.cls.clear();
    return RK_OK;
}

extern "C" int rk_profile_get(rk_ctx* ctx, double* ms, int64_t* counts) {
    if (!ctx || !ms || !counts) return RK_EINVAL;
    CK(cudaStreamSynchronize(ctx->stream));
    for (int c = 0; c < RK_PROF_N; ++c) { ms[c] = 0.0; counts[c] = 0; }
    for (size_t p = 0; p < ctx->prof.cls.size(); ++p) {
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, ctx->prof.ev[2 * p], ctx->prof.ev[2 * p + 1]));
        ms[ctx->prof.cls[p]] += t;
        counts[ctx->prof.cls[p]] += 1;
    }
    counts[RK_PROF_N] = ctx->prof.launches;
    return RK_OK;
}
