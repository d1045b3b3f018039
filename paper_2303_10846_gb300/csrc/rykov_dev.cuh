// Device side of librykov: kernels of one implicit iteration (Sec. 3.5, Steps 2-6)
// of the conservative implicit Rykov scheme, templated on the storage/arithmetic
// type T of the per-velocity work (double: FP64 mode; float: mixed mode, where the
// reductions over the discrete velocity space use compensated FP32 accumulation
// combined in FP64, and everything per cell or per face stays FP64).
//
// Layout in HBM (k fastest, K padded to a multiple of 32):
//   phi, res, dphi : T[2][N][Kp]      face : T[2][F][Kp] (phi(x_ij - u s), then phi_ij)
// Per-cell and per-face scalars are FP64 arrays of structs ([N][6], [F][16], ...).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace rk {

constexpr int MAXF = 8;        // faces per cell
constexpr int EQN = 24;        // constants of one Rykov equilibrium (see make_eq)
constexpr int CEQ = 28;        // per-cell record: EQN constants, 1/tau~, diagonal base
constexpr int FST = 16;        // face state record
constexpr double PI = 3.14159265358979323846;

template <typename T>
struct Dev {
    int N, F, K, Kp, C, Fi, Fb, nnz;
    // gas / scheme parameters
    double R, Z, omega_vis, mu_ref, T_ref, omega0, omega1, delta, cfl_s, lim_k;
    // cells
    const double *vol, *cx;            // [N], [3][N]
    double *dt, *eps2;                 // [N]
    const int *colour, *slot_off;      // [N], [N+1]
    // slots (cell -> face incidences, CSR in increasing face order)
    const int *slot_face, *slot_nbr, *slot_left, *slot_ncol;
    const double *slot_n;              // face normal as given (from left to right) [3][nnz]
    double *slot_AV;                   // A_f / V_i  [nnz]
    double *slot_d;                    // x_f - x_i  [3][nnz]
    double *slot_lsq;                  // LSQ weight vector M_i^{-1}(x_j - x_i), 0 at boundaries [3][nnz]
    T *slot_nT, *slot_AVT, *slot_dT, *slot_lsqT, *slot_sT;
    // faces
    const int* fc;                     // [F][2]
    const double *fn, *fa, *fxc;       // [3][F], [F], [3][F]
    double *fs, *fdl, *rf;             // s_ij, distance used in r_ij, r_ij  [F]
    const int *face_int, *face_bnd;    // lists
    const double* bcv;                 // [64][5]: rho, U, T
    const int* bck;                    // [64] kind
    // discrete velocity space (SoA, padded with zero weights)
    const double *u, *w;               // [3][Kp], [Kp]
    const T *uT, *wT;
    // state
    T *phi, *face, *res, *dphi;
    double *W, *q, *Wold, *fstate, *mface, *wallq, *macroF, *dW, *Wt, *ceq, *taut, *S,
        *cellres, *res12;
    // macro PR-SGS work: flux primitives (rho, U, rho E + p, p, rho E_rot) of the
    // current iterate per cell, diagonal base per cell, per-slot Euler flux of the
    // neighbour's W^n and the coefficients A/(2V), A r/(2V)
    double *mPc, *mDb, *sG0, *sC;        // mDb: [N][4] = 1/D, 1/(D + 1/(Z tau)), 1/(Z tau)
    int* status;
};

// ------------------------------------------------------------------------------------
// small helpers
// ------------------------------------------------------------------------------------
// u.n with every product and sum rounded separately: the upwind decisions
// (u.n > 0) must be taken on exactly the same value as the CPU oracle's.
__device__ __forceinline__ double dot_rn(double ax, double ay, double az, double bx, double by,
                                         double bz) {
    return __dadd_rn(__dadd_rn(__dmul_rn(ax, bx), __dmul_rn(ay, by)), __dmul_rn(az, bz));
}
__device__ __forceinline__ float dot_rn(float ax, float ay, float az, float bx, float by, float bz) {
    return __fadd_rn(__fadd_rn(__fmul_rn(ax, bx), __fmul_rn(ay, by)), __fmul_rn(az, bz));
}
// u.n for the split of the micro operator into diagonal (u.n > 0) and neighbour
// (u.n < 0) parts: exact-rounded in FP64 (same split as the oracle), contracted in FP32
__device__ __forceinline__ double dot_split(double ax, double ay, double az, double bx, double by,
                                            double bz) {
    return dot_rn(ax, ay, az, bx, by, bz);
}
__device__ __forceinline__ float dot_split(float ax, float ay, float az, float bx, float by, float bz) {
    return fmaf(az, bz, fmaf(ay, by, ax * bx));
}
__device__ __forceinline__ double ex(double x) { return exp(x); }
__device__ __forceinline__ float ex(float x) { return expf(x); }

// Accumulators for sums over the velocity space.  FP64 mode: plain FP64 sum.  Mixed
// mode: Kahan-compensated FP32 sum (every operation rounded as written), combined in
// FP64: s - c carries the running sum and its lost low-order part.
template <typename T>
struct Acc;
template <>
struct Acc<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double x) { s += x; }
    __device__ __forceinline__ double get() const { return s; }
};
template <>
struct Acc<float> {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x) {
        const float y = __fsub_rn(x, c);
        const float t = __fadd_rn(s, y);
        c = __fsub_rn(__fsub_rn(t, s), y);
        s = t;
    }
    __device__ __forceinline__ double get() const { return (double)s - (double)c; }
};

// Values carried by the cross-lane reductions: FP64 mode reduces doubles; mixed mode
// reduces float-float pairs (hi + lo, two-sum arithmetic, ~44 significant bits), so
// that no FP64 instruction is spent per lane (GB300 issues FP64 at 1/64 of the FP32
// rate).  The two-sum of (a, b) and (b, a) gives the same bits, so butterfly results
// are identical on every lane.
struct FF {
    float hi, lo;
};
__device__ __forceinline__ FF ff_norm(float s, float e) {
    const float hi = __fadd_rn(s, e);
    return FF{hi, __fsub_rn(e, __fsub_rn(hi, s))};
}
__device__ __forceinline__ FF ff_add(FF a, FF b) {
    const float s = __fadd_rn(a.hi, b.hi);
    const float bb = __fsub_rn(s, a.hi);
    float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    return ff_norm(s, e);
}
template <typename T>
struct Red;
template <>
struct Red<double> {
    using V = double;
    static __device__ __forceinline__ V from(const Acc<double>& a) { return a.s; }
    static __device__ __forceinline__ V zero() { return 0.0; }
    static __device__ __forceinline__ V add(V a, V b) { return a + b; }
    static __device__ __forceinline__ V shfl_xor(V v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
    static __device__ __forceinline__ double to_d(V v) { return v; }
};
template <>
struct Red<float> {
    using V = FF;
    static __device__ __forceinline__ V from(const Acc<float>& a) { return ff_norm(a.s, -a.c); }
    static __device__ __forceinline__ V zero() { return FF{0.f, 0.f}; }
    static __device__ __forceinline__ V add(V a, V b) { return ff_add(a, b); }
    static __device__ __forceinline__ V shfl_xor(V v, int o) {
        return FF{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
    }
    static __device__ __forceinline__ double to_d(V v) { return (double)v.hi + (double)v.lo; }
};

template <typename T, int NV>
__device__ __forceinline__ void warp_red(typename Red<T>::V (&v)[NV]) {
#pragma unroll
    for (int j = 0; j < NV; ++j) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[j] = Red<T>::add(v[j], Red<T>::shfl_xor(v[j], o));
    }
}

// Block reduction of NV values: warp butterflies, then the warps in order on thread
// 0; every thread receives the totals as doubles.  smem: NV * (BS/32) values + NV doubles.
template <typename T, int NV, int BS>
__device__ __forceinline__ void block_red(typename Red<T>::V (&v)[NV], typename Red<T>::V* sm,
                                          double* out) {
    using R = Red<T>;
    constexpr int NW = BS / 32;
    warp_red<T, NV>(v);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) {
#pragma unroll
        for (int j = 0; j < NV; ++j) sm[j * NW + warp] = v[j];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int j = 0; j < NV; ++j) {
            typename R::V t = sm[j * NW];
            for (int q = 1; q < NW; ++q) t = R::add(t, sm[j * NW + q]);
            out[j] = R::to_d(t);
        }
    }
    __syncthreads();
}

// Butterfly sum over the 32 lanes of a warp (every lane ends with the same bits).
template <int NV>
__device__ __forceinline__ void warp_sum(double (&v)[NV]) {
#pragma unroll
    for (int j = 0; j < NV; ++j) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[j] += __shfl_xor_sync(0xffffffffu, v[j], o);
    }
}

// Deterministic block sum of NV doubles (fixed shuffle tree, then warps in order).
// Every thread receives the totals in v.  smem must hold NV * (BS/32) doubles.
template <int NV, int BS>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* smem) {
    constexpr int NW = BS / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < NV; ++j) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[j] += __shfl_down_sync(0xffffffffu, v[j], o);
    }
    __syncthreads();
    if (lane == 0) {
#pragma unroll
        for (int j = 0; j < NV; ++j) smem[j * NW + warp] = v[j];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            double t = smem[j * NW];
            for (int q = 1; q < NW; ++q) t += smem[j * NW + q];
            smem[j * NW] = t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < NV; ++j) v[j] = smem[j * NW];
    __syncthreads();
}

// ------------------------------------------------------------------------------------
// gas model
// ------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ double viscosity(const Dev<T>& c, double Ttr) {
    return c.mu_ref * pow(Ttr / c.T_ref, c.omega_vis);                 // Eq. T_solve_mu
}
template <typename T>
__device__ __forceinline__ double relax_time(const Dev<T>& c, double rho, double Ttr) {
    return viscosity(c, Ttr) / (rho * c.R * Ttr);                     // tau = mu / p_tr
}

struct Prim {
    double rho, U[3], T, Ttr, Trot;
};
// W -> primitives with K_tr = 3, K_rot = 2 (Eqs. f_solve_Energy - f_solve_EnergyRot).
__device__ __forceinline__ Prim prim_from_W(const double* W, double R) {
    Prim p;
    p.rho = W[0];
    p.U[0] = W[1] / p.rho; p.U[1] = W[2] / p.rho; p.U[2] = W[3] / p.rho;
    double ke = 0.5 * p.rho * (p.U[0] * p.U[0] + p.U[1] * p.U[1] + p.U[2] * p.U[2]);
    p.T = (W[4] - ke) / (2.5 * p.rho * R);
    p.Trot = W[5] / (p.rho * R);
    p.Ttr = (W[4] - ke - W[5]) / (1.5 * p.rho * R);
    return p;
}

// Constants of the Rykov reduced equilibria G*, R* (Eqs. eqdf_G* - eqdf_Rrot) for a
// state (rho, U, T, T_tr, T_rot, q_tr, q_rot), p = rho R T, p_tr = rho R T_tr,
// p_rot = rho R T_rot:
//  0-2 U  3-5 q_tr  6-8 q_rot  9 rho (2 pi R T_tr)^-1.5  10 1/(2 R T_tr)
//  11 1/(15 R T_tr p_tr)  12 1/(R T_tr)  13 rho (2 pi R T)^-1.5  14 1/(2 R T)
//  15 omega0/(15 R T p)  16 1/(R T)  17 R T_rot  18 R T  19 (1-delta)/(R T_tr p_rot)
//  20 omega1 (1-delta)/(R T p)  21 1 - 1/Z  22 1/Z
template <typename T, typename S>
__device__ void make_eq(const Dev<T>& c, S rho, const S* U, S Tq, S Ttr, S Trot, const S* qtr,
                        const S* qrot, S* e) {
    const S R = (S)c.R;
    const S RTtr = R * Ttr, RT = R * Tq, RTrot = R * Trot;
    const S ptr = rho * RTtr, p = rho * RT, prot = rho * RTrot;
    for (int d = 0; d < 3; ++d) { e[d] = U[d]; e[3 + d] = qtr[d]; e[6 + d] = qrot[d]; }
    const S a = S(2.0 * PI) * RTtr;
    e[9] = rho / (a * sqrt(a));
    e[10] = S(1) / (S(2) * RTtr);
    e[11] = S(1) / (S(15) * RTtr * ptr);
    e[12] = S(1) / RTtr;
    const S b = S(2.0 * PI) * RT;
    e[13] = rho / (b * sqrt(b));
    e[14] = S(1) / (S(2) * RT);
    e[15] = (S)c.omega0 / (S(15) * RT * p);
    e[16] = S(1) / RT;
    e[17] = RTrot;
    e[18] = RT;
    e[19] = (S(1) - (S)c.delta) / (RTtr * prot);
    e[20] = (S)c.omega1 * (S(1) - (S)c.delta) / (RT * p);
    e[21] = S(1) - S(1) / (S)c.Z;
    e[22] = S(1) / (S)c.Z;
}

template <typename T>
__device__ __forceinline__ void eval_eq(const T* e, T ux, T uy, T uz, T& G, T& H) {
    T cx = ux - e[0], cy = uy - e[1], cz = uz - e[2];
    T c2 = cx * cx + cy * cy + cz * cz;
    T cqt = cx * e[3] + cy * e[4] + cz * e[5];
    T cqr = cx * e[6] + cy * e[7] + cz * e[8];
    T mtr = e[9] * ex(-c2 * e[10]);
    T m = e[13] * ex(-c2 * e[14]);
    T Gtr = mtr * (T(1) + cqt * e[11] * (c2 * e[12] - T(5)));
    T Grot = m * (T(1) + cqt * e[15] * (c2 * e[16] - T(5)));
    T Htr = e[17] * (Gtr + e[19] * cqr * mtr);
    T Hrot = e[18] * (Grot + e[20] * cqr * m);
    G = e[21] * Gtr + e[22] * Grot;
    H = e[21] * Htr + e[22] * Hrot;
}

template <typename T>
__device__ __forceinline__ T maxwell(const T* mc, T ux, T uy, T uz) {
    // mc: U[3], rho (2 pi R T)^-1.5, 1/(2 R T)
    T cx = ux - mc[0], cy = uy - mc[1], cz = uz - mc[2];
    return mc[3] * ex(-(cx * cx + cy * cy + cz * cz) * mc[4]);
}

__device__ __forceinline__ double venkat(double d1, double d2, double eps2) {
    if (d2 == 0.0) return 1.0;
    return (d1 * d1 + eps2 + 2.0 * d1 * d2) / (d1 * d1 + 2.0 * d2 * d2 + d1 * d2 + eps2);
}
__device__ __forceinline__ float venkat(float d1, float d2, float eps2) {
    if (d2 == 0.f) return 1.f;
    return (d1 * d1 + eps2 + 2.f * d1 * d2) / (d1 * d1 + 2.f * d2 * d2 + d1 * d2 + eps2);
}

// ------------------------------------------------------------------------------------
// set-up kernels (once per bind / parameter change)
// ------------------------------------------------------------------------------------
// CFL step Delta t_i = cfl_s V_i / max_k sum_f A_f max(u_k . n_f,out, 0) and the
// Venkatakrishnan eps^2 = (K V^{1/3})^3.  One block per cell.
template <typename T>
__global__ void k_setup_dt(Dev<T> c) {
    __shared__ double red[8];
    const int i = blockIdx.x;
    const int s0 = c.slot_off[i], s1 = c.slot_off[i + 1];
    double vmax = 0.0;
    for (int k = threadIdx.x; k < c.K; k += blockDim.x) {
        double ux = c.u[k], uy = c.u[c.Kp + k], uz = c.u[2 * c.Kp + k];
        double sum = 0.0;
        for (int m = s0; m < s1; ++m) {
            const int f = c.slot_face[m];
            double un = dot_rn(ux, uy, uz, c.fn[f], c.fn[c.F + f], c.fn[2 * c.F + f]);
            if (!c.slot_left[m]) un = -un;
            if (un > 0.0) sum += c.fa[f] * un;
        }
        vmax = fmax(vmax, sum);
    }
    for (int o = 16; o > 0; o >>= 1) vmax = fmax(vmax, __shfl_down_sync(0xffffffffu, vmax, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = vmax;
    __syncthreads();
    if (threadIdx.x == 0) {
        double v = red[0];
        for (int q = 1; q < (int)(blockDim.x >> 5); ++q) v = fmax(v, red[q]);
        c.dt[i] = c.cfl_s * c.vol[i] / v;
        double h = cbrt(c.vol[i]) * c.lim_k;
        c.eps2[i] = h * h * h;
    }
}

// Least-squares weights: M_i = sum_m d_m d_m^T over face neighbours (d = x_j - x_i)
// and boundary face centroids (d = x_f - x_i, the reading for boundaries: a
// pseudo-neighbour holding the cell's own value, so it only enters M_i);
// weight of neighbour m = M_i^{-1} d_m.  Also x_f - x_i and A/V per slot.
template <typename T>
__global__ void k_setup_lsq(Dev<T> c) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= c.N) return;
    const int s0 = c.slot_off[i], s1 = c.slot_off[i + 1];
    const double xi = c.cx[i], yi = c.cx[c.N + i], zi = c.cx[2 * c.N + i];
    double M[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int m = s0; m < s1; ++m) {
        const int f = c.slot_face[m], j = c.slot_nbr[m];
        double d[3];
        if (j >= 0) { d[0] = c.cx[j] - xi; d[1] = c.cx[c.N + j] - yi; d[2] = c.cx[2 * c.N + j] - zi; }
        else { d[0] = c.fxc[f] - xi; d[1] = c.fxc[c.F + f] - yi; d[2] = c.fxc[2 * c.F + f] - zi; }
        for (int r = 0; r < 3; ++r)
            for (int s = 0; s < 3; ++s) M[3 * r + s] += d[r] * d[s];
        c.slot_d[m] = c.fxc[f] - xi;
        c.slot_d[c.nnz + m] = c.fxc[c.F + f] - yi;
        c.slot_d[2 * c.nnz + m] = c.fxc[2 * c.F + f] - zi;
        c.slot_AV[m] = c.fa[f] / c.vol[i];
    }
    double A = M[4] * M[8] - M[5] * M[7], B = M[5] * M[6] - M[3] * M[8], Cc = M[3] * M[7] - M[4] * M[6];
    double det = M[0] * A + M[1] * B + M[2] * Cc;
    double Mi[9] = {A / det, (M[2] * M[7] - M[1] * M[8]) / det, (M[1] * M[5] - M[2] * M[4]) / det,
                    B / det, (M[0] * M[8] - M[2] * M[6]) / det, (M[2] * M[3] - M[0] * M[5]) / det,
                    Cc / det, (M[1] * M[6] - M[0] * M[7]) / det, (M[0] * M[4] - M[1] * M[3]) / det};
    for (int m = s0; m < s1; ++m) {
        const int j = c.slot_nbr[m];
        double d[3] = {0.0, 0.0, 0.0};
        if (j >= 0) { d[0] = c.cx[j] - xi; d[1] = c.cx[c.N + j] - yi; d[2] = c.cx[2 * c.N + j] - zi; }
        for (int r = 0; r < 3; ++r)
            c.slot_lsq[r * c.nnz + m] = Mi[3 * r] * d[0] + Mi[3 * r + 1] * d[1] + Mi[3 * r + 2] * d[2];
    }
}

// s_ij = min(Delta t_i, Delta t_j) (Delta t_i at boundary faces) and the distance
// Delta l_ij of the spectral radius (2 |x_f - x_i| at boundary faces).
template <typename T>
__global__ void k_setup_face(Dev<T> c) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= c.F) return;
    const int a = c.fc[2 * f], b = c.fc[2 * f + 1];
    c.fs[f] = (b >= 0) ? fmin(c.dt[a], c.dt[b]) : c.dt[a];
    double dx, dy, dz, sc = 1.0;
    if (b >= 0) { dx = c.cx[b] - c.cx[a]; dy = c.cx[c.N + b] - c.cx[c.N + a]; dz = c.cx[2 * c.N + b] - c.cx[2 * c.N + a]; }
    else { dx = c.fxc[f] - c.cx[a]; dy = c.fxc[c.F + f] - c.cx[c.N + a]; dz = c.fxc[2 * c.F + f] - c.cx[2 * c.N + a]; sc = 2.0; }
    c.fdl[f] = sc * sqrt(dx * dx + dy * dy + dz * dz);
}

// copies of the slot geometry in the per-velocity arithmetic type
template <typename T>
__global__ void k_setup_slotT(Dev<T> c) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= c.nnz) return;
    c.slot_AVT[m] = (T)c.slot_AV[m];
    c.slot_sT[m] = (T)c.fs[c.slot_face[m]];
    for (int r = 0; r < 3; ++r) {
        c.slot_nT[r * c.nnz + m] = (T)c.slot_n[r * c.nnz + m];
        c.slot_dT[r * c.nnz + m] = (T)c.slot_d[r * c.nnz + m];
        c.slot_lsqT[r * c.nnz + m] = (T)c.slot_lsq[r * c.nnz + m];
    }
}

// Step 1: W from primitives, q, and the equilibrium distributions.
template <typename T>
__global__ void k_set_state(Dev<T> c, const double* prim, const double* qin) {
    __shared__ double e[EQN];
    __shared__ T eT[EQN];
    const int i = blockIdx.x;
    if (threadIdx.x == 0) {
        const double* pr = prim + 6 * (size_t)i;
        double rho = pr[0], U[3] = {pr[1], pr[2], pr[3]}, Ttr = pr[4], Trot = pr[5];
        double* W = c.W + 6 * (size_t)i;
        W[0] = rho;
        for (int d = 0; d < 3; ++d) W[1 + d] = rho * U[d];
        W[4] = 0.5 * rho * (U[0] * U[0] + U[1] * U[1] + U[2] * U[2]) + 1.5 * rho * c.R * Ttr + rho * c.R * Trot;
        W[5] = rho * c.R * Trot;
        double* q = c.q + 6 * (size_t)i;
        for (int d = 0; d < 6; ++d) q[d] = qin ? qin[6 * (size_t)i + d] : 0.0;
        Prim p = prim_from_W(W, c.R);
        make_eq(c, p.rho, p.U, p.T, p.Ttr, p.Trot, q, q + 3, e);
        e[EQN - 1] = 0.0;
        for (int d = 0; d < EQN; ++d) eT[d] = (T)e[d];
    }
    __syncthreads();
    T* g = c.phi + (size_t)i * c.Kp;
    T* h = c.phi + ((size_t)c.N + i) * c.Kp;
    for (int k = threadIdx.x; k < c.Kp; k += blockDim.x) {
        T G = T(0), H = T(0);
        if (k < c.K) eval_eq(eT, c.uT[k], c.uT[c.Kp + k], c.uT[2 * c.Kp + k], G, H);
        g[k] = G;
        h[k] = H;
    }
}

// ------------------------------------------------------------------------------------
// Step 2 (a): least-squares gradient, Venkatakrishnan limiter and reconstruction
// phi(x_ij - u_k s_ij) = phi_c + (x_ij - u_k s_ij - x_c) . L grad phi_c, written by
// the upwind cell c into the face array (Eq. flux_solve_phi_phi).  One block per
// cell, velocities strided over the block; the cell's face data staged in shared
// memory.
// ------------------------------------------------------------------------------------
template <typename T, int BS>
__global__ void __launch_bounds__(BS, 6) k_recon(Dev<T> c, int limiter) {
    __shared__ int s_face[MAXF], s_nbr[MAXF], s_left[MAXF];
    __shared__ T s_lsq[3][MAXF], s_d[3][MAXF], s_n[3][MAXF], s_s[MAXF];
    const int i = blockIdx.x;
    const int s0 = c.slot_off[i], ns = c.slot_off[i + 1] - s0;
    if (threadIdx.x < ns) {
        const int m = s0 + threadIdx.x, q = threadIdx.x;
        s_face[q] = c.slot_face[m];
        s_nbr[q] = c.slot_nbr[m];
        s_left[q] = c.slot_left[m];
        s_s[q] = c.slot_sT[m];
        for (int r = 0; r < 3; ++r) {
            s_lsq[r][q] = c.slot_lsqT[r * c.nnz + m];
            s_d[r][q] = c.slot_dT[r * c.nnz + m];
            s_n[r][q] = c.slot_nT[r * c.nnz + m];
        }
    }
    __syncthreads();
    const T eps2 = (T)c.eps2[i];
    const size_t NK = (size_t)c.N * c.Kp, FK = (size_t)c.F * c.Kp;
    const T* phg = c.phi + (size_t)i * c.Kp;
    const T* phh = c.phi + NK + (size_t)i * c.Kp;
    for (int k = threadIdx.x; k < c.K; k += BS) {
        const T pg = phg[k], ph = phh[k];
        T g[2][3] = {{T(0), T(0), T(0)}, {T(0), T(0), T(0)}};
        T dmax[2] = {T(0), T(0)}, dmin[2] = {T(0), T(0)};
#pragma unroll 1
        for (int q = 0; q < ns; ++q) {
            const int j = s_nbr[q];
            if (j < 0) continue;
            const T dg = c.phi[(size_t)j * c.Kp + k] - pg;
            const T dh = c.phi[NK + (size_t)j * c.Kp + k] - ph;
            const T lx = s_lsq[0][q], ly = s_lsq[1][q], lz = s_lsq[2][q];
            g[0][0] += lx * dg; g[0][1] += ly * dg; g[0][2] += lz * dg;
            g[1][0] += lx * dh; g[1][1] += ly * dh; g[1][2] += lz * dh;
            dmax[0] = dg > dmax[0] ? dg : dmax[0]; dmin[0] = dg < dmin[0] ? dg : dmin[0];
            dmax[1] = dh > dmax[1] ? dh : dmax[1]; dmin[1] = dh < dmin[1] ? dh : dmin[1];
        }
        T L[2] = {T(1), T(1)};
        if (limiter == 2) {
            L[0] = L[1] = T(0);
        } else if (limiter == 1) {
            // min over faces of Venkatakrishnan's psi = num/den, kept as a fraction
            // (den > 0) so that only the minimum is divided; capped at 1 (reading)
            T bn[2] = {T(1), T(1)}, bd[2] = {T(1), T(1)};
#pragma unroll 1
            for (int q = 0; q < ns; ++q) {
                const T dx = s_d[0][q], dy = s_d[1][q], dz = s_d[2][q];
#pragma unroll
                for (int fd = 0; fd < 2; ++fd) {
                    const T d2 = g[fd][0] * dx + g[fd][1] * dy + g[fd][2] * dz;
                    if (d2 == T(0)) continue;
                    const T d1 = d2 > T(0) ? dmax[fd] : dmin[fd];
                    const T num = d1 * d1 + eps2 + T(2) * d1 * d2;
                    const T den = d1 * d1 + T(2) * d2 * d2 + d1 * d2 + eps2;
                    if (num * bd[fd] < bn[fd] * den) { bn[fd] = num; bd[fd] = den; }
                }
            }
            L[0] = bn[0] / bd[0];
            L[1] = bn[1] / bd[1];
        }
        const T ux = c.uT[k], uy = c.uT[c.Kp + k], uz = c.uT[2 * c.Kp + k];
#pragma unroll 1
        for (int q = 0; q < ns; ++q) {
            const T un = dot_rn(ux, uy, uz, s_n[0][q], s_n[1][q], s_n[2][q]);
            const bool up = s_left[q] ? (un > T(0)) : (un <= T(0));
            if (!up) continue;
            const T sq = s_s[q];
            const T rx = s_d[0][q] - ux * sq, ry = s_d[1][q] - uy * sq, rz = s_d[2][q] - uz * sq;
            const size_t o = (size_t)s_face[q] * c.Kp + k;
            c.face[o] = pg + L[0] * (g[0][0] * rx + g[0][1] * ry + g[0][2] * rz);
            c.face[FK + o] = ph + L[1] * (g[1][0] * rx + g[1][1] * ry + g[1][2] * rz);
        }
    }
}

// ------------------------------------------------------------------------------------
// Step 2 (b)-(d) at interior faces: one warp per face.
//   pass 1: the 17 raw moments of phi(x_ij - u s) about a reference velocity U_r
//           (mean of the two cells' U^n): sum w g, w g c', w h, w g c'c' (6),
//           w g |c'|^2 c', w h c'.  They give rho, rho U, rho E (Eqs.
//           halftime_solve_rho/U/E) and, shifted to the interface velocity
//           U = U_r + d, the heat-flux sums of Eqs. halftime_solve_qtra/qrot without
//           cancellation at high speed.
//   state : tau, rho E_rot (Eq. halftime_solve_Erot), q_tr, q_rot
//   pass 2: phi* and phi_ij = (tau phi0 + s phi*)/(tau + s) in place (Eq.
//           flux_solve_phi) and the DVS quadrature of the macro flux (Eq.
//           implicit_mac_equ_mac_flux)
// ------------------------------------------------------------------------------------
template <typename T, int WPB>
__global__ void __launch_bounds__(WPB * 32) k_face_interior(Dev<T> c) {
    using R = Red<T>;
    using V = typename R::V;
    const int lane = threadIdx.x & 31;
    const int fi = blockIdx.x * WPB + (threadIdx.x >> 5);
    if (fi >= c.Fi) return;                      // whole warp: no block barriers below
    const int f = c.face_int[fi];
    const size_t FK = (size_t)c.F * c.Kp;
    T* g0 = c.face + (size_t)f * c.Kp;
    T* h0 = c.face + FK + (size_t)f * c.Kp;
    // reference velocity U_r (any value is exact; the mean of the cells' U^n keeps
    // the shifted moments small)
    T Ur[3] = {T(0), T(0), T(0)};
    if (lane == 0) {
        const int a = c.fc[2 * f], b = c.fc[2 * f + 1];
        const double* Wa = c.W + 6 * (size_t)a;
        const double* Wb = c.W + 6 * (size_t)b;
        const T ia = T(1) / (T)Wa[0], ib = T(1) / (T)Wb[0];
        for (int d = 0; d < 3; ++d) Ur[d] = T(0.5) * ((T)Wa[1 + d] * ia + (T)Wb[1 + d] * ib);
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) Ur[d] = __shfl_sync(0xffffffffu, Ur[d], 0);
    V v[17];
    {
        Acc<T> m[17];
        for (int k = lane; k < c.K; k += 32) {
            const T cx = c.uT[k] - Ur[0], cy = c.uT[c.Kp + k] - Ur[1], cz = c.uT[2 * c.Kp + k] - Ur[2];
            const T w = c.wT[k];
            const T wg = w * g0[k], wh = w * h0[k];
            m[0].add(wg);
            m[1].add(wg * cx); m[2].add(wg * cy); m[3].add(wg * cz);
            m[4].add(wh);
            m[5].add(wg * cx * cx); m[6].add(wg * cy * cy); m[7].add(wg * cz * cz);
            m[8].add(wg * cx * cy); m[9].add(wg * cx * cz); m[10].add(wg * cy * cz);
            const T wgc2 = wg * (cx * cx + cy * cy + cz * cz);
            m[11].add(wgc2 * cx); m[12].add(wgc2 * cy); m[13].add(wgc2 * cz);
            m[14].add(wh * cx); m[15].add(wh * cy); m[16].add(wh * cz);
        }
#pragma unroll
        for (int j = 0; j < 17; ++j) v[j] = R::from(m[j]);
    }
    warp_red<T, 17>(v);
    // interface state on lane 0, in the per-velocity arithmetic type T (the moments
    // themselves are carried with compensation)
    constexpr int NB = EQN + 2;
    T cst[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) cst[j] = T(0);
    if (lane == 0) {
        T x[17];
        for (int j = 0; j < 17; ++j) x[j] = (T)R::to_d(v[j]);
        const T Rg = (T)c.R, Z = (T)c.Z, s = (T)c.fs[f];
        const T rho = x[0];
        const T d[3] = {x[1] / rho, x[2] / rho, x[3] / rho};
        const T U[3] = {Ur[0] + d[0], Ur[1] + d[1], Ur[2] + d[2]};
        const T tr = x[5] + x[6] + x[7];
        const T dd = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        const T etr = T(0.5) * (tr - rho * dd);            // rho E - 1/2 rho |U|^2 - sum w h
        const T Er0 = x[4];
        const T Tq = (etr + Er0) / (T(2.5) * rho * Rg);
        // tau from the translational temperature of the free-transport moments
        // (reading of the circular definition of the interface tau)
        const T Ttr0 = etr / (T(1.5) * rho * Rg);
        const T tau = (T)c.mu_ref * pow(Ttr0 / (T)c.T_ref, (T)c.omega_vis) / (rho * Rg * Ttr0);
        const T Erot = (Z * tau * Er0 + s * rho * Rg * Tq) / (Z * tau + s);
        const T Trot = Erot / (rho * Rg);
        const T Ttr = (etr + Er0 - Erot) / (T(1.5) * rho * Rg);
        // sum w c|c|^2 g and sum w c h about U = U_r + d (c = c' - d)
        const T Sd[3] = {x[5] * d[0] + x[8] * d[1] + x[9] * d[2],
                         x[8] * d[0] + x[6] * d[1] + x[10] * d[2],
                         x[9] * d[0] + x[10] * d[1] + x[7] * d[2]};
        const T dtr = tau + s - s / T(3) * (T(1) - T(1) / Z + (T)c.omega0 / Z);
        const T drot = tau + s - s * (T(1) - (T)c.delta) * (T(1) - T(1) / Z + (T)c.omega1 / Z);
        T qtr[3], qrot[3];
        for (int k = 0; k < 3; ++k) {
            const T Qtr = x[11 + k] - T(2) * Sd[k] - tr * d[k] + T(2) * rho * dd * d[k];
            qtr[k] = tau * T(0.5) * Qtr / dtr;
            qrot[k] = tau * (x[14 + k] - d[k] * Er0) / drot;
        }
        make_eq(c, rho, U, Tq, Ttr, Trot, qtr, qrot, cst + 2);
        cst[0] = tau / (tau + s);
        cst[1] = s / (tau + s);
        double* st = c.fstate + (size_t)f * FST;
        st[0] = rho; st[1] = U[0]; st[2] = U[1]; st[3] = U[2];
        st[4] = Tq; st[5] = Ttr; st[6] = Trot; st[7] = tau;
        for (int k = 0; k < 3; ++k) { st[8 + k] = qtr[k]; st[11 + k] = qrot[k]; }
        st[14] = s; st[15] = 0.0;
    }
    T e[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) e[j] = __shfl_sync(0xffffffffu, cst[j], 0);
    const T nx = (T)c.fn[f], ny = (T)c.fn[c.F + f], nz = (T)c.fn[2 * c.F + f];
    const T a = e[0], b = e[1];
    V r6[6];
    {
        Acc<T> m[6];
        for (int k = lane; k < c.K; k += 32) {
            const T ux = c.uT[k], uy = c.uT[c.Kp + k], uz = c.uT[2 * c.Kp + k], w = c.wT[k];
            T G, H;
            eval_eq(e + 2, ux, uy, uz, G, H);
            const T gf = a * g0[k] + b * G;
            const T hf = a * h0[k] + b * H;
            g0[k] = gf;
            h0[k] = hf;
            const T wu = w * (ux * nx + uy * ny + uz * nz);
            const T wg = wu * gf;
            m[0].add(wg); m[1].add(wg * ux); m[2].add(wg * uy); m[3].add(wg * uz);
            m[4].add(wu * (T(0.5) * (ux * ux + uy * uy + uz * uz) * gf + hf));
            m[5].add(wu * hf);
        }
#pragma unroll
        for (int j = 0; j < 6; ++j) r6[j] = R::from(m[j]);
    }
    warp_red<T, 6>(r6);
    if (lane == 0)
        for (int d = 0; d < 6; ++d) c.mface[(size_t)f * 6 + d] = R::to_d(r6[d]);
}

// Boundary faces (reading; the paper names diffuse reflection but gives no formula):
// leaving particles carry the reconstructed interior value; entering particles
// follow the wall Maxwellian rho_w g^eq(u; 1, U_w, T_w), h = R T_w g, with rho_w
// giving zero discrete mass flux, or the freestream Maxwellian at a farfield face.
// Also the wall sums of Eqs. cp, cf, ch: p_w, sum w (u.n) u G, q_w.
template <typename T, int BS>
__global__ void __launch_bounds__(BS) k_face_boundary(Dev<T> c) {
    __shared__ double red[7 * (BS / 32)];
    __shared__ T mc[6];
    __shared__ double rw;
    const int b = blockIdx.x;
    const int f = c.face_bnd[b];
    const int bc = -1 - c.fc[2 * f + 1];
    const int kind = c.bck[bc];
    const size_t FK = (size_t)c.F * c.Kp;
    T* g0 = c.face + (size_t)f * c.Kp;
    T* h0 = c.face + FK + (size_t)f * c.Kp;
    const double nxd = c.fn[f], nyd = c.fn[c.F + f], nzd = c.fn[2 * c.F + f];
    const T nx = (T)nxd, ny = (T)nyd, nz = (T)nzd;
    if (threadIdx.x == 0) {
        const double* bv = c.bcv + 5 * bc;
        const double RT = c.R * bv[4];
        const double a = 2.0 * PI * RT;
        const double rho = (kind == 0) ? 1.0 : bv[0];
        mc[0] = (T)bv[1]; mc[1] = (T)bv[2]; mc[2] = (T)bv[3];
        mc[3] = (T)(rho / (a * sqrt(a)));
        mc[4] = (T)(1.0 / (2.0 * RT));
        mc[5] = (T)RT;
    }
    __syncthreads();
    if (kind == 0) {
        double v[2];
        Acc<T> an, ad;
        for (int k = threadIdx.x; k < c.K; k += BS) {
            const T ux = c.uT[k], uy = c.uT[c.Kp + k], uz = c.uT[2 * c.Kp + k], w = c.wT[k];
            const T un = dot_rn(ux, uy, uz, nx, ny, nz);
            if (un > T(0)) an.add(w * un * g0[k]);
            else ad.add(-w * un * maxwell(mc, ux, uy, uz));
        }
        v[0] = an.get(); v[1] = ad.get();
        block_sum<2, BS>(v, red);
        if (threadIdx.x == 0) rw = v[0] / v[1];
        __syncthreads();
    } else if (threadIdx.x == 0) {
        rw = 1.0;
    }
    __syncthreads();
    const T scale = (T)rw;
    double v[7];
    {
        Acc<T> a[7];
        for (int k = threadIdx.x; k < c.K; k += BS) {
            const T ux = c.uT[k], uy = c.uT[c.Kp + k], uz = c.uT[2 * c.Kp + k], w = c.wT[k];
            const T un = dot_rn(ux, uy, uz, nx, ny, nz);
            T gf, hf;
            if (un > T(0)) {
                gf = g0[k];
                hf = h0[k];
            } else {
                gf = scale * maxwell(mc, ux, uy, uz);
                hf = mc[5] * gf;
                g0[k] = gf;
                h0[k] = hf;
            }
            const T wu = w * un;
            const T wg = wu * gf;
            a[0].add(wg); a[1].add(wg * ux); a[2].add(wg * uy); a[3].add(wg * uz);
            a[4].add(wu * (T(0.5) * (ux * ux + uy * uy + uz * uz) * gf + hf));
            a[5].add(wu * hf);
            a[6].add(wg * un);           // p_w = sum w (u.n)^2 G
        }
        for (int j = 0; j < 7; ++j) v[j] = a[j].get();
    }
    block_sum<7, BS>(v, red);
    if (threadIdx.x == 0) {
        for (int d = 0; d < 6; ++d) c.mface[(size_t)f * 6 + d] = v[d];
        double* wq = c.wallq + 8 * (size_t)b;
        wq[0] = v[6];                                // p_w
        wq[1] = v[1]; wq[2] = v[2]; wq[3] = v[3];    // sum w (u.n) u G
        wq[4] = v[4];                                // q_w = sum w (u.n)(|u|^2/2 G + R)
        wq[5] = (kind == 0) ? rw : 0.0;
        wq[6] = wq[7] = 0.0;
        double* fsr = c.fstate + (size_t)f * FST;
        for (int d = 0; d < FST; ++d) fsr[d] = 0.0;
        fsr[14] = c.fs[f];
        fsr[15] = (kind == 0) ? rw : 0.0;
    }
}

// ------------------------------------------------------------------------------------
// Step 3 / Step 4 ingredients
// ------------------------------------------------------------------------------------
// spectral radius r_ij (Eq. implicit_mac_equ_spectral_radius) from the arithmetic
// mean of the cells' W^n (W_i at boundary faces)
template <typename T>
__global__ void k_face_radius(Dev<T> c) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= c.F) return;
    const int a = c.fc[2 * f], b = c.fc[2 * f + 1];
    double Wm[6];
    for (int m = 0; m < 6; ++m)
        Wm[m] = (b >= 0) ? 0.5 * (c.W[6 * (size_t)a + m] + c.W[6 * (size_t)b + m]) : c.W[6 * (size_t)a + m];
    Prim p = prim_from_W(Wm, c.R);
    const double a_s = sqrt(1.4 * c.R * p.T);
    const double Un = p.U[0] * c.fn[f] + p.U[1] * c.fn[c.F + f] + p.U[2] * c.fn[2 * c.F + f];
    c.rf[f] = fabs(Un) + a_s + 2.0 * viscosity(c, p.Ttr) / (p.rho * c.fdl[f]);
}

// macro flux F_i = (1/V_i) sum_j A_ij [sum_k w (u.n_ij) Phi phi_ij] (Eq. implicit_mac_equ_mac_flux)
template <typename T>
__global__ void k_cell_macro_flux(Dev<T> c) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= c.N) return;
    double M[6] = {0, 0, 0, 0, 0, 0};
    for (int m = c.slot_off[i]; m < c.slot_off[i + 1]; ++m) {
        const int f = c.slot_face[m];
        const double sg = c.slot_left[m] ? 1.0 : -1.0;
        for (int d = 0; d < 6; ++d) M[d] += sg * c.fa[f] * c.mface[6 * (size_t)f + d];
    }
    const double iv = 1.0 / c.vol[i];
    for (int d = 0; d < 6; ++d) c.macroF[6 * (size_t)i + d] = M[d] * iv;
}

__device__ __forceinline__ void euler_flux(const double* W, double nx, double ny, double nz, double* G) {
    const double rho = W[0];
    const double U[3] = {W[1] / rho, W[2] / rho, W[3] / rho};
    const double p = 0.4 * (W[4] - 0.5 * rho * (U[0] * U[0] + U[1] * U[1] + U[2] * U[2]));
    const double Un = U[0] * nx + U[1] * ny + U[2] * nz;
    G[0] = rho * Un;
    G[1] = W[1] * Un + p * nx;
    G[2] = W[2] * Un + p * ny;
    G[3] = W[3] * Un + p * nz;
    G[4] = (W[4] + p) * Un;
    G[5] = W[5] * Un;
}

// flux primitives (rho, U, rho E + p, p, rho E_rot) with p = rho R T = 0.4 (rho E -
// 1/2 rho |U|^2); false if the state is not admissible (rho, T_tr or T_rot <= 0)
__device__ __forceinline__ bool flux_prim(const double* W, double* P) {
    const double rho = W[0], ir = 1.0 / rho;
    const double U[3] = {W[1] * ir, W[2] * ir, W[3] * ir};
    const double ke = 0.5 * rho * (U[0] * U[0] + U[1] * U[1] + U[2] * U[2]);
    const double p = 0.4 * (W[4] - ke);
    P[0] = rho; P[1] = U[0]; P[2] = U[1]; P[3] = U[2]; P[4] = W[4] + p; P[5] = p; P[6] = W[5];
    P[7] = 0.0;
    return rho > 0.0 && (W[4] - ke - W[5]) > 0.0 && W[5] > 0.0;
}

// Per-iteration set-up of the macro PR-SGS: per cell 1/D_i with
// D_i = 1/dt + sum_j A r/(2V) (and + 1/(Z tau) for rho E_rot, tau frozen at its W^n
// value: reading of the tilde quantities in the source), 1/(Z tau); per slot the
// neighbour's Euler flux G_ij(W_j^n) and the coefficients A/(2V), A r/(2V); the flux
// primitives of W^n; dW~ = 0.
template <typename T>
__global__ void k_macro_prep(Dev<T> c, double cfl) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= c.N) return;
    const double iv = 1.0 / c.vol[i];
    double D = 1.0 / (cfl * c.dt[i]);
    for (int m = c.slot_off[i]; m < c.slot_off[i + 1]; ++m) {
        const int f = c.slot_face[m], j = c.slot_nbr[m];
        const double A = c.fa[f] * iv;
        D += 0.5 * A * c.rf[f];
        c.sC[2 * (size_t)m] = 0.5 * A;
        c.sC[2 * (size_t)m + 1] = 0.5 * A * c.rf[f];
        if (j >= 0) {
            const double sg = c.slot_left[m] ? 1.0 : -1.0;
            euler_flux(c.W + 6 * (size_t)j, sg * c.fn[f], sg * c.fn[c.F + f], sg * c.fn[2 * c.F + f],
                       c.sG0 + 6 * (size_t)m);
        }
    }
    const Prim p = prim_from_W(c.W + 6 * (size_t)i, c.R);
    const double izt = 1.0 / (c.Z * relax_time(c, p.rho, p.Ttr));
    c.mDb[4 * (size_t)i] = 1.0 / D;
    c.mDb[4 * (size_t)i + 1] = 1.0 / (D + izt);
    c.mDb[4 * (size_t)i + 2] = izt;
    flux_prim(c.W + 6 * (size_t)i, c.mPc + 8 * (size_t)i);
    for (int q = 0; q < 6; ++q) c.dW[6 * (size_t)i + q] = 0.0;
}

// One point update of the macro PR-SGS (Eq. implicit_mac_equ_fin) for every cell of
// one colour, one thread per cell:
//   dW~_i = [Res_i - sum_j (A/2V) ((G(W_j + dW~_j) - G(W_j)) - r dW~_j)] / D_i,
// the flux Jacobian applied matrix-free with the neighbours' cached flux
// primitives; rho~ R T~ of the rotational source from the cell's current iterate.
// An update whose predicted state is not admissible (rho, T_tr or T_rot not
// positive) is skipped.
template <typename T>
__global__ void __launch_bounds__(128) k_macro_sweep(Dev<T> c, const int* cells, int n, int colour,
                                                     int first_forward) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int i = cells[t];
    double o[6] = {0, 0, 0, 0, 0, 0};
    for (int m = c.slot_off[i]; m < c.slot_off[i + 1]; ++m) {
        const int j = c.slot_nbr[m];
        if (j < 0 || (first_forward && c.slot_ncol[m] > colour)) continue;
        const int f = c.slot_face[m];
        const double sg = c.slot_left[m] ? 1.0 : -1.0;
        const double nx = sg * c.fn[f], ny = sg * c.fn[c.F + f], nz = sg * c.fn[2 * c.F + f];
        const double* P = c.mPc + 8 * (size_t)j;
        const double Un = P[1] * nx + P[2] * ny + P[3] * nz;
        const double rU = P[0] * Un;
        const double G1[6] = {rU, rU * P[1] + P[5] * nx, rU * P[2] + P[5] * ny, rU * P[3] + P[5] * nz,
                              P[4] * Un, P[6] * Un};
        const double* G0 = c.sG0 + 6 * (size_t)m;
        const double* dWj = c.dW + 6 * (size_t)j;
        const double c1 = c.sC[2 * (size_t)m], c2 = c.sC[2 * (size_t)m + 1];
#pragma unroll
        for (int q = 0; q < 6; ++q) o[q] += c1 * (G1[q] - G0[q]) - c2 * dWj[q];
    }
    const double* W = c.W + 6 * (size_t)i;
    double* dW = c.dW + 6 * (size_t)i;
    // rho R T of the current iterate: (2/5)(rho E - |rho U|^2 / (2 rho))
    const double rc = W[0] + dW[0];
    const double mx = W[1] + dW[1], my = W[2] + dW[2], mz = W[3] + dW[3];
    const double rRT = 0.4 * (W[4] + dW[4] - 0.5 * (mx * mx + my * my + mz * mz) / rc);
    const double* F = c.macroF + 6 * (size_t)i;
    const double iD = c.mDb[4 * (size_t)i], iDr = c.mDb[4 * (size_t)i + 1], izt = c.mDb[4 * (size_t)i + 2];
    double cand[6];
    for (int q = 0; q < 5; ++q) cand[q] = (-F[q] - o[q]) * iD;
    cand[5] = ((rRT - W[5]) * izt - F[5] - o[5]) * iDr;
    double Wn[6], Pn[8];
    for (int q = 0; q < 6; ++q) Wn[q] = W[q] + cand[q];
    if (!flux_prim(Wn, Pn)) return;
    for (int q = 0; q < 6; ++q) dW[q] = cand[q];
    for (int q = 0; q < 8; ++q) c.mPc[8 * (size_t)i + q] = Pn[q];
}

// W~ = W^n + dW~, tau~ and the per-cell record of the micro sweeps: constants of the
// predicted equilibrium phi~* built from (W~, q^n) (reading: the prediction gives no
// heat flux, so the last Step-6 value is used), 1/tau~, and 1/dt + 1/tau~.
template <typename T>
__global__ void k_macro_finish(Dev<T> c, double cfl) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= c.N) return;
    double* Wt = c.Wt + 6 * (size_t)i;
    for (int m = 0; m < 6; ++m) Wt[m] = c.W[6 * (size_t)i + m] + c.dW[6 * (size_t)i + m];
    const Prim p = prim_from_W(Wt, c.R);
    const double tau = relax_time(c, p.rho, p.Ttr);
    c.taut[i] = tau;
    const double* q = c.q + 6 * (size_t)i;
    double* e = c.ceq + (size_t)i * CEQ;
    make_eq(c, p.rho, p.U, p.T, p.Ttr, p.Trot, q, q + 3, e);
    e[23] = 1.0 / tau;
    e[24] = 1.0 / (cfl * c.dt[i]) + 1.0 / tau;
}

// ------------------------------------------------------------------------------------
// Step 5 (micro PR-SGS, Eq. implicit_mic_final_equ) and Step 6 (update and integral
// error compensation, Eqs. solve_rho - solve_qrot).  One block per cell of one
// colour, velocities strided over the block.
//   first sweep : Res = (phi~* - phi^n)/tau~ - F_{i,k}, F from the face array
//                 (Eq. implicit_mic_flux), stored
//   every sweep : dphi_i = (Res - sum_j (A/V) min(u.n, 0) dphi_j) / D_{i,k},
//                 D = 1/dt + 1/tau~ + sum_f (A/V) max(u.n, 0); boundary ghosts 0
//   last sweep  : phi^{n+1} = phi^n + dphi and the sums of Step 6 over k
// ------------------------------------------------------------------------------------
template <typename T, int BS>
__global__ void __launch_bounds__(BS, 3) k_micro_sweep(Dev<T> c, const int* cells, int colour,
                                                    int first, int first_forward, int last) {
    using R = Red<T>;
    __shared__ T e[EQN + 2];
    __shared__ typename R::V red[12 * (BS / 32)];
    __shared__ double tot[12];
    __shared__ int sh_face[MAXF], sh_nbr[MAXF], sh_ok[MAXF];
    __shared__ T sh_n[3][MAXF], sh_AV[MAXF];
    const int i = cells[blockIdx.x];
    const int s0 = c.slot_off[i], ns = c.slot_off[i + 1] - s0;
    if (threadIdx.x < EQN + 2) e[threadIdx.x] = (T)c.ceq[(size_t)i * CEQ + threadIdx.x];
    if (threadIdx.x < ns) {
        const int m = s0 + threadIdx.x;
        sh_face[threadIdx.x] = c.slot_face[m];
        sh_nbr[threadIdx.x] = c.slot_nbr[m];
        sh_ok[threadIdx.x] = (c.slot_nbr[m] >= 0) && !(first_forward && c.slot_ncol[m] > colour);
        const T sg = c.slot_left[m] ? T(1) : T(-1);
        sh_n[0][threadIdx.x] = sg * c.slot_nT[m];
        sh_n[1][threadIdx.x] = sg * c.slot_nT[c.nnz + m];
        sh_n[2][threadIdx.x] = sg * c.slot_nT[2 * c.nnz + m];
        sh_AV[threadIdx.x] = c.slot_AVT[m];
    }
    __syncthreads();
    const T itau = e[EQN - 1], base = e[EQN];
    const size_t NK = (size_t)c.N * c.Kp, FK = (size_t)c.F * c.Kp;
    const size_t oi = (size_t)i * c.Kp;
    Acc<T> a[12];
    for (int k = threadIdx.x; k < c.K; k += BS) {
        const T ux = c.uT[k], uy = c.uT[c.Kp + k], uz = c.uT[2 * c.Kp + k];
        T rg, rh;
        T D = base, og = T(0), oh = T(0);
        T Fg = T(0), Fh = T(0);
#pragma unroll 1
        for (int q = 0; q < ns; ++q) {
            const T un = dot_split(ux, uy, uz, sh_n[0][q], sh_n[1][q], sh_n[2][q]);
            const T AV = sh_AV[q];
            if (first) {
                const size_t of = (size_t)sh_face[q] * c.Kp + k;
                Fg += AV * un * c.face[of];
                Fh += AV * un * c.face[FK + of];
            }
            if (un > T(0)) {
                D += AV * un;
            } else if (sh_ok[q]) {
                const size_t oj = (size_t)sh_nbr[q] * c.Kp + k;
                og += AV * un * c.dphi[oj];
                oh += AV * un * c.dphi[NK + oj];
            }
        }
        T G = T(0), H = T(0);
        if (first || last) eval_eq(e, ux, uy, uz, G, H);
        if (first) {
            rg = (G - c.phi[oi + k]) * itau - Fg;
            rh = (H - c.phi[NK + oi + k]) * itau - Fh;
            c.res[oi + k] = rg;
            c.res[NK + oi + k] = rh;
        } else {
            rg = c.res[oi + k];
            rh = c.res[NK + oi + k];
        }
        const T iD = T(1) / D;
        const T dg = (rg - og) * iD, dh = (rh - oh) * iD;
        c.dphi[oi + k] = dg;
        c.dphi[NK + oi + k] = dh;
        if (last) {
            const T g1 = c.phi[oi + k] + dg, h1 = c.phi[NK + oi + k] + dh;
            c.phi[oi + k] = g1;
            c.phi[NK + oi + k] = h1;
            const T w = c.wT[k];
            const T Dg = g1 - G, Dh = h1 - H;
            const T cx = ux - e[0], cy = uy - e[1], cz = uz - e[2];
            const T c2 = cx * cx + cy * cy + cz * cz;
            const T wg = w * Dg, wh = w * Dh;
            a[0].add(wg); a[1].add(wg * ux); a[2].add(wg * uy); a[3].add(wg * uz);
            a[4].add(T(0.5) * (ux * ux + uy * uy + uz * uz) * wg + wh);
            a[5].add(wh);
            const T wgc = wg * c2;
            a[6].add(wgc * cx); a[7].add(wgc * cy); a[8].add(wgc * cz);
            a[9].add(wh * cx); a[10].add(wh * cy); a[11].add(wh * cz);
        }
    }
    if (last) {
        typename R::V v[12];
#pragma unroll
        for (int j = 0; j < 12; ++j) v[j] = R::from(a[j]);
        block_red<T, 12, BS>(v, red, tot);
        if (threadIdx.x < 12) c.S[(size_t)i * 12 + threadIdx.x] = tot[threadIdx.x];
    }
}

// Step 6 per cell (compensation) and the residual contributions, summed per block
// (deterministic) into cellres[block][12].
template <typename T>
__global__ void __launch_bounds__(128) k_cell_update(Dev<T> c) {
    __shared__ double red[12 * 4];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double r[12];
    for (int m = 0; m < 12; ++m) r[m] = 0.0;
    if (i < c.N) {
        const double Z = c.Z;
        const double* S = c.S + (size_t)i * 12;
        const double* Wt = c.Wt + 6 * (size_t)i;
        double* W = c.W + 6 * (size_t)i;
        double* q = c.q + 6 * (size_t)i;
        double Wo[6];
        for (int m = 0; m < 6; ++m) Wo[m] = W[m];
        const Prim p = prim_from_W(Wt, c.R);
        for (int m = 0; m < 5; ++m) W[m] = S[m] + Wt[m];
        W[5] = S[5] + p.rho * c.R * ((1.0 - 1.0 / Z) * p.Trot + p.T / Z);   // K_rot/2 = 1
        const double atr = (1.0 / 3.0) * (1.0 - (1.0 - c.omega0) / Z);
        const double arot = (1.0 - c.delta) * (1.0 - (1.0 - c.omega1) / Z);
        for (int d = 0; d < 3; ++d) {
            const double qt = q[d], qr = q[3 + d];
            q[d] = 0.5 * S[6 + d] + qt * atr;
            q[3 + d] = S[9 + d] + qr * arot;
        }
        for (int m = 0; m < 6; ++m) r[m] = fabs(W[m] - Wo[m]);
        const double mom = sqrt(Wo[1] * Wo[1] + Wo[2] * Wo[2] + Wo[3] * Wo[3]);
        r[6] = fabs(Wo[0]); r[7] = mom; r[8] = mom; r[9] = mom; r[10] = fabs(Wo[4]); r[11] = fabs(Wo[5]);
    }
    block_sum<12, 128>(r, red);
    if (threadIdx.x == 0)
        for (int m = 0; m < 12; ++m) c.cellres[(size_t)blockIdx.x * 12 + m] = r[m];
}

// deterministic reduction of the per-block residual partials (one block of 256)
template <typename T>
__global__ void __launch_bounds__(256) k_residual_reduce(Dev<T> c, int nblocks) {
    __shared__ double red[12 * 8];
    double v[12];
    for (int j = 0; j < 12; ++j) v[j] = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += 256)
        for (int j = 0; j < 12; ++j) v[j] += c.cellres[(size_t)b * 12 + j];
    block_sum<12, 256>(v, red);
    if (threadIdx.x == 0) {
        for (int m = 0; m < 6; ++m) c.res12[m] = v[m] / (v[6 + m] > 1e-300 ? v[6 + m] : 1e-300);
        int bad = 0;
        for (int m = 0; m < 6; ++m) bad |= !isfinite(c.res12[m]);
        if (bad) atomicOr(c.status, 2);
    }
}

// micro flux F_{i,k} of the current face array, materialised for verification only
template <typename T>
__global__ void k_debug_micro_flux(Dev<T> c, T* out) {
    const int i = blockIdx.x;
    const int k = blockIdx.y * blockDim.x + threadIdx.x;
    if (k >= c.K) return;
    const size_t FK = (size_t)c.F * c.Kp, NK = (size_t)c.N * c.Kp;
    const T ux = c.uT[k], uy = c.uT[c.Kp + k], uz = c.uT[2 * c.Kp + k];
    T Fg = T(0), Fh = T(0);
    for (int m = c.slot_off[i]; m < c.slot_off[i + 1]; ++m) {
        const T sg = c.slot_left[m] ? T(1) : T(-1);
        const T un = dot_rn(ux, uy, uz, sg * c.slot_nT[m], sg * c.slot_nT[c.nnz + m], sg * c.slot_nT[2 * c.nnz + m]);
        const size_t of = (size_t)c.slot_face[m] * c.Kp + k;
        Fg += c.slot_AVT[m] * un * c.face[of];
        Fh += c.slot_AVT[m] * un * c.face[FK + of];
    }
    out[(size_t)i * c.Kp + k] = Fg;
    out[NK + (size_t)i * c.Kp + k] = Fh;
}

}  // namespace rk

namespace rk {

// (T, T_tr, T_rot) per cell from W
template <typename T>
__global__ void k_temps(Dev<T> c, double* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= c.N) return;
    const Prim p = prim_from_W(c.W + 6 * (size_t)i, c.R);
    out[3 * (size_t)i] = p.T;
    out[3 * (size_t)i + 1] = p.Ttr;
    out[3 * (size_t)i + 2] = p.Trot;
}

// Wall coefficients of Eqs. cp, cf, ch from the per-face wall sums written by
// k_face_boundary; out[w][8] = p_w, tau (3), q_w, Cp, C_tau, C_h, and per-face force
// and heat contributions for the totals.
template <typename T>
__global__ void k_surface(Dev<T> c, const int* wall_b, int nw, double p_inf, double qdyn,
                          double Umag, double* out, double* contrib) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nw) return;
    const int b = wall_b[t];
    const int f = c.face_bnd[b];
    const double* wq = c.wallq + 8 * (size_t)b;
    const double n[3] = {c.fn[f], c.fn[c.F + f], c.fn[2 * c.F + f]};
    const double pw = wq[0];
    const double tw[3] = {wq[1] - n[0] * pw, wq[2] - n[1] * pw, wq[3] - n[2] * pw};
    double* o = out + 8 * (size_t)t;
    o[0] = pw; o[1] = tw[0]; o[2] = tw[1]; o[3] = tw[2]; o[4] = wq[4];
    o[5] = (pw - p_inf) / qdyn;
    o[6] = sqrt(tw[0] * tw[0] + tw[1] * tw[1] + tw[2] * tw[2]) / qdyn;
    o[7] = wq[4] / (qdyn * Umag);
    double* cb = contrib + 4 * (size_t)t;
    cb[0] = c.fa[f] * wq[1]; cb[1] = c.fa[f] * wq[2]; cb[2] = c.fa[f] * wq[3]; cb[3] = c.fa[f] * wq[4];
}

static __global__ void __launch_bounds__(256) k_sum4(const double* contrib, int n, double* tot) {
    __shared__ double red[4 * 8];
    double v[4] = {0, 0, 0, 0};
    for (int i = threadIdx.x; i < n; i += 256)
        for (int j = 0; j < 4; ++j) v[j] += contrib[4 * (size_t)i + j];
    block_sum<4, 256>(v, red);
    if (threadIdx.x == 0)
        for (int j = 0; j < 4; ++j) tot[j] = v[j];
}

}  // namespace rk
