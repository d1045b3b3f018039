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

#include <type_traits>

namespace rk {

constexpr int MAXF = 8;        // faces per cell
// micro sweep tuning: faces per load group, velocities per lane in the middle sweeps
// (mixed mode), minimum resident blocks of the first / middle / last sweeps
#ifndef MICRO_PF
#define MICRO_PF 1
#endif
#ifndef RECON_NV
#define RECON_NV 4           // velocities per lane of k_recon in mixed mode (16-byte accesses)
#endif
#ifndef FACE_NV
#define FACE_NV 4            // velocities per lane of k_face_interior in mixed mode (16-byte accesses)
#endif
#ifndef FACE_CG
#define FACE_CG 1            // k_face_interior reads the face rows through L2 only
#endif
#ifndef FACE_PADSEL
#define FACE_PADSEL 1        // 1: the K padding zeroed by a select per velocity (0: in a tail
                             // branch; measured 43.9 vs 38.6 ms at scale: code generation)
#endif
#ifndef FACE_FW
#define FACE_FW 1            // warps per interior face in mixed mode (k_face_interior; 2, 4
                             // and 8 measured slower: the kernel is issue-bound)
#endif
#ifndef MICRO_FLUX_NV
#define MICRO_FLUX_NV 4
#endif
#ifndef MICRO_MID_NV
#define MICRO_MID_NV 4
#endif
#ifndef MICRO_FIRST_MINB
#define MICRO_FIRST_MINB 3
#endif
#ifndef MICRO_FIRST_NV
#define MICRO_FIRST_NV 4
#endif
#ifndef MICRO_MID_MINB
#define MICRO_MID_MINB 5
#endif
#ifndef MICRO_LAST_MINB
#define MICRO_LAST_MINB 2
#endif
#ifndef MICRO_LAST_NV
#define MICRO_LAST_NV 4
#endif
#ifndef MICRO_LAST_PF
#define MICRO_LAST_PF MICRO_PF
#endif
// limiter ratio in mixed mode: 1 = approximate division (__fdividef, 2 ulp)
#ifndef RECON_FASTDIV
#define RECON_FASTDIV 1
#endif
// mixed-mode limiter: 1 = both evaluations computed and selected without branches
#ifndef RECON_BF
#define RECON_BF 1
#endif
constexpr int EQN = 24;        // constants of one Rykov equilibrium (see make_eq)
constexpr int CEQ = 28;        // per-cell record: EQN constants, 1/tau~, diagonal base
constexpr int FST = 16;        // face state record
constexpr double PI = 3.14159265358979323846;

// Fields that do not depend on the per-velocity type T (FP64 geometry, per-cell and
// per-face state, parameters); Dev<T> adds the per-velocity arrays and their T copies.
struct DevBase {
    int N, F, K, Kp, C, Fi, Fb, nnz;
    int debug;                         // write verification-only records (face states)
    int packed;                        // mixed mode: kernels on the packed FP32 pipe
    // implicit-step schedule, evaluated on the device each iteration (k_iter_begin)
    double cfl_imp, cfl_imp0, cfl_ramp;
    int first_order_iters, limiter, limiter_freeze;
    int viscosity_law;                 // 0 power law, 1 Sutherland
    double sutherland_c;               // Sutherland constant C_s
    // [0] cfl, [1] reconstruction mode (0 unlimited, 1 limited, 2 first order,
    // 3 limited with the stored limiter values, 4 limited and store them), [2] counter
    double* iterp;
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
    // faces
    const int* fc;                     // [F][2]
    const double *fn, *fa, *fxc;       // [3][F], [F], [3][F]
    double *fs, *fdl, *rf;             // s_ij, distance used in r_ij, r_ij  [F]
    const int *face_int, *face_bnd;    // lists
    const double* bcv;                 // [64][5]: rho, U, T
    const int* bck;                    // [64] kind
    // discrete velocity space (SoA, padded with zero weights)
    const double *u, *w;               // [3][Kp], [Kp]
    // per-cell / per-face state
    double *W, *q, *Wold, *fstate, *mface, *wallq, *macroF, *dW, *Wt, *ceq, *taut, *S,
        *cellres, *res12;
    // macro PR-SGS work: flux primitives (rho, U, rho E + p, p, rho E_rot) of the
    // current iterate per cell, diagonal base per cell, per-slot Euler flux of the
    // neighbour's W^n and the coefficients A/(2V), A r/(2V)
    double *mPc, *mDb, *sG0, *sC;        // mDb: [N][4] = 1/D, 1/(D + 1/(Z tau)), 1/(Z tau)
    double* mB;                          // [N][12]: F_i - sum_j (A/2V) G_ij(W_j^n), all / lower-colour j
    // the slots again, ordered by colour position (cells in col_cell order), so that a
    // macro point update finds its slot range from its position without first loading
    // the cell index: slot base per position [N+1], position of each cell [N],
    // neighbour, neighbour colour [nnz], outward normal [3][nnz]; sG0 and sC are
    // indexed by these position-ordered slots
    const int *pos_off, *cell_pos, *pslot_nbr, *pslot_ncol;
    const double* pslot_n;
    unsigned int* bar;                   // grid-barrier state of the cooperative macro solve
    const int* col_off_d;                // colour offsets on the device (C + 1)
    int* status;
};

template <typename T>
struct Dev : DevBase {
    // R, Z, mu_ref, T_ref, omega_vis, omega0, omega1, delta in T (no conversions in kernels)
    T tp[8];
    T *slot_nT, *slot_AVT, *slot_dT, *slot_lsqT, *slot_sT;
    T *fnT, *fsT;                      // face normal [3][F] and s_ij [F] in T
    const T *uT, *wT;
    // per-velocity state
    T *phi, *face, *res, *dphi, *lstore;   // lstore: [2][N][Kp] frozen limiter values
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
// exp of the per-velocity arithmetic: FP64 exp in FP64 mode; the hardware exp2-based
// __expf in mixed mode (relative error ~1e-6 over the arguments that matter, below
// the 1e-5 target of the mixed mode)
__device__ __forceinline__ double ex(double x) { return exp(x); }
__device__ __forceinline__ float ex(float x) { return __expf(x); }
// 2^x for the equilibria (exponents pre-scaled by log2(e)): FP64 exp2 in FP64 mode;
// in mixed mode the hardware approximation (PTX ex2.approx.f32: relative error ~2^-22,
// subnormal results kept), one instruction where the accurate exp2f takes a longer
// path for the very negative exponents of the high-speed tails of the DVS
__device__ __forceinline__ double ex2(double x) { return exp2(x); }
__device__ __forceinline__ float ex2(float x) {
    float y;
    asm("ex2.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
__device__ __forceinline__ float rcp(float x) { return __fdividef(1.0f, x); }
// quotient of the limiter function: exact in FP64 mode
__device__ __forceinline__ double lim_div(double a, double b) { return a / b; }
__device__ __forceinline__ float lim_div(float a, float b) {
#if RECON_FASTDIV
    // the approximate quotient takes the reciprocal of b, which overflows for b below
    // ~1e-38 (the distribution tails give such differences): both operands are then
    // scaled by 2^64 first (exact), which leaves the quotient unchanged
    const float sc = b < 1e-30f ? 18446744073709551616.0f : 1.0f;
    return __fdividef(a * sc, b * sc);
#else
    return a / b;
#endif
}

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
    static __device__ __forceinline__ V shfl(V v, int l) { return __shfl_sync(0xffffffffu, v, l); }
    static __device__ __forceinline__ double to_d(V v) { return v; }
    static __device__ __forceinline__ double to_T(V v) { return v; }
    static __device__ __forceinline__ void store(double* p, V v) { *p = v; }
    static __device__ __forceinline__ double load(const double* p) { return *p; }
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
    static __device__ __forceinline__ V shfl(V v, int l) {
        return FF{__shfl_sync(0xffffffffu, v.hi, l), __shfl_sync(0xffffffffu, v.lo, l)};
    }
    static __device__ __forceinline__ double to_d(V v) { return (double)v.hi + (double)v.lo; }
    static __device__ __forceinline__ float to_T(V v) { return __fadd_rn(v.hi, v.lo); }
    // a double slot holds the float-float pair (hi, lo)
    static __device__ __forceinline__ void store(double* p, V v) {
        *reinterpret_cast<float2*>(p) = make_float2(v.hi, v.lo);
    }
    static __device__ __forceinline__ double load(const double* p) {
        const float2 x = *reinterpret_cast<const float2*>(p);
        return (double)x.x + (double)x.y;
    }
};

template <typename T, int NV>
__device__ __forceinline__ void warp_red(typename Red<T>::V (&v)[NV]) {
#pragma unroll
    for (int j = 0; j < NV; ++j) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[j] = Red<T>::add(v[j], Red<T>::shfl_xor(v[j], o));
    }
}

// Sum over the 32 lanes of N values whose totals are needed on lane 0 only
// (reduce-scatter, then a gather): at the level with lane offset o every lane keeps
// half of its slots, sending the other half to its partner (one shuffle per kept
// slot instead of one per value), so the five levels cost ceil(N/2) + ... shuffles
// and additions instead of 5 N; lane 0 then fetches each total from the lane that
// holds it.  Fixed order: deterministic.  Other lanes' values are partial sums.
#ifndef WARP_RED_SCATTER
#define WARP_RED_SCATTER 1
#endif
template <typename T, int NI, int NO>
__device__ __forceinline__ void red_level(const typename Red<T>::V (&in)[NI], typename Red<T>::V (&out)[NO],
                                          int off) {
    using R = Red<T>;
    const bool upper = (threadIdx.x & off) != 0;
#pragma unroll
    for (int p = 0; p < NO; ++p) {
        const typename R::V lo = in[p];
        const typename R::V hi = (p + NO < NI) ? in[p + NO] : R::zero();
        const typename R::V recv = R::shfl_xor(upper ? lo : hi, off);
        out[p] = R::add(upper ? hi : lo, recv);
    }
}
template <typename T, int N>
__device__ __forceinline__ void warp_red0(typename Red<T>::V (&v)[N]) {
    using R = Red<T>;
    using V = typename R::V;
    static_assert(N >= 1 && N <= 32, "warp_red0: 1..32 values");
    constexpr int N1 = (N + 1) / 2, N2 = (N1 + 1) / 2, N3 = (N2 + 1) / 2, N4 = (N3 + 1) / 2,
                  N5 = (N4 + 1) / 2;
    static_assert(N5 == 1, "warp_red0: one slot per lane at the end");
    V a1[N1], a2[N2], a3[N3], a4[N4], a5[N5];
    red_level<T, N, N1>(v, a1, 16);
    red_level<T, N1, N2>(a1, a2, 8);
    red_level<T, N2, N3>(a2, a3, 4);
    red_level<T, N3, N4>(a3, a4, 2);
    red_level<T, N4, N5>(a4, a5, 1);
    // value j sits on the lane whose offset bits select it at each level
#pragma unroll
    for (int j = 0; j < N; ++j) {
        int q = j, lane = 0;
        if (q >= N1) { q -= N1; lane |= 16; }
        if (q >= N2) { q -= N2; lane |= 8; }
        if (q >= N3) { q -= N3; lane |= 4; }
        if (q >= N4) { q -= N4; lane |= 2; }
        if (q >= N5) { q -= N5; lane |= 1; }
        v[j] = R::shfl(a5[0], lane);
    }
}
template <typename T, int N>
__device__ __forceinline__ void warp_red_lane0(typename Red<T>::V (&v)[N]) {
#if WARP_RED_SCATTER
    warp_red0<T, N>(v);
#else
    warp_red<T, N>(v);
#endif
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

// Per-lane vector width of the velocity loops: two consecutive velocities (8-byte
// loads) in mixed mode, one in FP64 mode.  Rows are padded to 32 velocities, so the
// vector accesses never leave a row and stay aligned.
template <typename T>
struct VW;
template <>
struct VW<float> {
    static constexpr int N = 2;
};
template <>
struct VW<double> {
    static constexpr int N = 1;
};
__device__ __forceinline__ void vload(const float* p, float (&x)[2]) {
    const float2 v = *reinterpret_cast<const float2*>(p);
    x[0] = v.x;
    x[1] = v.y;
}
__device__ __forceinline__ void vload(const float* p, float (&x)[4]) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
}
__device__ __forceinline__ void vstore(float* p, const float (&x)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(x[0], x[1], x[2], x[3]);
}
// streaming loads cached in L2 only (ld.global.cg): rows read once per pass leave the
// L1 lines of the velocity tables in place
__device__ __forceinline__ void vload_cg(const float* p, float (&x)[4]) {
    const float4 v = __ldcg(reinterpret_cast<const float4*>(p));
    x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
}
__device__ __forceinline__ void vload_cg(const float* p, float (&x)[2]) {
    const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
    x[0] = v.x; x[1] = v.y;
}
__device__ __forceinline__ void vload_cg(const float* p, float (&x)[1]) { x[0] = __ldcg(p); }
__device__ __forceinline__ void vload_cg(const double* p, double (&x)[1]) { x[0] = __ldcg(p); }
__device__ __forceinline__ void vload(const double* p, double (&x)[1]) { x[0] = *p; }
__device__ __forceinline__ void vload(const float* p, float (&x)[1]) { x[0] = *p; }
__device__ __forceinline__ void vstore(float* p, const float (&x)[1]) { *p = x[0]; }
__device__ __forceinline__ void vstore(float* p, const float (&x)[2]) {
    *reinterpret_cast<float2*>(p) = make_float2(x[0], x[1]);
}
__device__ __forceinline__ void vstore(double* p, const double (&x)[1]) { *p = x[0]; }
template <typename T, int NV>
__device__ __forceinline__ void vload_row(const T* p, T (&x)[NV]) {
#if FACE_CG
    vload_cg(p, x);
#else
    vload(p, x);
#endif
}

// ------------------------------------------------------------------------------------
// gas model
// ------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ double viscosity(const Dev<T>& c, double Ttr) {
    if (c.viscosity_law == 1)                                         // Eq. T_solve_mu_Sut
        return c.mu_ref * pow(Ttr / c.T_ref, 1.5) * (c.T_ref + c.sutherland_c) / (Ttr + c.sutherland_c);
    return c.mu_ref * pow(Ttr / c.T_ref, c.omega_vis);                 // Eq. T_solve_mu
}
// d ln mu / d ln T_tr of the viscosity law (for the adjoint)
template <typename T>
__device__ __forceinline__ double viscosity_slope(const Dev<T>& c, double Ttr) {
    if (c.viscosity_law == 1) return 1.5 - Ttr / (Ttr + c.sutherland_c);
    return c.omega_vis;
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
// gas parameter j (0 R, 1 Z, 2 mu_ref, 3 T_ref, 4 omega_vis, 5 omega0, 6 omega1,
// 7 delta) in arithmetic type S
template <typename S, typename T>
__device__ __forceinline__ S par(const Dev<T>& c, int j) {
    if constexpr (std::is_same<S, T>::value) {
        return c.tp[j];
    } else {
        const double v[8] = {c.R, c.Z, c.mu_ref, c.T_ref, c.omega_vis, c.omega0, c.omega1, c.delta};
        return (S)v[j];
    }
}

// the same law in the per-velocity arithmetic type S
template <typename S, typename T>
__device__ __forceinline__ S viscosity_T(const Dev<T>& c, S Ttr) {
    if (c.viscosity_law == 1) {
        const S Cs = (S)c.sutherland_c, Tr = par<S>(c, 3), x = Ttr / Tr;
        return par<S>(c, 2) * x * sqrt(x) * (Tr + Cs) / (Ttr + Cs);
    }
    return par<S>(c, 2) * pow(Ttr / par<S>(c, 3), par<S>(c, 4));
}

// The constants of one reduced Rykov equilibrium G+ = (1 - 1/Z) G_tr + G_rot / Z,
// H+ likewise (Eqs. eqdf_G* - eqdf_Rrot), with the weights 1 - 1/Z and 1/Z folded
// into the Maxwellians, the heat-flux factors into the q vectors and log2(e) into the
// exponents, so that eval_eq needs no more than one operation per factor:
//   e[0..2] U;  e[3..5] q_tr / (15 R T_tr p_tr);  e[6..8] q_rot
//   e[9]  (1 - 1/Z) rho (2 pi R T_tr)^-3/2;  e[10] -log2(e) / (2 R T_tr);  e[11] 1 / R T_tr
//   e[12] omega0 (R T_tr p_tr) / (R T p)  (ratio of the two heat-flux factors)
//   e[13] rho (2 pi R T)^-3/2 / Z;  e[14] -log2(e) / (2 R T);  e[15] 1 / R T
//   e[16] R T_rot;  e[17] R T;  e[18] R T_rot (1 - delta) / (R T_tr p_rot);
//   e[19] omega1 (1 - delta) / p;  e[20..22] unused (zero)
template <typename T, typename S>
__device__ void make_eq(const Dev<T>& c, S rho, const S* U, S Tq, S Ttr, S Trot, const S* qtr,
                        const S* qrot, S* e) {
    const S R = par<S>(c, 0), Z = par<S>(c, 1), om0 = par<S>(c, 5), om1 = par<S>(c, 6),
            del = par<S>(c, 7);
    const S RTtr = R * Ttr, RT = R * Tq, RTrot = R * Trot;
    const S ptr = rho * RTtr, p = rho * RT, prot = rho * RTrot;
    const S qf = S(1) / (S(15) * RTtr * ptr);
    for (int d = 0; d < 3; ++d) { e[d] = U[d]; e[3 + d] = qtr[d] * qf; e[6 + d] = qrot[d]; }
    const S l2e = S(1.4426950408889634);
    const S a = S(2.0 * PI) * RTtr;
    e[9] = (S(1) - S(1) / Z) * rho / (a * sqrt(a));
    e[10] = -l2e / (S(2) * RTtr);
    e[11] = S(1) / RTtr;
    e[12] = om0 * (RTtr * ptr) / (RT * p);
    const S b = S(2.0 * PI) * RT;
    e[13] = rho / (b * sqrt(b)) / Z;
    e[14] = -l2e / (S(2) * RT);
    e[15] = S(1) / RT;
    e[16] = RTrot;
    e[17] = RT;
    e[18] = RTrot * (S(1) - del) / (RTtr * prot);
    e[19] = om1 * (S(1) - del) / p;
    e[20] = e[21] = e[22] = S(0);
}

// G+ and H+ at velocity u from make_eq's constants:
//   G_tr = M_tr (1 + c.q_tr (c^2 / R T_tr - 5) / (15 R T_tr p_tr)), G_rot likewise at T
//   with omega0; H = R T_rot G_tr + R T G_rot + c.q_rot (weighted Maxwellian terms)
template <typename T>
__device__ __forceinline__ void eval_eq(const T* e, T ux, T uy, T uz, T& G, T& H) {
    const T cx = ux - e[0], cy = uy - e[1], cz = uz - e[2];
    const T c2 = cx * cx + cy * cy + cz * cz;
    const T cqt = cx * e[3] + cy * e[4] + cz * e[5];
    const T cqr = cx * e[6] + cy * e[7] + cz * e[8];
    const T mtr = e[9] * ex2(c2 * e[10]);
    const T m = e[13] * ex2(c2 * e[14]);
    const T Gtr = mtr + mtr * (cqt * (c2 * e[11] - T(5)));
    const T Grot = m + m * ((cqt * e[12]) * (c2 * e[15] - T(5)));
    G = Gtr + Grot;
    H = e[16] * Gtr + e[17] * Grot + cqr * (e[18] * mtr + e[19] * m);
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
    if (m < c.F) {
        c.fsT[m] = (T)c.fs[m];
        for (int r = 0; r < 3; ++r) c.fnT[r * c.F + m] = (T)c.fn[r * c.F + m];
    }
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
// per-slot records of the reconstruction, one 16-byte (mixed) or 32-byte (FP64)
// shared-memory load each
template <typename T>
struct alignas(4 * sizeof(T)) Q4 {
    T x, y, z, w;
};
#ifndef RECON_MINB
#define RECON_MINB 3         // mixed mode: 80 registers, three blocks of eight warps per SM
                             // (FP64: four blocks, 64 registers)
#endif
template <typename T, int WPB>
__global__ void __launch_bounds__(WPB * 32, sizeof(T) == 8 ? 4 : RECON_MINB) k_recon(Dev<T> c) {
    constexpr int NV = sizeof(T) == 8 ? 1 : RECON_NV;
    __shared__ Q4<T> s_A[WPB][MAXF];              // LSQ weight vector, s_ij
    __shared__ Q4<T> s_B[WPB][MAXF];              // x_f - x_i, s_ij
    __shared__ Q4<T> s_C[WPB][MAXF];              // face normal
    __shared__ int4 s_I[WPB][MAXF];               // neighbour, face, left side
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int i = blockIdx.x * WPB + w;
    if (i >= c.N) return;                         // whole warp
    const int s0 = c.slot_off[i], ns = c.slot_off[i + 1] - s0;
    if (lane < ns) {
        const int m = s0 + lane;
        const T sq = c.slot_sT[m];
        s_A[w][lane] = Q4<T>{c.slot_lsqT[m], c.slot_lsqT[c.nnz + m], c.slot_lsqT[2 * c.nnz + m], sq};
        s_B[w][lane] = Q4<T>{c.slot_dT[m], c.slot_dT[c.nnz + m], c.slot_dT[2 * c.nnz + m], sq};
        s_C[w][lane] = Q4<T>{c.slot_nT[m], c.slot_nT[c.nnz + m], c.slot_nT[2 * c.nnz + m], T(0)};
        s_I[w][lane] = make_int4(c.slot_nbr[m], c.slot_face[m], c.slot_left[m], 0);
    }
    __syncwarp();
    const T eps2 = (T)c.eps2[i];
    const int limiter = (int)c.iterp[1];
    const size_t NK = (size_t)c.N * c.Kp, FK = (size_t)c.F * c.Kp;
    const T* phg = c.phi + (size_t)i * c.Kp;
    const T* phh = c.phi + NK + (size_t)i * c.Kp;
    // the velocity loop; the face loops are not unrolled (a fully unrolled four-face
    // variant measured slower: more registers, fewer resident warps)
    auto body = [&]() {
        auto for_faces = [&](auto&& f) {
#pragma unroll 1
            for (int q = 0; q < ns; ++q) f(q);
        };
        for (int k0 = NV * lane; k0 < c.K; k0 += 32 * NV) {
            T pg[NV], ph[NV];
            vload(phg + k0, pg);
            vload(phh + k0, ph);
            T g[2][3][NV], dmax[2][NV], dmin[2][NV];
#pragma unroll
            for (int e = 0; e < NV; ++e)
                for (int fd = 0; fd < 2; ++fd) {
                    g[fd][0][e] = g[fd][1][e] = g[fd][2][e] = T(0);
                    dmax[fd][e] = dmin[fd][e] = T(0);
                }
            for_faces([&](int q) {
                const int j = s_I[w][q].x;
                if (j < 0) return;
                T xg[NV], xh[NV];
                vload(c.phi + (size_t)j * c.Kp + k0, xg);
                vload(c.phi + NK + (size_t)j * c.Kp + k0, xh);
                const Q4<T> A = s_A[w][q];
#pragma unroll
                for (int e = 0; e < NV; ++e) {
                    const T dg = xg[e] - pg[e], dh = xh[e] - ph[e];
                    g[0][0][e] += A.x * dg; g[0][1][e] += A.y * dg; g[0][2][e] += A.z * dg;
                    g[1][0][e] += A.x * dh; g[1][1][e] += A.y * dh; g[1][2][e] += A.z * dh;
                    dmax[0][e] = dg > dmax[0][e] ? dg : dmax[0][e]; dmin[0][e] = dg < dmin[0][e] ? dg : dmin[0][e];
                    dmax[1][e] = dh > dmax[1][e] ? dh : dmax[1][e]; dmin[1][e] = dh < dmin[1][e] ? dh : dmin[1][e];
                }
            });
            T L[2][NV];
#pragma unroll
            for (int e = 0; e < NV; ++e) L[0][e] = L[1][e] = (limiter == 2) ? T(0) : T(1);
            if (limiter == 3) {
                // frozen limiter values
                vload(c.lstore + (size_t)i * c.Kp + k0, L[0]);
                vload(c.lstore + NK + (size_t)i * c.Kp + k0, L[1]);
            } else if (limiter == 1 || limiter == 4) {
                // min over faces of Venkatakrishnan's psi(d1, d2), capped at 1, threshold
                // eps^2 phi_i^2 relative to the cell value (unlike the published absolute
                // eps^2, which diverged on the sphere).  psi < 1 needs
                // y = d2/d1 > 1/2, where psi decreases in y; so the minimum over the faces
                // with d2 > 0 is psi(Delta_max, max d2) and over d2 < 0 psi(Delta_min, min d2):
                // two evaluations instead of one per face (the same value up to rounding)
                T d2hi[2][NV], d2lo[2][NV];
#pragma unroll
                for (int e = 0; e < NV; ++e) d2hi[0][e] = d2hi[1][e] = d2lo[0][e] = d2lo[1][e] = T(0);
                for_faces([&](int q) {
                    const Q4<T> B = s_B[w][q];
#pragma unroll
                    for (int e = 0; e < NV; ++e)
#pragma unroll
                        for (int fd = 0; fd < 2; ++fd) {
                            const T d2 = g[fd][0][e] * B.x + g[fd][1][e] * B.y + g[fd][2][e] * B.z;
                            d2hi[fd][e] = d2 > d2hi[fd][e] ? d2 : d2hi[fd][e];
                            d2lo[fd][e] = d2 < d2lo[fd][e] ? d2 : d2lo[fd][e];
                        }
                });
#pragma unroll
                for (int e = 0; e < NV; ++e)
#pragma unroll
                    for (int fd = 0; fd < 2; ++fd) {
                        const T ph0 = fd == 0 ? pg[e] : ph[e];
                        const T ep = eps2 * ph0 * ph0;
                        T Lv = T(1);
#if RECON_BF
                        if constexpr (sizeof(T) == 4) {
                            // the same minimum without branches: both quotients are formed
                            // (their denominators are positive whenever they are selected)
                            const T a1 = dmax[fd][e], a2 = d2hi[fd][e];
                            const T b1 = dmin[fd][e], b2 = d2lo[fd][e];
                            const T ra = lim_div(a1 * a1 + ep + T(2) * a1 * a2, a1 * a1 + T(2) * a2 * a2 + a1 * a2 + ep);
                            const T rb = lim_div(b1 * b1 + ep + T(2) * b1 * b2, b1 * b1 + T(2) * b2 * b2 + b1 * b2 + ep);
                            Lv = (a2 > T(0) && ra < Lv) ? ra : Lv;
                            Lv = (b2 < T(0) && rb < Lv) ? rb : Lv;
                            L[fd][e] = Lv;
                            continue;
                        }
#endif
                        if (d2hi[fd][e] > T(0)) {
                            const T d1 = dmax[fd][e], d2 = d2hi[fd][e];
                            const T num = d1 * d1 + ep + T(2) * d1 * d2;
                            const T den = d1 * d1 + T(2) * d2 * d2 + d1 * d2 + ep;
                            if (num < den) Lv = lim_div(num, den);
                        }
                        if (d2lo[fd][e] < T(0)) {
                            const T d1 = dmin[fd][e], d2 = d2lo[fd][e];
                            const T num = d1 * d1 + ep + T(2) * d1 * d2;
                            const T den = d1 * d1 + T(2) * d2 * d2 + d1 * d2 + ep;
                            if (num < Lv * den) Lv = lim_div(num, den);
                        }
                        L[fd][e] = Lv;
                    }
                if (limiter == 4) {
                    vstore(c.lstore + (size_t)i * c.Kp + k0, L[0]);
                    vstore(c.lstore + NK + (size_t)i * c.Kp + k0, L[1]);
                }
            }
            T ux[NV], uy[NV], uz[NV];
            vload(c.uT + k0, ux);
            vload(c.uT + c.Kp + k0, uy);
            vload(c.uT + 2 * c.Kp + k0, uz);
            for_faces([&](int q) {
                const Q4<T> Cn = s_C[w][q], B = s_B[w][q];
                const int4 I = s_I[w][q];
                const bool left = I.z;
                const size_t o = (size_t)I.y * c.Kp + k0;
                T vg[NV], vh[NV];
                bool up[NV], all = true;
#pragma unroll
                for (int e = 0; e < NV; ++e) {
                    const T un = dot_rn(ux[e], uy[e], uz[e], Cn.x, Cn.y, Cn.z);
                    up[e] = left ? (un > T(0)) : (un <= T(0));
                    all = all && up[e];
                    const T rx = B.x - ux[e] * B.w, ry = B.y - uy[e] * B.w, rz = B.z - uz[e] * B.w;
                    vg[e] = pg[e] + L[0][e] * (g[0][0][e] * rx + g[0][1][e] * ry + g[0][2][e] * rz);
                    vh[e] = ph[e] + L[1][e] * (g[1][0][e] * rx + g[1][1][e] * ry + g[1][2][e] * rz);
                }
                if (all) {
                    vstore(c.face + o, vg);
                    vstore(c.face + FK + o, vh);
                } else {
#pragma unroll
                    for (int e = 0; e < NV; ++e)
                        if (up[e]) { c.face[o + e] = vg[e]; c.face[FK + o + e] = vh[e]; }
                }
            });
        }
    };
    body();
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
#ifndef FACE_MINB
#define FACE_MINB 3          // 80 registers, three blocks of eight warps per SM
#endif
// FW warps share one face (each takes every FW-th chunk of 32 x NV velocities; their
// partial sums are combined in a fixed order through shared memory), so that fewer
// faces are in flight and pass 2 finds the face rows of pass 1 still in L2.
template <typename T, int WPB, int FW>
__global__ void __launch_bounds__(WPB * 32, FACE_MINB) k_face_interior(Dev<T> c) {
    using R = Red<T>;
    using V = typename R::V;
    constexpr int NV = sizeof(T) == 8 ? 1 : FACE_NV;
    constexpr int FPB = WPB / FW;                // faces per block
    constexpr int NB = EQN + 2;
    __shared__ V s_v[FW > 1 ? FPB : 1][FW][17];
    __shared__ T s_cst[FW > 1 ? FPB : 1][NB];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int fib = wib / FW, sub = wib % FW;
    const int fi = blockIdx.x * FPB + fib;
    if (FW == 1 && fi >= c.Fi) return;           // whole warp: no block barriers below
    const bool active = fi < c.Fi;               // (FW > 1: every warp meets the barriers)
    const int f = active ? c.face_int[fi] : c.face_int[0];
    const size_t FK = (size_t)c.F * c.Kp;
    T* g0 = c.face + (size_t)f * c.Kp;
    T* h0 = c.face + FK + (size_t)f * c.Kp;
    // reference velocity U_r (any value is exact; the mean of the cells' U^n keeps
    // the shifted moments small)
    T Ur[3] = {T(0), T(0), T(0)};
    if (lane == 0 && active) {
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
        // compensated: the conserved moments (0-4); plain per-lane FP32 sums (<= K/32
        // terms each, then float-float across lanes): the second and third moments,
        // which only enter the heat-flux correction
        // NV consecutive velocities per lane (8-byte loads in mixed mode); their terms
        // are summed plainly, then added with compensation
        Acc<T> m[5];
        T p2[12];
#pragma unroll
        for (int j = 0; j < 12; ++j) p2[j] = T(0);
        for (int k0 = NV * (lane + 32 * sub); active && k0 < c.K; k0 += 32 * NV * FW) {
            T ux[NV], uy[NV], uz[NV], wv[NV], gv[NV], hv[NV], t[5];
            vload(c.uT + k0, ux);
            vload(c.uT + c.Kp + k0, uy);
            vload(c.uT + 2 * c.Kp + k0, uz);
            vload(c.wT + k0, wv);
            vload_row(g0 + k0, gv);
            vload_row(h0 + k0, hv);
#pragma unroll
            for (int e = 0; e < NV; ++e) {
                const T cx = ux[e] - Ur[0], cy = uy[e] - Ur[1], cz = uz[e] - Ur[2];
                const T wg = wv[e] * gv[e], wh = wv[e] * hv[e];
                const T tv[5] = {wg, wg * cx, wg * cy, wg * cz, wh};
#pragma unroll
                for (int j = 0; j < 5; ++j) t[j] = e == 0 ? tv[j] : t[j] + tv[j];
                p2[0] += wg * cx * cx; p2[1] += wg * cy * cy; p2[2] += wg * cz * cz;
                p2[3] += wg * cx * cy; p2[4] += wg * cx * cz; p2[5] += wg * cy * cz;
                const T wgc2 = wg * (cx * cx + cy * cy + cz * cz);
                p2[6] += wgc2 * cx; p2[7] += wgc2 * cy; p2[8] += wgc2 * cz;
                p2[9] += wh * cx; p2[10] += wh * cy; p2[11] += wh * cz;
            }
#pragma unroll
            for (int j = 0; j < 5; ++j) m[j].add(t[j]);
        }
#pragma unroll
        for (int j = 0; j < 5; ++j) v[j] = R::from(m[j]);
#pragma unroll
        for (int j = 0; j < 12; ++j) {
            Acc<T> t;
            t.add(p2[j]);
            v[5 + j] = R::from(t);
        }
    }
    warp_red_lane0<T, 17>(v);
    if constexpr (FW > 1) {
        if (lane == 0)
            for (int j = 0; j < 17; ++j) s_v[fib][sub][j] = v[j];
        __syncthreads();
        if (lane == 0 && sub == 0)
            for (int j = 0; j < 17; ++j) {
                V t = s_v[fib][0][j];
                for (int q = 1; q < FW; ++q) t = R::add(t, s_v[fib][q][j]);
                v[j] = t;
            }
    }
    // interface state on lane 0, in the per-velocity arithmetic type T (the moments
    // themselves are carried with compensation)
    T cst[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) cst[j] = T(0);
    if (lane == 0 && sub == 0 && active) {
        T x[17];
        for (int j = 0; j < 17; ++j) x[j] = (T)R::to_T(v[j]);
        const T Rg = par<T>(c, 0), Z = par<T>(c, 1), s = c.fsT[f];
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
        const T tau = viscosity_T<T>(c, Ttr0) / (rho * Rg * Ttr0);
        const T Erot = (Z * tau * Er0 + s * rho * Rg * Tq) / (Z * tau + s);
        const T Trot = Erot / (rho * Rg);
        const T Ttr = (etr + Er0 - Erot) / (T(1.5) * rho * Rg);
        // sum w c|c|^2 g and sum w c h about U = U_r + d (c = c' - d)
        const T Sd[3] = {x[5] * d[0] + x[8] * d[1] + x[9] * d[2],
                         x[8] * d[0] + x[6] * d[1] + x[10] * d[2],
                         x[9] * d[0] + x[10] * d[1] + x[7] * d[2]};
        const T dtr = tau + s - s / T(3) * (T(1) - T(1) / Z + par<T>(c, 5) / Z);
        const T drot = tau + s - s * (T(1) - par<T>(c, 7)) * (T(1) - T(1) / Z + par<T>(c, 6) / Z);
        T qtr[3], qrot[3];
        for (int k = 0; k < 3; ++k) {
            const T Qtr = x[11 + k] - T(2) * Sd[k] - tr * d[k] + T(2) * rho * dd * d[k];
            qtr[k] = tau * T(0.5) * Qtr / dtr;
            qrot[k] = tau * (x[14 + k] - d[k] * Er0) / drot;
        }
        make_eq(c, rho, U, Tq, Ttr, Trot, qtr, qrot, cst + 2);
        cst[0] = tau / (tau + s);
        cst[1] = s / (tau + s);
        if (c.debug) {
            double* st = c.fstate + (size_t)f * FST;
            st[0] = rho; st[1] = U[0]; st[2] = U[1]; st[3] = U[2];
            st[4] = Tq; st[5] = Ttr; st[6] = Trot; st[7] = tau;
            for (int k = 0; k < 3; ++k) { st[8 + k] = qtr[k]; st[11 + k] = qrot[k]; }
            st[14] = c.fs[f]; st[15] = 0.0;
        }
    }
    T e[NB];
    if constexpr (FW > 1) {
        if (lane == 0 && sub == 0)
            for (int j = 0; j < NB; ++j) s_cst[fib][j] = cst[j];
        __syncthreads();
#pragma unroll
        for (int j = 0; j < NB; ++j) e[j] = s_cst[fib][j];
    } else {
#pragma unroll
        for (int j = 0; j < NB; ++j) e[j] = __shfl_sync(0xffffffffu, cst[j], 0);
    }
    const T nx = c.fnT[f], ny = c.fnT[c.F + f], nz = c.fnT[2 * c.F + f];
    const T a = e[0], b = e[1];
    V r6[6];
    {
        Acc<T> m[6];
        for (int k0 = NV * (lane + 32 * sub); active && k0 < c.K; k0 += 32 * NV * FW) {
            T ux[NV], uy[NV], uz[NV], wv[NV], u2[NV], gv[NV], hv[NV], t[6];
            vload(c.uT + k0, ux);
            vload(c.uT + c.Kp + k0, uy);
            vload(c.uT + 2 * c.Kp + k0, uz);
            vload(c.wT + k0, wv);
#pragma unroll
            for (int q = 0; q < NV; ++q) u2[q] = T(0.5) * (ux[q] * ux[q] + uy[q] * uy[q] + uz[q] * uz[q]);
            vload_row(g0 + k0, gv);
            vload_row(h0 + k0, hv);
#pragma unroll
            for (int q = 0; q < NV; ++q) {
                T G, H;
                eval_eq(e + 2, ux[q], uy[q], uz[q], G, H);
#if FACE_PADSEL
                const bool pad = k0 + q >= c.K;
                const T gf = pad ? T(0) : a * gv[q] + b * G;
                const T hf = pad ? T(0) : a * hv[q] + b * H;
#else
                const T gf = a * gv[q] + b * G;
                const T hf = a * hv[q] + b * H;
#endif
                gv[q] = gf;
                hv[q] = hf;
                // zero weight in the K padding: no flux terms there
                const T wu = wv[q] * (ux[q] * nx + uy[q] * ny + uz[q] * nz);
                const T wg = wu * gf;
                const T tv[6] = {wg, wg * ux[q], wg * uy[q], wg * uz[q], wu * (u2[q] * gf + hf), wu * hf};
#pragma unroll
                for (int j = 0; j < 6; ++j) t[j] = q == 0 ? tv[j] : t[j] + tv[j];
            }
            if (!FACE_PADSEL && k0 + NV > c.K) {
                // the K padding keeps zero face values
#pragma unroll
                for (int q = 0; q < NV; ++q)
                    if (k0 + q >= c.K) gv[q] = hv[q] = T(0);
            }
            vstore(g0 + k0, gv);
            vstore(h0 + k0, hv);
#pragma unroll
            for (int j = 0; j < 6; ++j) m[j].add(t[j]);
        }
#pragma unroll
        for (int j = 0; j < 6; ++j) r6[j] = R::from(m[j]);
    }
    warp_red_lane0<T, 6>(r6);
    if constexpr (FW > 1) {
        if (lane == 0)
            for (int j = 0; j < 6; ++j) s_v[fib][sub][j] = r6[j];
        __syncthreads();
        if (lane == 0 && sub == 0 && active) {
            for (int d = 0; d < 6; ++d) {
                V t = s_v[fib][0][d];
                for (int q = 1; q < FW; ++q) t = R::add(t, s_v[fib][q][d]);
                R::store(c.mface + (size_t)f * 6 + d, t);
            }
        }
    } else {
        if (lane == 0)
            for (int d = 0; d < 6; ++d) R::store(c.mface + (size_t)f * 6 + d, r6[d]);
    }
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
        for (int d = 0; d < 6; ++d) {
            if (sizeof(T) == 8) {
                c.mface[(size_t)f * 6 + d] = v[d];
            } else {
                const float hi = (float)v[d];
                *reinterpret_cast<float2*>(c.mface + (size_t)f * 6 + d) = make_float2(hi, (float)(v[d] - (double)hi));
            }
        }
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
        for (int d = 0; d < 6; ++d) M[d] += sg * c.fa[f] * Red<T>::load(c.mface + 6 * (size_t)f + d);
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
// implicit-step factor and reconstruction order of the current iteration:
// cfl = min(cfl_imp, cfl_imp0 cfl_ramp^n) (cfl_imp if no ramp), first order for
// n < first_order_iters (the paper fixes neither the implicit step nor a start-up:
// both are parameters of this implementation)
template <typename T>
__global__ void k_iter_begin(Dev<T> c) {
    const double n = c.iterp[2];
    double cfl = c.cfl_imp;
    if (c.cfl_imp0 > 0.0 && c.cfl_ramp > 1.0) {
        const double r = c.cfl_imp0 * pow(c.cfl_ramp, n);
        cfl = r < c.cfl_imp ? r : c.cfl_imp;
    }
    c.iterp[0] = cfl;
    double mode = (n < (double)c.first_order_iters) ? 2.0 : (double)c.limiter;
    // limiter freezing (reading; see rk_params.limiter_freeze)
    if (mode == 1.0 && c.limiter_freeze > 0) {
        if (n >= (double)c.limiter_freeze) mode = 3.0;
        else if (n == (double)(c.limiter_freeze - 1)) mode = 4.0;
    }
    c.iterp[1] = mode;
}

template <typename T>
__global__ void k_macro_prep(Dev<T> c) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= c.N) return;
    const double cfl = c.iterp[0];
    const double iv = 1.0 / c.vol[i];
    double D = 1.0 / (cfl * c.dt[i]);
    const int ps = c.pos_off[c.cell_pos[i]];
    // the constant part of every point update: macro flux minus the neighbours' W^n
    // fluxes, over all interior neighbours (later sweeps) and over the lower-colour
    // ones only (the first forward sweep, where the others are still zero)
    double B[6], Bff[6];
    for (int q = 0; q < 6; ++q) B[q] = Bff[q] = c.macroF[6 * (size_t)i + q];
    const int col = c.colour[i];
    for (int m = c.slot_off[i]; m < c.slot_off[i + 1]; ++m) {
        const int f = c.slot_face[m], j = c.slot_nbr[m];
        const size_t mp = (size_t)(ps + m - c.slot_off[i]);
        const double A = c.fa[f] * iv;
        D += 0.5 * A * c.rf[f];
        c.sC[2 * mp] = 0.5 * A;
        c.sC[2 * mp + 1] = 0.5 * A * c.rf[f];
        if (j >= 0) {
            const double sg = c.slot_left[m] ? 1.0 : -1.0;
            double* G0 = c.sG0 + 6 * mp;
            euler_flux(c.W + 6 * (size_t)j, sg * c.fn[f], sg * c.fn[c.F + f], sg * c.fn[2 * c.F + f], G0);
            const bool lower = c.slot_ncol[m] < col;
            for (int q = 0; q < 6; ++q) {
                B[q] -= 0.5 * A * G0[q];
                if (lower) Bff[q] -= 0.5 * A * G0[q];
            }
        }
    }
    for (int q = 0; q < 6; ++q) {
        c.mB[12 * (size_t)i + q] = B[q];
        c.mB[12 * (size_t)i + 6 + q] = Bff[q];
    }
    const Prim p = prim_from_W(c.W + 6 * (size_t)i, c.R);
    const double izt = 1.0 / (c.Z * relax_time(c, p.rho, p.Ttr));
    if (i == 0) c.bar[0] = 0u;            // arrival count of the cooperative solve
    c.mDb[4 * (size_t)i] = 1.0 / D;
    c.mDb[4 * (size_t)i + 1] = 1.0 / (D + izt);
    c.mDb[4 * (size_t)i + 2] = izt;
    flux_prim(c.W + 6 * (size_t)i, c.mPc + 8 * (size_t)i);
    for (int q = 0; q < 6; ++q) c.dW[6 * (size_t)i + q] = 0.0;
}

// Launched with programmatic stream serialisation: each phase waits for the previous
// one to complete, its writes visible, before it reads anything (griddepcontrol.wait),
// and only then lets the next one be launched (griddepcontrol.launch_dependents), so
// that the launch latency of the next colour overlaps this one while at most one phase
// waits ahead.  Both are no-ops in a plain launch.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// One point update of the macro PR-SGS (Eq. implicit_mac_equ_fin) for every cell of
// one colour, one thread per cell:
//   dW~_i = [Res_i - sum_j (A/2V) ((G(W_j + dW~_j) - G(W_j)) - r dW~_j)] / D_i,
// the flux Jacobian applied matrix-free with the neighbours' cached flux
// primitives; rho~ R T~ of the rotational source from the cell's current iterate.
// An update whose predicted state is not admissible (rho, T_tr or T_rot not
// positive) is skipped.
// MACRO_LANES threads share one cell: each takes every MACRO_LANES-th face, and the
// partial sums are combined by a butterfly within the group (every lane of the group
// ends with the same bits, lane 0 stores).
#ifndef MACRO_LANES
#define MACRO_LANES 2
#endif
#ifndef MACRO_FINAL_ONE
#define MACRO_FINAL_ONE 0
#endif
template <typename T>
__device__ __forceinline__ void macro_point(const Dev<T>& c, int p, int i, int colour, int first_forward,
                                            int g) {
    // o = F - sum_j (A/2V) G_ij(W_j^n) + sum_j (A/2V) G_ij(W_j + dW~_j) - (A r/2V) dW~_j:
    // lane 0 starts from the per-cell constant part, every lane adds its faces
    double o[6] = {0, 0, 0, 0, 0, 0};
    if (g == 0) {
        const double* B = c.mB + 12 * (size_t)i + (first_forward ? 6 : 0);
#pragma unroll
        for (int q = 0; q < 6; ++q) o[q] = B[q];
    }
    for (int m = c.pos_off[p] + g; m < c.pos_off[p + 1]; m += MACRO_LANES) {
        const int j = c.pslot_nbr[m];
        if (j < 0 || (first_forward && c.pslot_ncol[m] > colour)) continue;
        // (A/2V) n: the flux coefficient is folded into the slot's normal
        const double nx = c.pslot_n[m], ny = c.pslot_n[c.nnz + m], nz = c.pslot_n[2 * c.nnz + m];
        // the iterate of neighbours is read through L2: in the cooperative solve it was
        // written by other blocks during this kernel
        double P[8], dWj[6];
#pragma unroll
        for (int q = 0; q < 8; ++q) P[q] = __ldcg(c.mPc + 8 * (size_t)j + q);
#pragma unroll
        for (int q = 0; q < 6; ++q) dWj[q] = __ldcg(c.dW + 6 * (size_t)j + q);
        // (A/2V) G_ij(W_j + dW_j): the Euler flux of the neighbour's current iterate
        const double Un = P[1] * nx + P[2] * ny + P[3] * nz;
        const double rU = P[0] * Un;
        o[0] += rU;
        o[1] += rU * P[1] + P[5] * nx;
        o[2] += rU * P[2] + P[5] * ny;
        o[3] += rU * P[3] + P[5] * nz;
        o[4] += P[4] * Un;
        o[5] += P[6] * Un;
        const double c2 = c.sC[2 * (size_t)m + 1];
#pragma unroll
        for (int q = 0; q < 6; ++q) o[q] -= c2 * dWj[q];
    }
    if (MACRO_LANES > 1) {
        const unsigned mask = MACRO_LANES == 32 ? 0xffffffffu
                                                : ((1u << MACRO_LANES) - 1u) << ((threadIdx.x & 31) & ~(MACRO_LANES - 1));
#pragma unroll
        for (int off = 1; off < MACRO_LANES; off <<= 1)
#pragma unroll
            for (int q = 0; q < 6; ++q) o[q] += __shfl_xor_sync(mask, o[q], off);
    }
#if MACRO_FINAL_ONE
    if (g != 0) return;                  // the update itself on one lane of the group
#endif
    const double* W = c.W + 6 * (size_t)i;
    // rho R T of the current iterate: its cached pressure p = (2/5)(rho E - 1/2 rho |U|^2)
    const double rRT = __ldcg(c.mPc + 8 * (size_t)i + 5);
    const double iD = c.mDb[4 * (size_t)i], iDr = c.mDb[4 * (size_t)i + 1], izt = c.mDb[4 * (size_t)i + 2];
    double cand[6];
    for (int q = 0; q < 5; ++q) cand[q] = -o[q] * iD;
    cand[5] = ((rRT - W[5]) * izt - o[5]) * iDr;
    double Wn[6], Pn[8];
    for (int q = 0; q < 6; ++q) Wn[q] = W[q] + cand[q];
    if (!flux_prim(Wn, Pn) || g != 0) return;
    double* dW = c.dW + 6 * (size_t)i;
    for (int q = 0; q < 6; ++q) __stcg(dW + q, cand[q]);
    for (int q = 0; q < 8; ++q) __stcg(c.mPc + 8 * (size_t)i + q, Pn[q]);
}

template <typename T>
__global__ void __launch_bounds__(128) k_macro_sweep(Dev<T> c, const int* col_cell, int lo, int n, int colour,
                                                     int first_forward) {
    // phases launched with programmatic stream serialisation (see pdl_wait)
    pdl_wait();
    pdl_launch_dependents();
    const int t = (blockIdx.x * blockDim.x + threadIdx.x) / MACRO_LANES;
    if (t >= n) return;                           // whole lane group
    macro_point(c, lo + t, col_cell[lo + t], colour, first_forward, (int)(threadIdx.x % MACRO_LANES));
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier of a cooperative launch (all blocks co-resident): a counter that
// only grows within one macro solve (k_macro_prep zeroes it); barrier number nb is
// passed when it reaches (nb + 1) blocks x grid (+ extra: a count that no block
// reaches, used by a test to make the wait run out).  The wait is bounded: thread 0
// reads the clock every 1024 polls and after limit_ns without the barrier opening
// records status bit 4 and stops waiting, so a failure returns RK_ETIMEOUT to the host
// instead of hanging the GPU (every other block gives up as soon as it sees the bit).
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned int* p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ bool grid_barrier(unsigned int* bar, int* status, unsigned int& nb,
                                             unsigned int extra, unsigned long long limit_ns) {
    __shared__ int s_fail;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int target = (nb + 1u) * gridDim.x + extra;
        int fail = 0;
        __threadfence();
        atomicAdd(bar, 1u);
        unsigned int polls = 0;
        unsigned long long t0 = 0;
        while (ld_acquire_gpu(bar) < target) {
            if ((++polls & 1023u) == 0u) {
                const unsigned long long t = global_ns();
                if (t0 == 0) t0 = t;
                else if (t - t0 > limit_ns || (*(volatile int*)status & 4)) {
                    atomicOr(status, 4);
                    fail = 1;
                    break;
                }
            }
        }
        __threadfence();
        s_fail = fail;
    }
    ++nb;
    __syncthreads();
    return s_fail == 0;
}

template <typename T>
__global__ void __launch_bounds__(128) k_macro_coop(Dev<T> c, const int* col_cell, const int* col_off,
                                                    int C, int n_macro, unsigned int* bar,
                                                    unsigned int extra, unsigned long long limit_ns) {
    const int stride = (gridDim.x * blockDim.x) / MACRO_LANES;
    const int gid = (blockIdx.x * blockDim.x + threadIdx.x) / MACRO_LANES;
    const int g = (int)(threadIdx.x % MACRO_LANES);
    unsigned int nb = 0;
    for (int it = 0; it < n_macro; ++it) {
        for (int dir = 0; dir < 2; ++dir) {
            for (int cc = 0; cc < C; ++cc) {
                const int col = dir == 0 ? cc : C - 1 - cc;
                const int lo = col_off[col], hi = col_off[col + 1];
                const int ff = (it == 0 && dir == 0);
                for (int t = lo + gid; t < hi; t += stride) macro_point(c, t, col_cell[t], col, ff, g);
                if (!grid_barrier(bar, c.status, nb, extra, limit_ns)) return;
            }
        }
    }
}

// ------------------------------------------------------------------------------------
// Macro PR-SGS in FP32, delta form (mixed contexts)
// ------------------------------------------------------------------------------------
// The same point updates as macro_point, with the flux difference
// G_ij(W_j + dW~_j) - G_ij(W_j^n) written in the increments themselves, so that FP32
// loses nothing to cancellation.  With m = rho U, H = rho E + p, U_n = U.n (n scaled
// by A/2V), ~ the current iterate and unmarked quantities those of W^n:
//   dG_0 = dm.n,   dG_d = dm_d U_n + m~_d dU_n + dp n_d   (d = x, y, z),
//   dG_4 = dH U_n + H~ dU_n,   dG_5 = d(rho E_rot) U_n + (rho E_rot)~ dU_n,
//   dU = (dm - U d rho) / rho~,   dp = (2/5) (d(rho E) - (dm.U + m~.dU) / 2).
// The constant part of every update, F_i (and for rho E_rot minus the source at W^n,
// (p - rho E_rot)/(Z tau)), is formed in FP64 and rounded once; it vanishes with the
// steady residual.  Every other FP32 rounding is relative to the increments, which
// vanish too, so the converged state is that of the FP64 solve, and each iterate
// differs from it by a relative 1e-6 or so of its own increment.
// Records, float4 views of the FP64 macro buffers (which this form leaves unused),
// indexed by the cell's colour position (cell_pos), so that a point update reads its
// own records without first loading its cell index and one colour's are contiguous:
//   base  [N][3] in mPc: (U, H) | (m, rho E_rot) | (rho, rho E, p, 1/(Z tau))   at W^n
//   delta [N][3] in mB:  (d rho, dm) | (d(rho E), d(rho E_rot), dp, 0) | (dU, 0)
//   own   [N][2] in mDb: (F_0..3) | (F_4, F_5 - (p - rho E_rot)/(Z tau), 1/D, 1/(D + 1/(Z tau)))
//   slot  [nnz]  in sG0: ((A/2V) n, A r/(2V)), position-ordered like pslot_nbr, then
//         [nnz] int2 after them: (neighbour's colour position or -1, its colour)
template <typename T>
__global__ void k_macro_prep32(Dev<T> c) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= c.N) return;
    const double cfl = c.iterp[0];
    const double iv = 1.0 / c.vol[i];
    double D = 1.0 / (cfl * c.dt[i]);
    const int pi = c.cell_pos[i], ps = c.pos_off[pi];
    float4* sl = reinterpret_cast<float4*>(c.sG0);
    int2* si = reinterpret_cast<int2*>(sl + c.nnz);
    for (int m = c.slot_off[i]; m < c.slot_off[i + 1]; ++m) {
        const int f = c.slot_face[m];
        const size_t mp = (size_t)(ps + m - c.slot_off[i]);
        const double c2 = 0.5 * c.fa[f] * iv * c.rf[f];
        D += c2;
        sl[mp] = make_float4((float)c.pslot_n[mp], (float)c.pslot_n[c.nnz + mp],
                             (float)c.pslot_n[2 * c.nnz + mp], (float)c2);
        const int j = c.pslot_nbr[mp];
        si[mp] = make_int2(j >= 0 ? c.cell_pos[j] : -1, c.pslot_ncol[mp]);
    }
    const double* W = c.W + 6 * (size_t)i;
    const Prim pr = prim_from_W(W, c.R);
    const double izt = 1.0 / (c.Z * relax_time(c, pr.rho, pr.Ttr));
    const double rho = W[0], ir = 1.0 / rho;
    const double U[3] = {W[1] * ir, W[2] * ir, W[3] * ir};
    const double p = 0.4 * (W[4] - 0.5 * rho * (U[0] * U[0] + U[1] * U[1] + U[2] * U[2]));
    const double* F = c.macroF + 6 * (size_t)i;
    float4* base = reinterpret_cast<float4*>(c.mPc) + 3 * (size_t)pi;
    base[0] = make_float4((float)U[0], (float)U[1], (float)U[2], (float)(W[4] + p));
    base[1] = make_float4((float)W[1], (float)W[2], (float)W[3], (float)W[5]);
    base[2] = make_float4((float)rho, (float)W[4], (float)p, (float)izt);
    float4* own = reinterpret_cast<float4*>(c.mDb) + 2 * (size_t)pi;
    own[0] = make_float4((float)F[0], (float)F[1], (float)F[2], (float)F[3]);
    own[1] = make_float4((float)F[4], (float)(F[5] - (p - W[5]) * izt), (float)(1.0 / D),
                         (float)(1.0 / (D + izt)));
    float4* dl = reinterpret_cast<float4*>(c.mB) + 3 * (size_t)pi;
    dl[0] = dl[1] = dl[2] = make_float4(0.f, 0.f, 0.f, 0.f);
}


// LN threads per cell, each taking every LN-th face, the partial sums combined by a
// butterfly (every lane of the group ends with the same bits; lane 0 stores).
template <typename T, int LN>
__global__ void __launch_bounds__(128) k_macro_sweep32(Dev<T> c, int lo, int n, int colour,
                                                       int first_forward) {
    pdl_wait();
    pdl_launch_dependents();
    const int t = (blockIdx.x * blockDim.x + threadIdx.x) / LN;
    if (t >= n) return;                           // whole lane group
    const int g = (int)(threadIdx.x % LN);
    const int p = lo + t;                         // colour position of the cell
    const float4* base = reinterpret_cast<const float4*>(c.mPc);
    const float4* own = reinterpret_cast<const float4*>(c.mDb);
    const float4* sl = reinterpret_cast<const float4*>(c.sG0);
    const int2* si = reinterpret_cast<const int2*>(sl + c.nnz);
    float4* dl = reinterpret_cast<float4*>(c.mB);
    float o[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (g == 0) {
        const float4 a = own[2 * (size_t)p], b = own[2 * (size_t)p + 1];
        o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w; o[4] = b.x; o[5] = b.y;
    }
    for (int m = c.pos_off[p] + g; m < c.pos_off[p + 1]; m += LN) {
        const int2 nb = si[m];
        const int j = nb.x;
        if (j < 0 || (first_forward && nb.y > colour)) continue;
        const float4 s = sl[m];
        // the neighbour's increments are read through L2 (written by earlier launches)
        const float4 d0 = __ldcg(dl + 3 * (size_t)j), d1 = __ldcg(dl + 3 * (size_t)j + 1),
                     d2 = __ldcg(dl + 3 * (size_t)j + 2);
        const float4 b0 = base[3 * (size_t)j], b1 = base[3 * (size_t)j + 1];
        const float Un = b0.x * s.x + b0.y * s.y + b0.z * s.z;
        const float dUn = d2.x * s.x + d2.y * s.y + d2.z * s.z;
        const float dH = d1.x + d1.z;
        o[0] += d0.y * s.x + d0.z * s.y + d0.w * s.z - s.w * d0.x;
        o[1] += d0.y * Un + (b1.x + d0.y) * dUn + d1.z * s.x - s.w * d0.y;
        o[2] += d0.z * Un + (b1.y + d0.z) * dUn + d1.z * s.y - s.w * d0.z;
        o[3] += d0.w * Un + (b1.z + d0.w) * dUn + d1.z * s.z - s.w * d0.w;
        o[4] += dH * Un + (b0.w + dH) * dUn - s.w * d1.x;
        o[5] += d1.y * Un + (b1.w + d1.y) * dUn - s.w * d1.y;
    }
    if (LN > 1) {
        const unsigned mask = LN == 32 ? 0xffffffffu : ((1u << LN) - 1u) << ((threadIdx.x & 31) & ~(LN - 1));
#pragma unroll
        for (int off = 1; off < LN; off <<= 1)
#pragma unroll
            for (int q = 0; q < 6; ++q) o[q] += __shfl_xor_sync(mask, o[q], off);
    }
    if (g != 0) return;
    const size_t i = (size_t)p;
    const float4 b0 = base[3 * i], b1 = base[3 * i + 1], b2 = base[3 * i + 2];
    const float4 ob = own[2 * i + 1];
    // dp of the current iterate: the implicit part of the rotational source
    const float dpi = __ldcg(reinterpret_cast<const float*>(dl + 3 * i + 1) + 2);
    float cand[6];
#pragma unroll
    for (int q = 0; q < 5; ++q) cand[q] = -o[q] * ob.z;
    cand[5] = (dpi * b2.w - o[5]) * ob.w;
    // the candidate iterate, skipped if not admissible (rho, T_tr or T_rot <= 0)
    const float rho = b2.x + cand[0];
    if (!(rho > 0.f)) return;
    const float mx = b1.x + cand[1], my = b1.y + cand[2], mz = b1.z + cand[3];
    const float dUx = (cand[1] - b0.x * cand[0]) / rho, dUy = (cand[2] - b0.y * cand[0]) / rho,
                dUz = (cand[3] - b0.z * cand[0]) / rho;
    const float dke = 0.5f * (cand[1] * b0.x + cand[2] * b0.y + cand[3] * b0.z + mx * dUx + my * dUy + mz * dUz);
    const float ke = 0.5f * (mx * (b0.x + dUx) + my * (b0.y + dUy) + mz * (b0.z + dUz));
    const float er = b1.w + cand[5];
    if (!((b2.y + cand[4]) - ke - er > 0.f && er > 0.f)) return;
    __stcg(dl + 3 * i, make_float4(cand[0], cand[1], cand[2], cand[3]));
    __stcg(dl + 3 * i + 1, make_float4(cand[4], cand[5], 0.4f * (cand[4] - dke), 0.f));
    __stcg(dl + 3 * i + 2, make_float4(dUx, dUy, dUz, 0.f));
}

// W~ = W^n + dW~, tau~ and the per-cell record of the micro sweeps: constants of the
// predicted equilibrium phi~* built from (W~, q^n) (reading: the prediction gives no
// heat flux, so the last Step-6 value is used), 1/tau~, and 1/dt + 1/tau~.  dW~ is
// the FP64 iterate, or with m32 the first six floats of the cell's FP32 delta record.
template <typename T>
__global__ void k_macro_finish(Dev<T> c, int m32) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= c.N) return;
    const double cfl = c.iterp[0];
    double* Wt = c.Wt + 6 * (size_t)i;
    const float* d32 = reinterpret_cast<const float*>(c.mB) + (m32 ? 12 * (size_t)c.cell_pos[i] : 0);
    for (int m = 0; m < 6; ++m)
        Wt[m] = c.W[6 * (size_t)i + m] + (m32 ? (double)d32[m] : c.dW[6 * (size_t)i + m]);
    const Prim p = prim_from_W(Wt, c.R);
    const double tau = relax_time(c, p.rho, p.Ttr);
    c.taut[i] = tau;
    const double* q = c.q + 6 * (size_t)i;
    double* e = c.ceq + (size_t)i * CEQ;
    make_eq(c, p.rho, p.U, p.T, p.Ttr, p.Trot, q, q + 3, e);
    e[23] = 1.0 / tau;
    e[24] = 1.0 / (cfl * c.dt[i]) + 1.0 / tau;
}

// Micro flux F_{i,k} = sum_j (A/V_i)(u_k . n_ij) phi_ij,k (Eq. implicit_mic_flux) of
// every cell, gathered from the face array into res (the first micro sweep turns it
// into the residual in place).  It needs only the face distributions, so it runs
// while the macro PR-SGS (which it does not touch) solves on another stream.  One warp
// per cell, faces in slot order.
template <typename T, int WPB>
__global__ void __launch_bounds__(WPB * 32) k_micro_flux(Dev<T> c) {
    // velocities per lane: 16-byte accesses in mixed mode
    constexpr int NV = sizeof(T) == 8 ? 1 : MICRO_FLUX_NV;
    __shared__ int s_face[WPB][MAXF];
    __shared__ T s_n[WPB][3][MAXF], s_AV[WPB][MAXF];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int i = blockIdx.x * WPB + w;
    if (i >= c.N) return;
    const int s0 = c.slot_off[i], ns = c.slot_off[i + 1] - s0;
    if (lane < ns) {
        const int m = s0 + lane;
        s_face[w][lane] = c.slot_face[m];
        const T sg = c.slot_left[m] ? T(1) : T(-1);
        s_n[w][0][lane] = sg * c.slot_nT[m];
        s_n[w][1][lane] = sg * c.slot_nT[c.nnz + m];
        s_n[w][2][lane] = sg * c.slot_nT[2 * c.nnz + m];
        s_AV[w][lane] = c.slot_AVT[m];
    }
    __syncwarp();
    const size_t NK = (size_t)c.N * c.Kp, FK = (size_t)c.F * c.Kp;
    const size_t oi = (size_t)i * c.Kp;
    for (int k0 = NV * lane; k0 < c.K; k0 += 32 * NV) {
        T ux[NV], uy[NV], uz[NV], Fg[NV], Fh[NV];
        vload(c.uT + k0, ux);
        vload(c.uT + c.Kp + k0, uy);
        vload(c.uT + 2 * c.Kp + k0, uz);
#pragma unroll
        for (int v = 0; v < NV; ++v) Fg[v] = Fh[v] = T(0);
#pragma unroll 1
        for (int q = 0; q < ns; ++q) {
            const T nx = s_n[w][0][q], ny = s_n[w][1][q], nz = s_n[w][2][q], AV = s_AV[w][q];
            T fg[NV], fh[NV];
            const size_t of = (size_t)s_face[w][q] * c.Kp + k0;
            vload(c.face + of, fg);
            vload(c.face + FK + of, fh);
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                const T un = dot_split(ux[v], uy[v], uz[v], nx, ny, nz);
                Fg[v] += AV * un * fg[v];
                Fh[v] += AV * un * fh[v];
            }
        }
        vstore(c.res + oi + k0, Fg);
        vstore(c.res + NK + oi + k0, Fh);
    }
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
// FIRST (forms Res; the first sweep is the forward one) and LAST (update and Step-6
// sums) are separate instantiations, so that the middle sweeps carry neither the
// face reads nor the twelve accumulators
// The part of one micro point update that follows the face loop (shared by both
// sweep kernels): Res (first sweep: from phi and the micro flux F, written in place of
// F), the increment dphi = (Res - offdiag) / D, and in the last sweep phi^{n+1} and
// the lane's Step-6 sums.  r0 holds F (first sweep) or Res (later sweeps).
template <typename T, int NV, bool FIRST, bool LAST>
__device__ __forceinline__ void micro_tail(const Dev<T>& c, const T* e, T itau, size_t oi, size_t NK, int k0,
                                           const T (&ux)[NV], const T (&uy)[NV], const T (&uz)[NV],
                                           const T (&D)[NV], const T (&og)[NV], const T (&oh)[NV],
                                           const T (&pg)[NV], const T (&ph)[NV], const T (&r0g)[NV],
                                           const T (&r0h)[NV], Acc<T> (&a)[12]) {
    constexpr bool first = FIRST, last = LAST;
    T G[NV], H[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        G[v] = H[v] = T(0);
        if (first || last) eval_eq(e, ux[v], uy[v], uz[v], G[v], H[v]);
    }
    T rg[NV], rh[NV];
    if (first) {
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            rg[v] = (G[v] - pg[v]) * itau - r0g[v];
            rh[v] = (H[v] - ph[v]) * itau - r0h[v];
        }
        vstore(c.res + oi + k0, rg);
        vstore(c.res + NK + oi + k0, rh);
    } else {
#pragma unroll
        for (int v = 0; v < NV; ++v) { rg[v] = r0g[v]; rh[v] = r0h[v]; }
    }
    T xg[NV], xh[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        const T iD = rcp(D[v]);
        xg[v] = (rg[v] - og[v]) * iD;
        xh[v] = (rh[v] - oh[v]) * iD;
        // the lane's last group can reach into the K padding, which must stay zero
        // (with nonzero increments there, the sphere run turned non-finite after
        // ~200 iterations once the last sweep also updated the padded phi)
        if (k0 + v >= c.K) xg[v] = xh[v] = T(0);
    }
    vstore(c.dphi + oi + k0, xg);
    vstore(c.dphi + NK + oi + k0, xh);
    if (last) {
        T g1[NV], h1[NV], wv[NV];
        vload(c.wT + k0, wv);
        // the lane's NV terms are summed plainly, then added with compensation
        T t[12];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            g1[v] = pg[v] + xg[v];
            h1[v] = ph[v] + xh[v];
            const T Dg = g1[v] - G[v], Dh = h1[v] - H[v];
            const T cx = ux[v] - e[0], cy = uy[v] - e[1], cz = uz[v] - e[2];
            const T c2 = cx * cx + cy * cy + cz * cz;
            const T wg = wv[v] * Dg, wh = wv[v] * Dh;
            const T wgc = wg * c2;
            const T tv[12] = {wg, wg * ux[v], wg * uy[v], wg * uz[v],
                              T(0.5) * (ux[v] * ux[v] + uy[v] * uy[v] + uz[v] * uz[v]) * wg + wh, wh,
                              wgc * cx, wgc * cy, wgc * cz, wh * cx, wh * cy, wh * cz};
#pragma unroll
            for (int j = 0; j < 12; ++j) t[j] = v == 0 ? tv[j] : t[j] + tv[j];
        }
#pragma unroll
        for (int j = 0; j < 12; ++j) a[j].add(t[j]);
        vstore(c.phi + oi + k0, g1);
        vstore(c.phi + NK + oi + k0, h1);
    }
}

template <typename T, int WPB, bool FIRST, bool LAST>
__global__ void __launch_bounds__(WPB * 32, sizeof(T) == 8 ? 2 : (LAST ? MICRO_LAST_MINB : (FIRST ? MICRO_FIRST_MINB : MICRO_MID_MINB)))
    k_micro_sweep(Dev<T> c, const int* cells, int ncells, int colour) {
    constexpr bool first = FIRST, last = LAST, first_forward = FIRST;
    using R = Red<T>;
    // velocities per lane: 16-byte accesses in the middle sweeps of the mixed mode
    constexpr int NV = sizeof(T) == 8 ? 1 : (FIRST ? MICRO_FIRST_NV : (LAST ? MICRO_LAST_NV : MICRO_MID_NV));
    // faces whose loads are issued together
    constexpr int PF = LAST ? MICRO_LAST_PF : MICRO_PF;
    __shared__ T s_e[WPB][EQN + 2];
    __shared__ Q4<T> s_NA[WPB][MAXF];             // signed outward normal, A/V
    __shared__ int2 s_NO[WPB][MAXF];              // neighbour, neighbour term used
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int t = blockIdx.x * WPB + w;
    if (t >= ncells) return;                      // whole warp: no block barriers below
    const int i = cells[t];
    const int s0 = c.slot_off[i], ns = c.slot_off[i + 1] - s0;
    if (lane < EQN + 2) s_e[w][lane] = (T)c.ceq[(size_t)i * CEQ + lane];
    if (lane < ns) {
        const int m = s0 + lane;
        const T sg = c.slot_left[m] ? T(1) : T(-1);
        s_NA[w][lane] = Q4<T>{sg * c.slot_nT[m], sg * c.slot_nT[c.nnz + m], sg * c.slot_nT[2 * c.nnz + m],
                              c.slot_AVT[m]};
        s_NO[w][lane] = make_int2(c.slot_nbr[m], (c.slot_nbr[m] >= 0) && !(first_forward && c.slot_ncol[m] > colour));
    }
    __syncwarp();
    const T* e = s_e[w];
    const T itau = e[EQN - 1], base = e[EQN];
    const size_t NK = (size_t)c.N * c.Kp, FK = (size_t)c.F * c.Kp;
    const size_t oi = (size_t)i * c.Kp;
    Acc<T> a[12];
    for (int k0 = NV * lane; k0 < c.K; k0 += 32 * NV) {
        T ux[NV], uy[NV], uz[NV];
        vload(c.uT + k0, ux);
        vload(c.uT + c.Kp + k0, uy);
        vload(c.uT + 2 * c.Kp + k0, uz);
        T D[NV], og[NV], oh[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) { D[q] = base; og[q] = oh[q] = T(0); }
        // faces in groups of PF: all loads of a group are issued before its arithmetic,
        // so that PF neighbour rows are in flight per thread (the accumulation order
        // over the faces is unchanged)
#pragma unroll 1
        for (int qb = 0; qb < ns; qb += PF) {
            T un[PF][NV], dg[PF][NV], dh[PF][NV], AVq[PF];
            bool okq[PF];
#pragma unroll
            for (int qq = 0; qq < PF; ++qq) {
                const int q = qb + qq;
                okq[qq] = false;
                if (q < ns) {
                    const Q4<T> NA = s_NA[w][q];
                    const int2 NO = s_NO[w][q];
                    AVq[qq] = NA.w;
                    bool neg = false;
#pragma unroll
                    for (int v = 0; v < NV; ++v) {
                        un[qq][v] = dot_split(ux[v], uy[v], uz[v], NA.x, NA.y, NA.z);
                        neg = neg || !(un[qq][v] > T(0));
                    }
                    okq[qq] = NO.y && neg;
                    if (okq[qq]) {
                        const size_t oj = (size_t)NO.x * c.Kp + k0;
                        vload(c.dphi + oj, dg[qq]);
                        vload(c.dphi + NK + oj, dh[qq]);
                    }
                }
            }
#pragma unroll
            for (int qq = 0; qq < PF; ++qq) {
                const int q = qb + qq;
                if (q >= ns) break;
                const T AV = AVq[qq];
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    if (un[qq][v] > T(0)) {
                        D[v] += AV * un[qq][v];
                    } else if (okq[qq]) {
                        og[v] += AV * un[qq][v] * dg[qq][v];
                        oh[v] += AV * un[qq][v] * dh[qq][v];
                    }
                }
            }
        }
        T pg[NV], ph[NV], r0g[NV], r0h[NV];
        if (first || last) {
            vload(c.phi + oi + k0, pg);
            vload(c.phi + NK + oi + k0, ph);
        }
        // F in the first sweep (k_micro_flux), Res in the later ones
        vload(c.res + oi + k0, r0g);
        vload(c.res + NK + oi + k0, r0h);
        micro_tail<T, NV, FIRST, LAST>(c, e, itau, oi, NK, k0, ux, uy, uz, D, og, oh, pg, ph, r0g, r0h, a);
    }
    if (last) {
        typename R::V v[12];
#pragma unroll
        for (int j = 0; j < 12; ++j) v[j] = R::from(a[j]);
        warp_red_lane0<T, 12>(v);
        if (lane == 0)
            for (int j = 0; j < 12; ++j) c.S[(size_t)i * 12 + j] = R::to_d(v[j]);
    }
}

// Asynchronous copies global -> shared (cp.async; completion per thread, counted by
// commit groups).  16-byte copies bypass L1 (.cg); smaller ones go through it (.ca).
template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    if constexpr (BYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(sa), "l"(gmem), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// The micro point update of k_micro_sweep with its row loads staged through shared
// memory: while a warp computes one chunk of 32 x NV velocities, the rows of the next
// chunk (the neighbours' dphi at the faces that have an inflow velocity in the lane's
// group, the cell's own phi and F/Res) are already in flight as asynchronous copies,
// double-buffered, so the loads do not wait in registers.  Every lane copies and
// reads back only its own NV values, so the copies need no barrier beyond the
// thread's own wait.  Same arithmetic in the same order as k_micro_sweep.
// Dynamic shared memory: WPB x 2 stages x (2 maxs + 4) rows x 32 lanes x NV values.
#ifndef MICRO_ST_WPB
#define MICRO_ST_WPB 4
#endif
template <typename T, bool FIRST, bool LAST>
__host__ __device__ constexpr int micro_nv() {
    return sizeof(T) == 8 ? 1 : (FIRST ? MICRO_FIRST_NV : (LAST ? MICRO_LAST_NV : MICRO_MID_NV));
}
template <typename T, int WPB, bool FIRST, bool LAST>
__global__ void __launch_bounds__(WPB * 32)
    k_micro_sweep_st(Dev<T> c, const int* cells, int ncells, int colour, int maxs) {
    constexpr bool first = FIRST, last = LAST, first_forward = FIRST;
    using R = Red<T>;
    constexpr int NV = micro_nv<T, FIRST, LAST>();
    constexpr int BY = NV * (int)sizeof(T);
    extern __shared__ __align__(16) unsigned char st_raw[];
    __shared__ T s_e[WPB][EQN + 2];
    __shared__ Q4<T> s_NA[WPB][MAXF];             // signed outward normal, A/V
    __shared__ int2 s_NO[WPB][MAXF];              // neighbour, neighbour term used
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int t = blockIdx.x * WPB + w;
    if (t >= ncells) return;                      // whole warp: no block barriers below
    const int i = cells[t];
    const int s0 = c.slot_off[i], ns = c.slot_off[i + 1] - s0;
    if (lane < EQN + 2) s_e[w][lane] = (T)c.ceq[(size_t)i * CEQ + lane];
    if (lane < ns) {
        const int m = s0 + lane;
        const T sg = c.slot_left[m] ? T(1) : T(-1);
        s_NA[w][lane] = Q4<T>{sg * c.slot_nT[m], sg * c.slot_nT[c.nnz + m], sg * c.slot_nT[2 * c.nnz + m],
                              c.slot_AVT[m]};
        s_NO[w][lane] = make_int2(c.slot_nbr[m], (c.slot_nbr[m] >= 0) && !(first_forward && c.slot_ncol[m] > colour));
    }
    __syncwarp();
    const T* e = s_e[w];
    const T itau = e[EQN - 1], base = e[EQN];
    const size_t NK = (size_t)c.N * c.Kp;
    const size_t oi = (size_t)i * c.Kp;
    const int nrow = 2 * maxs + 4;                // rows per stage: 2 per face, phi g/h, F|Res g/h
    T* buf = reinterpret_cast<T*>(st_raw) + (size_t)w * 2 * nrow * 32 * NV + (size_t)lane * NV;
    // this lane's slot of row r in stage st
    auto slot = [&](int st, int r) { return buf + (size_t)(st * nrow + r) * 32 * NV; };
    const int nch = (c.K + 32 * NV - 1) / (32 * NV);
    // issue the copies of chunk ch into stage st; returns the faces copied (bit mask)
    auto prefetch = [&](int ch, int st) -> unsigned {
        const int k0 = ch * 32 * NV + NV * lane;
        unsigned mk = 0u;
        if (k0 < c.K) {
            T ux[NV], uy[NV], uz[NV];
            vload(c.uT + k0, ux);
            vload(c.uT + c.Kp + k0, uy);
            vload(c.uT + 2 * c.Kp + k0, uz);
#pragma unroll 1
            for (int q = 0; q < ns; ++q) {
                const int2 NO = s_NO[w][q];
                if (!NO.y) continue;
                const Q4<T> NA = s_NA[w][q];
                bool neg = false;
#pragma unroll
                for (int v = 0; v < NV; ++v) neg = neg || !(dot_split(ux[v], uy[v], uz[v], NA.x, NA.y, NA.z) > T(0));
                if (neg) {
                    const size_t oj = (size_t)NO.x * c.Kp + k0;
                    cp_async<BY>(slot(st, 2 * q), c.dphi + oj);
                    cp_async<BY>(slot(st, 2 * q + 1), c.dphi + NK + oj);
                    mk |= 1u << q;
                }
            }
            if (first || last) {
                cp_async<BY>(slot(st, 2 * maxs), c.phi + oi + k0);
                cp_async<BY>(slot(st, 2 * maxs + 1), c.phi + NK + oi + k0);
            }
            cp_async<BY>(slot(st, 2 * maxs + 2), c.res + oi + k0);
            cp_async<BY>(slot(st, 2 * maxs + 3), c.res + NK + oi + k0);
        }
        cp_async_commit();
        return mk;
    };
    Acc<T> a[12];
    unsigned m_next = prefetch(0, 0);
    for (int ch = 0; ch < nch; ++ch) {
        const int st = ch & 1;
        const unsigned m_cur = m_next;
        if (ch + 1 < nch) m_next = prefetch(ch + 1, st ^ 1);
        else cp_async_commit();                   // an empty group keeps the count
        cp_async_wait<1>();                       // this thread's copies of chunk ch are done
        const int k0 = ch * 32 * NV + NV * lane;
        if (k0 >= c.K) continue;
        T ux[NV], uy[NV], uz[NV];
        vload(c.uT + k0, ux);
        vload(c.uT + c.Kp + k0, uy);
        vload(c.uT + 2 * c.Kp + k0, uz);
        T D[NV], og[NV], oh[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) { D[q] = base; og[q] = oh[q] = T(0); }
#pragma unroll 1
        for (int q = 0; q < ns; ++q) {
            const Q4<T> NA = s_NA[w][q];
            T un[NV], dg[NV], dh[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) un[v] = dot_split(ux[v], uy[v], uz[v], NA.x, NA.y, NA.z);
            const bool okq = (m_cur >> q) & 1u;
            if (okq) {
                vload(slot(st, 2 * q), dg);
                vload(slot(st, 2 * q + 1), dh);
            }
            const T AV = NA.w;
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                if (un[v] > T(0)) {
                    D[v] += AV * un[v];
                } else if (okq) {
                    og[v] += AV * un[v] * dg[v];
                    oh[v] += AV * un[v] * dh[v];
                }
            }
        }
        T pg[NV], ph[NV], r0g[NV], r0h[NV];
        if (first || last) {
            vload(slot(st, 2 * maxs), pg);
            vload(slot(st, 2 * maxs + 1), ph);
        }
        vload(slot(st, 2 * maxs + 2), r0g);
        vload(slot(st, 2 * maxs + 3), r0h);
        micro_tail<T, NV, FIRST, LAST>(c, e, itau, oi, NK, k0, ux, uy, uz, D, og, oh, pg, ph, r0g, r0h, a);
    }
    cp_async_wait<0>();
    if (last) {
        typename R::V v[12];
#pragma unroll
        for (int j = 0; j < 12; ++j) v[j] = R::from(a[j]);
        warp_red_lane0<T, 12>(v);
        if (lane == 0)
            for (int j = 0; j < 12; ++j) c.S[(size_t)i * 12 + j] = R::to_d(v[j]);
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
        c.iterp[2] += 1.0;              // end of the implicit iteration
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

// Wall loads per wall face (the lift, drag and pitching-moment integrals of Sec. 4):
// A_f m_f and A_f (x_f - x_ref) x m_f, with m_f = sum_k w (u.n) u g_f the wall
// momentum flux that the boundary-face kernel leaves in wallq[1..3].
template <typename T>
__global__ void k_aero(Dev<T> c, const int* wall_b, int nw, double x0, double y0, double z0,
                       double* contrib) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nw) return;
    const int b = wall_b[t];
    const int f = c.face_bnd[b];
    const double* wq = c.wallq + 8 * (size_t)b;
    const double A = c.fa[f];
    const double m[3] = {A * wq[1], A * wq[2], A * wq[3]};
    const double r[3] = {c.fxc[f] - x0, c.fxc[c.F + f] - y0, c.fxc[2 * c.F + f] - z0};
    double* cb = contrib + 6 * (size_t)t;
    cb[0] = m[0]; cb[1] = m[1]; cb[2] = m[2];
    cb[3] = r[1] * m[2] - r[2] * m[1];
    cb[4] = r[2] * m[0] - r[0] * m[2];
    cb[5] = r[0] * m[1] - r[1] * m[0];
}

static __global__ void __launch_bounds__(256) k_sum6(const double* contrib, int n, double* tot) {
    __shared__ double red[6 * 8];
    double v[6] = {0, 0, 0, 0, 0, 0};
    for (int i = threadIdx.x; i < n; i += 256)
        for (int j = 0; j < 6; ++j) v[j] += contrib[6 * (size_t)i + j];
    block_sum<6, 256>(v, red);
    if (threadIdx.x == 0)
        for (int j = 0; j < 6; ++j) tot[j] = v[j];
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
