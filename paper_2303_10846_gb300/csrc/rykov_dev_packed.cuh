// Mixed-precision kernels on the packed FP32 pipe of sm_100-class GPUs: every FP32
// add, multiply and fused multiply-add of the per-velocity arithmetic operates on a
// pair of consecutive velocities (one instruction for two values, each rounded as
// its scalar counterpart), which halves the issue slots of these issue-bound kernels.
// Same steps and equations as the scalar kernels of rykov_dev.cuh; the summation
// order over the velocities differs (two interleaved compensated sums per lane,
// combined at the end).
#pragma once

#include "rykov_dev.cuh"

namespace rk {

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// a - b, one rounding (b * -1 is exact)
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float hsum(float2 a) { return __fadd_rn(a.x, a.y); }

// Kahan-compensated FP32 sums of two interleaved sequences (the .x and .y halves),
// each exactly Acc<float>; get() combines the halves as float-float pairs.
struct Acc2 {
    float2 s = {0.f, 0.f}, c = {0.f, 0.f};
    __device__ __forceinline__ void add(float2 x) {
        const float2 y = sub2(x, c);
        const float2 t = add2(s, y);
        c = sub2(sub2(t, s), y);
        s = t;
    }
    __device__ __forceinline__ FF get() const { return ff_add(ff_norm(s.x, -c.x), ff_norm(s.y, -c.y)); }
};
// a plain packed sum turned into a float-float pair
__device__ __forceinline__ FF ff_of(float2 a) { return ff_add(FF{a.x, 0.f}, FF{a.y, 0.f}); }

// The reduced Rykov equilibria G*, R* (Eqs. eqdf_G* - eqdf_Rrot) at two velocities,
// from the constants of make_eq (eval_eq's arithmetic, packed).
__device__ __forceinline__ void eval_eq2(const float* e, float2 ux, float2 uy, float2 uz, float2& G,
                                         float2& H) {
    const float2 cx = sub2(ux, f2(e[0])), cy = sub2(uy, f2(e[1])), cz = sub2(uz, f2(e[2]));
    const float2 c2 = fma2(cz, cz, fma2(cy, cy, mul2(cx, cx)));
    const float2 cqt = fma2(cz, f2(e[5]), fma2(cy, f2(e[4]), mul2(cx, f2(e[3]))));
    const float2 cqr = fma2(cz, f2(e[8]), fma2(cy, f2(e[7]), mul2(cx, f2(e[6]))));
    const float2 a1 = mul2(c2, f2(e[10])), a2 = mul2(c2, f2(e[14]));
    const float2 mtr = mul2(f2(e[9]), make_float2(ex2(a1.x), ex2(a1.y)));
    const float2 m = mul2(f2(e[13]), make_float2(ex2(a2.x), ex2(a2.y)));
    const float2 Gtr = fma2(mtr, mul2(cqt, fma2(c2, f2(e[11]), f2(-5.f))), mtr);
    const float2 Grot = fma2(m, mul2(mul2(cqt, f2(e[12])), fma2(c2, f2(e[15]), f2(-5.f))), m);
    G = add2(Gtr, Grot);
    H = fma2(cqr, fma2(f2(e[18]), mtr, mul2(f2(e[19]), m)), fma2(f2(e[16]), Gtr, mul2(f2(e[17]), Grot)));
}

// ------------------------------------------------------------------------------------
// Step 2 (a), mixed precision on the packed pipe: least-squares gradient,
// Venkatakrishnan limiter and reconstruction phi(x_ij - u_k s_ij) = phi_c +
// (x_ij - u_k s_ij - x_c) . L grad phi_c written by the upwind cell c (Eq.
// flux_solve_phi_phi).  The steps of k_recon (one warp per cell, four velocities per
// lane, the limiter's two candidate quotients formed without branches); u.n of the
// upwind choice is rounded product by product, as in the scalar kernels.
// ------------------------------------------------------------------------------------
// Two blocks of eight warps per SM (up to 128 registers) with the face loops taken in
// pairs: measured at scale 41.6 ms against 41.9 ms for three blocks with single faces
// (paired loops spill at three blocks: 43.3 ms; single faces at two blocks: 46.1 ms)
#ifndef RECONP_MINB
#define RECONP_MINB 2
#endif
__device__ __forceinline__ float2 max2(float2 a, float2 b) { return make_float2(fmaxf(a.x, b.x), fmaxf(a.y, b.y)); }
__device__ __forceinline__ float2 min2(float2 a, float2 b) { return make_float2(fminf(a.x, b.x), fminf(a.y, b.y)); }
// three-input max / min (PTX max.f32 / min.f32 with three sources, sm_100+): two
// faces' values folded into a running extreme per instruction
__device__ __forceinline__ float max3f(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ float min3f(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ float2 max3_2(float2 a, float2 b, float2 c) {
    return make_float2(max3f(a.x, b.x, c.x), max3f(a.y, b.y, c.y));
}
__device__ __forceinline__ float2 min3_2(float2 a, float2 b, float2 c) {
    return make_float2(min3f(a.x, b.x, c.x), min3f(a.y, b.y, c.y));
}
#ifndef RECONP_PAIRS
#define RECONP_PAIRS 3       // bit 0: limiter loop, bit 1: neighbour loop over face pairs
#endif
// the limiter's quotient a/b (b > 0 where it is used): approximate division, with
// both operands scaled by 2^64 where b < 1e-30 (the approximate reciprocal overflows
// below ~1e-38)
__device__ __forceinline__ float lim_q(float a, float b) {
    const float sc = b < 1e-30f ? 18446744073709551616.0f : 1.0f;
    return __fdividef(a * sc, b * sc);
}
template <int WPB>
__global__ void __launch_bounds__(WPB * 32, RECONP_MINB) k_recon_p(Dev<float> c) {
    __shared__ float4 s_A[WPB][MAXF];             // LSQ weight vector, s_ij
    __shared__ float4 s_B[WPB][MAXF];             // x_f - x_i, s_ij
    __shared__ float4 s_C[WPB][MAXF];             // face normal
    __shared__ int4 s_I[WPB][MAXF];               // neighbour, face, left side
    __shared__ int2 s_J[WPB][MAXF];               // slots with a neighbour: (neighbour, slot)
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int i = blockIdx.x * WPB + w;
    if (i >= c.N) return;                         // whole warp
    const int s0 = c.slot_off[i], ns = c.slot_off[i + 1] - s0;
    if (lane < ns) {
        const int m = s0 + lane;
        const float sq = c.slot_sT[m];
        s_A[w][lane] = make_float4(c.slot_lsqT[m], c.slot_lsqT[c.nnz + m], c.slot_lsqT[2 * c.nnz + m], sq);
        s_B[w][lane] = make_float4(c.slot_dT[m], c.slot_dT[c.nnz + m], c.slot_dT[2 * c.nnz + m], sq);
        s_C[w][lane] = make_float4(c.slot_nT[m], c.slot_nT[c.nnz + m], c.slot_nT[2 * c.nnz + m], 0.f);
        s_I[w][lane] = make_int4(c.slot_nbr[m], c.slot_face[m], c.slot_left[m], 0);
    }
    // the slots with a neighbour cell, in slot order: (neighbour, slot)
    const bool hasn = lane < ns && c.slot_nbr[s0 + lane] >= 0;
    const unsigned bal = __ballot_sync(0xffffffffu, hasn);
    const int nn = __popc(bal);
    if (hasn) s_J[w][__popc(bal & ((1u << lane) - 1u))] = make_int2(c.slot_nbr[s0 + lane], lane);
    __syncwarp();
    const float eps2 = (float)c.eps2[i];
    const int limiter = (int)c.iterp[1];
    const size_t NK = (size_t)c.N * c.Kp, FK = (size_t)c.F * c.Kp;
    const float* phg = c.phi + (size_t)i * c.Kp;
    const float* phh = c.phi + NK + (size_t)i * c.Kp;
    for (int k0 = 4 * lane; k0 < c.K; k0 += 128) {
        const float4 pg4 = *reinterpret_cast<const float4*>(phg + k0);
        const float4 ph4 = *reinterpret_cast<const float4*>(phh + k0);
        const float2 pv[2][2] = {{lo2(pg4), hi2(pg4)}, {lo2(ph4), hi2(ph4)}};   // [field][pair]
        float2 g[2][3][2], dmax[2][2], dmin[2][2];                                 // [field][..][pair]
#pragma unroll
        for (int fd = 0; fd < 2; ++fd)
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                g[fd][0][p] = g[fd][1][p] = g[fd][2][p] = f2(0.f);
                dmax[fd][p] = dmin[fd][p] = f2(0.f);
            }
        // gradient sums in slot order; Delta_max/min over the neighbours (exact, any order)
        int qn = 0;
        if (RECONP_PAIRS & 2) {
#pragma unroll 1
            for (; qn + 1 < nn; qn += 2) {
                const int2 J0 = s_J[w][qn], J1 = s_J[w][qn + 1];
                const float4 xg0 = *reinterpret_cast<const float4*>(c.phi + (size_t)J0.x * c.Kp + k0);
                const float4 xh0 = *reinterpret_cast<const float4*>(c.phi + NK + (size_t)J0.x * c.Kp + k0);
                const float4 xg1 = *reinterpret_cast<const float4*>(c.phi + (size_t)J1.x * c.Kp + k0);
                const float4 xh1 = *reinterpret_cast<const float4*>(c.phi + NK + (size_t)J1.x * c.Kp + k0);
                const float4 A0 = s_A[w][J0.y], A1 = s_A[w][J1.y];
#pragma unroll
                for (int fd = 0; fd < 2; ++fd)
#pragma unroll
                    for (int p = 0; p < 2; ++p) {
                        const float4 x0 = fd ? xh0 : xg0, x1 = fd ? xh1 : xg1;
                        const float2 d0 = sub2(p ? hi2(x0) : lo2(x0), pv[fd][p]);
                        const float2 d1 = sub2(p ? hi2(x1) : lo2(x1), pv[fd][p]);
                        g[fd][0][p] = fma2(f2(A1.x), d1, fma2(f2(A0.x), d0, g[fd][0][p]));
                        g[fd][1][p] = fma2(f2(A1.y), d1, fma2(f2(A0.y), d0, g[fd][1][p]));
                        g[fd][2][p] = fma2(f2(A1.z), d1, fma2(f2(A0.z), d0, g[fd][2][p]));
                        dmax[fd][p] = max3_2(dmax[fd][p], d0, d1);
                        dmin[fd][p] = min3_2(dmin[fd][p], d0, d1);
                    }
            }
        }
#pragma unroll 1
        for (; qn < nn; ++qn) {
            const int2 J = s_J[w][qn];
            const float4 xg4 = *reinterpret_cast<const float4*>(c.phi + (size_t)J.x * c.Kp + k0);
            const float4 xh4 = *reinterpret_cast<const float4*>(c.phi + NK + (size_t)J.x * c.Kp + k0);
            const float4 A = s_A[w][J.y];
            const float2 Ax = f2(A.x), Ay = f2(A.y), Az = f2(A.z);
#pragma unroll
            for (int fd = 0; fd < 2; ++fd)
#pragma unroll
                for (int p = 0; p < 2; ++p) {
                    const float4 x4 = fd ? xh4 : xg4;
                    const float2 dv = sub2(p ? hi2(x4) : lo2(x4), pv[fd][p]);
                    g[fd][0][p] = fma2(Ax, dv, g[fd][0][p]);
                    g[fd][1][p] = fma2(Ay, dv, g[fd][1][p]);
                    g[fd][2][p] = fma2(Az, dv, g[fd][2][p]);
                    dmax[fd][p] = max2(dv, dmax[fd][p]);
                    dmin[fd][p] = min2(dv, dmin[fd][p]);
                }
        }
        float2 L[2][2];
#pragma unroll
        for (int fd = 0; fd < 2; ++fd)
#pragma unroll
            for (int p = 0; p < 2; ++p) L[fd][p] = f2(limiter == 2 ? 0.f : 1.f);
        if (limiter == 3) {
            const float4 l0 = *reinterpret_cast<const float4*>(c.lstore + (size_t)i * c.Kp + k0);
            const float4 l1 = *reinterpret_cast<const float4*>(c.lstore + NK + (size_t)i * c.Kp + k0);
            L[0][0] = lo2(l0); L[0][1] = hi2(l0); L[1][0] = lo2(l1); L[1][1] = hi2(l1);
        } else if (limiter == 1 || limiter == 4) {
            // min over faces of Venkatakrishnan's psi(d1, d2), capped at 1, threshold
            // eps^2 phi_i^2 (relative to the cell value, unlike the published absolute
            // eps^2, which diverged on the sphere); with d2 the gradient change to each face
            // centroid, psi < 1 needs d2/d1 > 1/2 where psi decreases in d2/d1, so the
            // minimum is psi(Delta_max, max d2) over d2 > 0 and psi(Delta_min, min d2)
            // over d2 < 0
            float2 d2hi[2][2], d2lo[2][2];
#pragma unroll
            for (int fd = 0; fd < 2; ++fd)
#pragma unroll
                for (int p = 0; p < 2; ++p) d2hi[fd][p] = d2lo[fd][p] = f2(0.f);
            int qb = 0;
            if (RECONP_PAIRS & 1) {
#pragma unroll 1
                for (; qb + 1 < ns; qb += 2) {
                    const float4 B0 = s_B[w][qb], B1 = s_B[w][qb + 1];
#pragma unroll
                    for (int fd = 0; fd < 2; ++fd)
#pragma unroll
                        for (int p = 0; p < 2; ++p) {
                            const float2 e0 = fma2(g[fd][2][p], f2(B0.z), fma2(g[fd][1][p], f2(B0.y), mul2(g[fd][0][p], f2(B0.x))));
                            const float2 e1 = fma2(g[fd][2][p], f2(B1.z), fma2(g[fd][1][p], f2(B1.y), mul2(g[fd][0][p], f2(B1.x))));
                            d2hi[fd][p] = max3_2(d2hi[fd][p], e0, e1);
                            d2lo[fd][p] = min3_2(d2lo[fd][p], e0, e1);
                        }
                }
            }
#pragma unroll 1
            for (; qb < ns; ++qb) {
                const float4 B = s_B[w][qb];
                const float2 Bx = f2(B.x), By = f2(B.y), Bz = f2(B.z);
#pragma unroll
                for (int fd = 0; fd < 2; ++fd)
#pragma unroll
                    for (int p = 0; p < 2; ++p) {
                        const float2 d2 = fma2(g[fd][2][p], Bz, fma2(g[fd][1][p], By, mul2(g[fd][0][p], Bx)));
                        d2hi[fd][p] = max2(d2, d2hi[fd][p]);
                        d2lo[fd][p] = min2(d2, d2lo[fd][p]);
                    }
            }
            const float2 two = f2(2.f), ep2 = f2(eps2);
#pragma unroll
            for (int fd = 0; fd < 2; ++fd)
#pragma unroll
                for (int p = 0; p < 2; ++p) {
                    const float2 ep = mul2(mul2(ep2, pv[fd][p]), pv[fd][p]);
                    const float2 a1 = dmax[fd][p], a2 = d2hi[fd][p], b1 = dmin[fd][p], b2 = d2lo[fd][p];
                    // numerators d1^2 + eps + 2 d1 d2 and denominators d1^2 + 2 d2^2 + d1 d2 + eps
                    const float2 a11 = fma2(a1, a1, ep), b11 = fma2(b1, b1, ep);
                    const float2 na = fma2(mul2(two, a1), a2, a11);
                    const float2 da = fma2(a1, a2, fma2(mul2(two, a2), a2, a11));
                    const float2 nb = fma2(mul2(two, b1), b2, b11);
                    const float2 db = fma2(b1, b2, fma2(mul2(two, b2), b2, b11));
                    float2 Lv = f2(1.f);
                    const float rax = lim_q(na.x, da.x), ray = lim_q(na.y, da.y);
                    const float rbx = lim_q(nb.x, db.x), rby = lim_q(nb.y, db.y);
                    Lv.x = (a2.x > 0.f && rax < Lv.x) ? rax : Lv.x;
                    Lv.y = (a2.y > 0.f && ray < Lv.y) ? ray : Lv.y;
                    Lv.x = (b2.x < 0.f && rbx < Lv.x) ? rbx : Lv.x;
                    Lv.y = (b2.y < 0.f && rby < Lv.y) ? rby : Lv.y;
                    L[fd][p] = Lv;
                }
            if (limiter == 4) {
                *reinterpret_cast<float4*>(c.lstore + (size_t)i * c.Kp + k0) =
                    make_float4(L[0][0].x, L[0][0].y, L[0][1].x, L[0][1].y);
                *reinterpret_cast<float4*>(c.lstore + NK + (size_t)i * c.Kp + k0) =
                    make_float4(L[1][0].x, L[1][0].y, L[1][1].x, L[1][1].y);
            }
        }
        const float4 ux4 = *reinterpret_cast<const float4*>(c.uT + k0);
        const float4 uy4 = *reinterpret_cast<const float4*>(c.uT + c.Kp + k0);
        const float4 uz4 = *reinterpret_cast<const float4*>(c.uT + 2 * c.Kp + k0);
        const float2 ux[2] = {lo2(ux4), hi2(ux4)}, uy[2] = {lo2(uy4), hi2(uy4)}, uz[2] = {lo2(uz4), hi2(uz4)};
#pragma unroll 1
        for (int q = 0; q < ns; ++q) {
            const float4 Cn = s_C[w][q], B = s_B[w][q];
            const int4 I = s_I[w][q];
            const bool left = I.z;
            const size_t o = (size_t)I.y * c.Kp + k0;
            float2 vg[2], vh[2];
            bool up[4], all = true;
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                // u.n with each product and sum rounded separately (the oracle's value)
                const float2 un = add2(add2(mul2(ux[p], f2(Cn.x)), mul2(uy[p], f2(Cn.y))), mul2(uz[p], f2(Cn.z)));
                up[2 * p] = left ? (un.x > 0.f) : (un.x <= 0.f);
                up[2 * p + 1] = left ? (un.y > 0.f) : (un.y <= 0.f);
                all = all && up[2 * p] && up[2 * p + 1];
                const float2 mB = f2(-B.w);
                const float2 rx = fma2(ux[p], mB, f2(B.x)), ry = fma2(uy[p], mB, f2(B.y)),
                             rz = fma2(uz[p], mB, f2(B.z));
                vg[p] = fma2(L[0][p], fma2(g[0][2][p], rz, fma2(g[0][1][p], ry, mul2(g[0][0][p], rx))), pv[0][p]);
                vh[p] = fma2(L[1][p], fma2(g[1][2][p], rz, fma2(g[1][1][p], ry, mul2(g[1][0][p], rx))), pv[1][p]);
            }
            if (all) {
                *reinterpret_cast<float4*>(c.face + o) = make_float4(vg[0].x, vg[0].y, vg[1].x, vg[1].y);
                *reinterpret_cast<float4*>(c.face + FK + o) = make_float4(vh[0].x, vh[0].y, vh[1].x, vh[1].y);
            } else {
                const float gv[4] = {vg[0].x, vg[0].y, vg[1].x, vg[1].y};
                const float hv[4] = {vh[0].x, vh[0].y, vh[1].x, vh[1].y};
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (up[e]) { c.face[o + e] = gv[e]; c.face[FK + o + e] = hv[e]; }
            }
        }
    }
}

// ------------------------------------------------------------------------------------
// Step 5 (micro PR-SGS, Eq. implicit_mic_final_equ) and Step 6 (update and integral
// error compensation, Eqs. solve_rho - solve_qrot), mixed precision on the packed
// pipe: the steps of k_micro_sweep (one warp per cell of one colour, four velocities
// per lane, faces in slot order), with the split of every face term into the
// diagonal (u.n > 0) and the neighbour part (u.n <= 0) taken by selects, which adds
// exact zeros where the scalar kernel skips the term.
// ------------------------------------------------------------------------------------
#ifndef MICROP_FIRST_MINB
#define MICROP_FIRST_MINB 3
#endif
#ifndef MICROP_MID_MINB
#define MICROP_MID_MINB 5
#endif
#ifndef MICROP_LAST_MINB
#define MICROP_LAST_MINB 2
#endif
__device__ __forceinline__ float2 pos2(float2 a) { return make_float2(a.x > 0.f ? a.x : 0.f, a.y > 0.f ? a.y : 0.f); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(a.x > 0.f ? 0.f : a.x, a.y > 0.f ? 0.f : a.y); }

template <int WPB, bool FIRST, bool LAST>
__global__ void __launch_bounds__(WPB * 32, LAST ? MICROP_LAST_MINB : (FIRST ? MICROP_FIRST_MINB : MICROP_MID_MINB))
    k_micro_sweep_p(Dev<float> c, const int* cells, int ncells, int colour) {
    __shared__ float s_e[WPB][EQN + 2];
    __shared__ float4 s_NA[WPB][MAXF];            // signed outward normal, A/V
    __shared__ int2 s_NO[WPB][MAXF];              // neighbour, neighbour term used
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int t = blockIdx.x * WPB + w;
    if (t >= ncells) return;                      // whole warp: no block barriers below
    const int i = cells[t];
    const int s0 = c.slot_off[i], ns = c.slot_off[i + 1] - s0;
    if (lane < EQN + 2) s_e[w][lane] = (float)c.ceq[(size_t)i * CEQ + lane];
    if (lane < ns) {
        const int m = s0 + lane;
        const float sg = c.slot_left[m] ? 1.f : -1.f;
        s_NA[w][lane] = make_float4(sg * c.slot_nT[m], sg * c.slot_nT[c.nnz + m], sg * c.slot_nT[2 * c.nnz + m],
                                    c.slot_AVT[m]);
        s_NO[w][lane] = make_int2(c.slot_nbr[m], (c.slot_nbr[m] >= 0) && !(FIRST && c.slot_ncol[m] > colour));
    }
    __syncwarp();
    const float* e = s_e[w];
    const float2 itau = f2(e[EQN - 1]), base = f2(e[EQN]);
    const size_t NK = (size_t)c.N * c.Kp;
    const size_t oi = (size_t)i * c.Kp;
    FF sums[12];
    Acc<float> a[12];
    for (int k0 = 4 * lane; k0 < c.K; k0 += 128) {
        const float4 ux4 = *reinterpret_cast<const float4*>(c.uT + k0);
        const float4 uy4 = *reinterpret_cast<const float4*>(c.uT + c.Kp + k0);
        const float4 uz4 = *reinterpret_cast<const float4*>(c.uT + 2 * c.Kp + k0);
        const float2 ux[2] = {lo2(ux4), hi2(ux4)}, uy[2] = {lo2(uy4), hi2(uy4)}, uz[2] = {lo2(uz4), hi2(uz4)};
        float2 D[2] = {base, base}, og[2] = {f2(0.f), f2(0.f)}, oh[2] = {f2(0.f), f2(0.f)};
#pragma unroll 1
        for (int q = 0; q < ns; ++q) {
            const float4 NA = s_NA[w][q];
            const int2 NO = s_NO[w][q];
            const float2 nx = f2(NA.x), ny = f2(NA.y), nz = f2(NA.z), AV = f2(NA.w);
            float2 un[2];
            bool neg = false;
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                un[p] = fma2(uz[p], nz, fma2(uy[p], ny, mul2(ux[p], nx)));
                neg = neg || !(un[p].x > 0.f) || !(un[p].y > 0.f);
            }
#pragma unroll
            for (int p = 0; p < 2; ++p) D[p] = fma2(AV, pos2(un[p]), D[p]);
            if (NO.y && neg) {
                const size_t oj = (size_t)NO.x * c.Kp + k0;
                const float4 dg4 = *reinterpret_cast<const float4*>(c.dphi + oj);
                const float4 dh4 = *reinterpret_cast<const float4*>(c.dphi + NK + oj);
#pragma unroll
                for (int p = 0; p < 2; ++p) {
                    const float2 an = mul2(AV, neg2(un[p]));
                    og[p] = fma2(an, p ? hi2(dg4) : lo2(dg4), og[p]);
                    oh[p] = fma2(an, p ? hi2(dh4) : lo2(dh4), oh[p]);
                }
            }
        }
        float4 pg4, ph4;
        if (FIRST || LAST) {
            pg4 = *reinterpret_cast<const float4*>(c.phi + oi + k0);
            ph4 = *reinterpret_cast<const float4*>(c.phi + NK + oi + k0);
        }
        // F in the first sweep (k_micro_flux), Res in the later ones
        const float4 r0g4 = *reinterpret_cast<const float4*>(c.res + oi + k0);
        const float4 r0h4 = *reinterpret_cast<const float4*>(c.res + NK + oi + k0);
        float2 G[2], H[2], rg[2], rh[2], xg[2], xh[2];
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            if (FIRST || LAST) eval_eq2(e, ux[p], uy[p], uz[p], G[p], H[p]);
            if (FIRST) {
                rg[p] = sub2(mul2(sub2(G[p], p ? hi2(pg4) : lo2(pg4)), itau), p ? hi2(r0g4) : lo2(r0g4));
                rh[p] = sub2(mul2(sub2(H[p], p ? hi2(ph4) : lo2(ph4)), itau), p ? hi2(r0h4) : lo2(r0h4));
            } else {
                rg[p] = p ? hi2(r0g4) : lo2(r0g4);
                rh[p] = p ? hi2(r0h4) : lo2(r0h4);
            }
            const float2 iD = make_float2(__fdividef(1.f, D[p].x), __fdividef(1.f, D[p].y));
            xg[p] = mul2(sub2(rg[p], og[p]), iD);
            xh[p] = mul2(sub2(rh[p], oh[p]), iD);
            // the K padding keeps zero increments
            const int kk = k0 + 2 * p;
            if (kk >= c.K) { xg[p].x = 0.f; xh[p].x = 0.f; }
            if (kk + 1 >= c.K) { xg[p].y = 0.f; xh[p].y = 0.f; }
        }
        if (FIRST) {
            *reinterpret_cast<float4*>(c.res + oi + k0) = make_float4(rg[0].x, rg[0].y, rg[1].x, rg[1].y);
            *reinterpret_cast<float4*>(c.res + NK + oi + k0) = make_float4(rh[0].x, rh[0].y, rh[1].x, rh[1].y);
        }
        *reinterpret_cast<float4*>(c.dphi + oi + k0) = make_float4(xg[0].x, xg[0].y, xg[1].x, xg[1].y);
        *reinterpret_cast<float4*>(c.dphi + NK + oi + k0) = make_float4(xh[0].x, xh[0].y, xh[1].x, xh[1].y);
        if (LAST) {
            const float4 w4 = *reinterpret_cast<const float4*>(c.wT + k0);
            float2 g1[2], h1[2], tt[12];
            const float2 E0 = f2(e[0]), E1 = f2(e[1]), E2 = f2(e[2]);
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                g1[p] = add2(p ? hi2(pg4) : lo2(pg4), xg[p]);
                h1[p] = add2(p ? hi2(ph4) : lo2(ph4), xh[p]);
                const float2 wv = p ? hi2(w4) : lo2(w4);
                const float2 wg = mul2(wv, sub2(g1[p], G[p])), wh = mul2(wv, sub2(h1[p], H[p]));
                const float2 cx = sub2(ux[p], E0), cy = sub2(uy[p], E1), cz = sub2(uz[p], E2);
                const float2 wgc = mul2(wg, fma2(cz, cz, fma2(cy, cy, mul2(cx, cx))));
                const float2 u2 = fma2(uz[p], uz[p], fma2(uy[p], uy[p], mul2(ux[p], ux[p])));
                const float2 tv[12] = {wg, mul2(wg, ux[p]), mul2(wg, uy[p]), mul2(wg, uz[p]),
                                       fma2(mul2(f2(0.5f), u2), wg, wh), wh,
                                       mul2(wgc, cx), mul2(wgc, cy), mul2(wgc, cz),
                                       mul2(wh, cx), mul2(wh, cy), mul2(wh, cz)};
#pragma unroll
                for (int j = 0; j < 12; ++j) tt[j] = p == 0 ? tv[j] : add2(tt[j], tv[j]);
            }
#pragma unroll
            for (int j = 0; j < 12; ++j) a[j].add(hsum(tt[j]));
            *reinterpret_cast<float4*>(c.phi + oi + k0) = make_float4(g1[0].x, g1[0].y, g1[1].x, g1[1].y);
            *reinterpret_cast<float4*>(c.phi + NK + oi + k0) = make_float4(h1[0].x, h1[0].y, h1[1].x, h1[1].y);
        }
    }
    if (LAST) {
#pragma unroll
        for (int j = 0; j < 12; ++j) sums[j] = Red<float>::from(a[j]);
        warp_red_lane0<float, 12>(sums);
        if (lane == 0)
            for (int j = 0; j < 12; ++j) c.S[(size_t)i * 12 + j] = Red<float>::to_d(sums[j]);
    }
}

// Bulk copies global -> shared with completion on an mbarrier (the cell's own rows of
// one 128-velocity chunk: one instruction per row, issued by one lane).
__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mb_init(unsigned long long* mb, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mb)), "r"(count) : "memory");
}
__device__ __forceinline__ void mb_expect_tx(unsigned long long* mb, unsigned bytes) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}"
                 ::"r"(smem_u32(mb)), "r"(bytes) : "memory");
}
// dst and src 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* mb) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(mb)) : "memory");
}
__device__ __forceinline__ bool mb_try_wait(unsigned long long* mb, unsigned parity) {
    unsigned ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok) : "r"(smem_u32(mb)), "r"(parity) : "memory");
    return ok != 0u;
}
// Bounded wait for the phase of parity `parity`: gives up after limit_ns (read from the
// global timer every 64 polls) and reports whether the phase completed
__device__ __forceinline__ bool mb_wait_bounded(unsigned long long* mb, unsigned parity,
                                                unsigned long long limit_ns) {
    unsigned polls = 0;
    unsigned long long t0 = 0;
    while (!mb_try_wait(mb, parity)) {
        if ((++polls & 63u) == 0u) {
            const unsigned long long t = global_ns();
            if (t0 == 0) t0 = t;
            else if (t - t0 > limit_ns) return false;
        }
    }
    return true;
}

// The packed micro sweep with its row loads staged through shared memory, as in
// k_micro_sweep_st: the next chunk's rows (inflow neighbours' dphi, the cell's phi and
// F/Res) are in flight while the current chunk computes, double-buffered.  The
// neighbours' rows are per-lane asynchronous copies of the 16 bytes a lane needs (only
// upwind ones); the cell's own rows too (BULK false), or whole-chunk bulk copies by
// lane 0 completing on the warp's mbarrier of that stage (BULK true; measured 10 %
// slower at scale, 39.4 vs 35.8 ms for the last sweeps).  A bulk wait that runs out
// (1 s) records status bit 4 (RK_ETIMEOUT on the host) and ends the warp's work after
// a second bounded wait.
template <int WPB, bool FIRST, bool LAST, bool BULK>
__global__ void __launch_bounds__(WPB * 32)
    k_micro_sweep_st_p(Dev<float> c, const int* cells, int ncells, int colour, int maxs) {
    extern __shared__ __align__(16) unsigned char st_raw[];
    __shared__ __align__(8) unsigned long long s_mb[WPB][2];
    __shared__ float s_e[WPB][EQN + 2];
    __shared__ float4 s_NA[WPB][MAXF];
    __shared__ int2 s_NO[WPB][MAXF];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int t = blockIdx.x * WPB + w;
    if (t >= ncells) return;                      // whole warp: no block barriers below
    const int i = cells[t];
    const int s0 = c.slot_off[i], ns = c.slot_off[i + 1] - s0;
    if (lane < EQN + 2) s_e[w][lane] = (float)c.ceq[(size_t)i * CEQ + lane];
    if (lane < ns) {
        const int m = s0 + lane;
        const float sg = c.slot_left[m] ? 1.f : -1.f;
        s_NA[w][lane] = make_float4(sg * c.slot_nT[m], sg * c.slot_nT[c.nnz + m], sg * c.slot_nT[2 * c.nnz + m],
                                    c.slot_AVT[m]);
        s_NO[w][lane] = make_int2(c.slot_nbr[m], (c.slot_nbr[m] >= 0) && !(FIRST && c.slot_ncol[m] > colour));
    }
    __syncwarp();
    const float* e = s_e[w];
    const float2 itau = f2(e[EQN - 1]), base = f2(e[EQN]);
    const size_t NK = (size_t)c.N * c.Kp;
    const size_t oi = (size_t)i * c.Kp;
    const int nrow = 2 * maxs + 4;                // rows per stage: 2 per face, phi g/h, F|Res g/h
    float* rows = reinterpret_cast<float*>(st_raw) + (size_t)w * 2 * nrow * 128;
    float* buf = rows + (size_t)lane * 4;
    auto slot = [&](int st_, int r) { return buf + (size_t)(st_ * nrow + r) * 128; };
    const int nch = (c.K + 127) / 128;
    if (BULK && lane == 0) {
        mb_init(&s_mb[w][0], 1);
        mb_init(&s_mb[w][1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (BULK) __syncwarp();
    // the cell's own rows of chunk ch into stage st_ (every lane calls this; the warp
    // has finished reading stage st_ when it is reissued)
    auto bulk_own = [&](int ch, int st_) {
        __syncwarp();
        if (lane == 0) {
            const int nk = min(128, c.Kp - ch * 128);      // a multiple of 32 (K_pad is)
            const unsigned by = 4u * (unsigned)nk;
            unsigned long long* mb = &s_mb[w][st_];
            float* base = rows + (size_t)st_ * nrow * 128;
            const size_t o = oi + (size_t)ch * 128;
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mb_expect_tx(mb, ((FIRST || LAST) ? 4u : 2u) * by);
            if (FIRST || LAST) {
                bulk_g2s(base + (size_t)(2 * maxs) * 128, c.phi + o, by, mb);
                bulk_g2s(base + (size_t)(2 * maxs + 1) * 128, c.phi + NK + o, by, mb);
            }
            bulk_g2s(base + (size_t)(2 * maxs + 2) * 128, c.res + o, by, mb);
            bulk_g2s(base + (size_t)(2 * maxs + 3) * 128, c.res + NK + o, by, mb);
        }
    };
    auto prefetch = [&](int ch, int st_) -> unsigned {
        const int k0 = ch * 128 + 4 * lane;
        unsigned mk = 0u;
        if (k0 < c.K) {
            const float4 ux4 = *reinterpret_cast<const float4*>(c.uT + k0);
            const float4 uy4 = *reinterpret_cast<const float4*>(c.uT + c.Kp + k0);
            const float4 uz4 = *reinterpret_cast<const float4*>(c.uT + 2 * c.Kp + k0);
#pragma unroll 1
            for (int q = 0; q < ns; ++q) {
                const int2 NO = s_NO[w][q];
                if (!NO.y) continue;
                const float4 NA = s_NA[w][q];
                const float2 u0 = fma2(lo2(uz4), f2(NA.z), fma2(lo2(uy4), f2(NA.y), mul2(lo2(ux4), f2(NA.x))));
                const float2 u1 = fma2(hi2(uz4), f2(NA.z), fma2(hi2(uy4), f2(NA.y), mul2(hi2(ux4), f2(NA.x))));
                if (!(u0.x > 0.f) || !(u0.y > 0.f) || !(u1.x > 0.f) || !(u1.y > 0.f)) {
                    const size_t oj = (size_t)NO.x * c.Kp + k0;
                    cp_async<16>(slot(st_, 2 * q), c.dphi + oj);
                    cp_async<16>(slot(st_, 2 * q + 1), c.dphi + NK + oj);
                    mk |= 1u << q;
                }
            }
            if (!BULK) {
                if (FIRST || LAST) {
                    cp_async<16>(slot(st_, 2 * maxs), c.phi + oi + k0);
                    cp_async<16>(slot(st_, 2 * maxs + 1), c.phi + NK + oi + k0);
                }
                cp_async<16>(slot(st_, 2 * maxs + 2), c.res + oi + k0);
                cp_async<16>(slot(st_, 2 * maxs + 3), c.res + NK + oi + k0);
            }
        }
        cp_async_commit();
        if (BULK) bulk_own(ch, st_);
        return mk;
    };
    Acc<float> a[12];
    unsigned m_next = prefetch(0, 0);
    for (int ch = 0; ch < nch; ++ch) {
        const int st_ = ch & 1;
        const unsigned m_cur = m_next;
        if (ch + 1 < nch) m_next = prefetch(ch + 1, st_ ^ 1);
        else cp_async_commit();                   // an empty group keeps the count
        cp_async_wait<1>();                       // this thread's copies of chunk ch are done
        if (BULK) {
            const unsigned par = (unsigned)(ch >> 1) & 1u;
            const bool done = mb_wait_bounded(&s_mb[w][st_], par, 1000000000ull);
            if (!__all_sync(0xffffffffu, done)) {
                if (lane == 0) atomicOr(c.status, 4);
                mb_wait_bounded(&s_mb[w][st_], par, 1000000000ull);
                if (ch + 1 < nch)                 // chunk ch + 1, already issued
                    mb_wait_bounded(&s_mb[w][st_ ^ 1], (unsigned)((ch + 1) >> 1) & 1u, 1000000000ull);
                cp_async_wait<0>();
                return;
            }
        }
        const int k0 = ch * 128 + 4 * lane;
        if (k0 >= c.K) continue;
        const float4 ux4 = *reinterpret_cast<const float4*>(c.uT + k0);
        const float4 uy4 = *reinterpret_cast<const float4*>(c.uT + c.Kp + k0);
        const float4 uz4 = *reinterpret_cast<const float4*>(c.uT + 2 * c.Kp + k0);
        const float2 ux[2] = {lo2(ux4), hi2(ux4)}, uy[2] = {lo2(uy4), hi2(uy4)}, uz[2] = {lo2(uz4), hi2(uz4)};
        float2 D[2] = {base, base}, og[2] = {f2(0.f), f2(0.f)}, oh[2] = {f2(0.f), f2(0.f)};
#pragma unroll 1
        for (int q = 0; q < ns; ++q) {
            const float4 NA = s_NA[w][q];
            const float2 nx = f2(NA.x), ny = f2(NA.y), nz = f2(NA.z), AV = f2(NA.w);
            float2 un[2];
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                un[p] = fma2(uz[p], nz, fma2(uy[p], ny, mul2(ux[p], nx)));
                D[p] = fma2(AV, pos2(un[p]), D[p]);
            }
            if ((m_cur >> q) & 1u) {
                const float4 dg4 = *reinterpret_cast<const float4*>(slot(st_, 2 * q));
                const float4 dh4 = *reinterpret_cast<const float4*>(slot(st_, 2 * q + 1));
#pragma unroll
                for (int p = 0; p < 2; ++p) {
                    const float2 an = mul2(AV, neg2(un[p]));
                    og[p] = fma2(an, p ? hi2(dg4) : lo2(dg4), og[p]);
                    oh[p] = fma2(an, p ? hi2(dh4) : lo2(dh4), oh[p]);
                }
            }
        }
        float4 pg4, ph4;
        if (FIRST || LAST) {
            pg4 = *reinterpret_cast<const float4*>(slot(st_, 2 * maxs));
            ph4 = *reinterpret_cast<const float4*>(slot(st_, 2 * maxs + 1));
        }
        const float4 r0g4 = *reinterpret_cast<const float4*>(slot(st_, 2 * maxs + 2));
        const float4 r0h4 = *reinterpret_cast<const float4*>(slot(st_, 2 * maxs + 3));
        float2 G[2], H[2], rg[2], rh[2], xg[2], xh[2];
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            if (FIRST || LAST) eval_eq2(e, ux[p], uy[p], uz[p], G[p], H[p]);
            if (FIRST) {
                rg[p] = sub2(mul2(sub2(G[p], p ? hi2(pg4) : lo2(pg4)), itau), p ? hi2(r0g4) : lo2(r0g4));
                rh[p] = sub2(mul2(sub2(H[p], p ? hi2(ph4) : lo2(ph4)), itau), p ? hi2(r0h4) : lo2(r0h4));
            } else {
                rg[p] = p ? hi2(r0g4) : lo2(r0g4);
                rh[p] = p ? hi2(r0h4) : lo2(r0h4);
            }
            const float2 iD = make_float2(__fdividef(1.f, D[p].x), __fdividef(1.f, D[p].y));
            xg[p] = mul2(sub2(rg[p], og[p]), iD);
            xh[p] = mul2(sub2(rh[p], oh[p]), iD);
            const int kk = k0 + 2 * p;
            if (kk >= c.K) { xg[p].x = 0.f; xh[p].x = 0.f; }
            if (kk + 1 >= c.K) { xg[p].y = 0.f; xh[p].y = 0.f; }
        }
        if (FIRST) {
            *reinterpret_cast<float4*>(c.res + oi + k0) = make_float4(rg[0].x, rg[0].y, rg[1].x, rg[1].y);
            *reinterpret_cast<float4*>(c.res + NK + oi + k0) = make_float4(rh[0].x, rh[0].y, rh[1].x, rh[1].y);
        }
        *reinterpret_cast<float4*>(c.dphi + oi + k0) = make_float4(xg[0].x, xg[0].y, xg[1].x, xg[1].y);
        *reinterpret_cast<float4*>(c.dphi + NK + oi + k0) = make_float4(xh[0].x, xh[0].y, xh[1].x, xh[1].y);
        if (LAST) {
            const float4 w4 = *reinterpret_cast<const float4*>(c.wT + k0);
            float2 g1[2], h1[2], tt[12];
            const float2 E0 = f2(e[0]), E1 = f2(e[1]), E2 = f2(e[2]);
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                g1[p] = add2(p ? hi2(pg4) : lo2(pg4), xg[p]);
                h1[p] = add2(p ? hi2(ph4) : lo2(ph4), xh[p]);
                const float2 wv = p ? hi2(w4) : lo2(w4);
                const float2 wg = mul2(wv, sub2(g1[p], G[p])), wh = mul2(wv, sub2(h1[p], H[p]));
                const float2 cx = sub2(ux[p], E0), cy = sub2(uy[p], E1), cz = sub2(uz[p], E2);
                const float2 wgc = mul2(wg, fma2(cz, cz, fma2(cy, cy, mul2(cx, cx))));
                const float2 u2 = fma2(uz[p], uz[p], fma2(uy[p], uy[p], mul2(ux[p], ux[p])));
                const float2 tv[12] = {wg, mul2(wg, ux[p]), mul2(wg, uy[p]), mul2(wg, uz[p]),
                                       fma2(mul2(f2(0.5f), u2), wg, wh), wh,
                                       mul2(wgc, cx), mul2(wgc, cy), mul2(wgc, cz),
                                       mul2(wh, cx), mul2(wh, cy), mul2(wh, cz)};
#pragma unroll
                for (int j = 0; j < 12; ++j) tt[j] = p == 0 ? tv[j] : add2(tt[j], tv[j]);
            }
#pragma unroll
            for (int j = 0; j < 12; ++j) a[j].add(hsum(tt[j]));
            *reinterpret_cast<float4*>(c.phi + oi + k0) = make_float4(g1[0].x, g1[0].y, g1[1].x, g1[1].y);
            *reinterpret_cast<float4*>(c.phi + NK + oi + k0) = make_float4(h1[0].x, h1[0].y, h1[1].x, h1[1].y);
        }
    }
    cp_async_wait<0>();
    if (LAST) {
        FF sums[12];
#pragma unroll
        for (int j = 0; j < 12; ++j) sums[j] = Red<float>::from(a[j]);
        warp_red_lane0<float, 12>(sums);
        if (lane == 0)
            for (int j = 0; j < 12; ++j) c.S[(size_t)i * 12 + j] = Red<float>::to_d(sums[j]);
    }
}

}  // namespace rk
