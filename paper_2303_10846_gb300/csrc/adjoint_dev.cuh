// Device side of the adjoint of the steady residual operator (FP64, or FP32 per-velocity
// arithmetic for mixed-precision contexts).
//
// Unknowns X = (phi, W, q) of a steady state of the implicit iteration (Sec. 3.5 with
// dphi = 0 and a zero macro increment), residual R(X; p) = (R_phi, R_W, R_q):
//   R_phi = (phi*(W, q) - phi)/tau(W) - F(phi; p)          Eq. implicit_mic_final_equ
//   R_W   = sum_k w Psi (phi - phi*)  (+ rho R((1-1/Z) T_rot + T/Z) - rho E_rot in
//           the rotational-energy row)                      Eqs. solve_rho - solve_Erot
//   R_q   = 1/2 sum_k w c|c|^2 (g - g*) + (a_tr - 1) q_tr,
//           sum_k w c (h - h*) + (a_rot - 1) q_rot           Eqs. solve_qtr, solve_qrot
// F is the micro flux of Eq. implicit_mic_flux with the interface distribution of
// Eq. flux_solve_phi and the limited reconstruction of Eq. flux_solve_phi_phi.
// Parameters p = (T_w shift of every wall, rho_inf, U_inf[3], T_inf of every farfield).
//
// The kernels below apply (dR/dX)^T v and (dR/dp)^T v by hand-written reverse mode of
// the forward kernels: per cell (collision terms and the compensation rows), per
// interior face (moments -> interface state -> phi* -> blend), per boundary face
// (wall density rho_w, farfield Maxwellian), and the gradient / Venkatakrishnan
// limiter / least-squares gather.  Every scatter of the forward pass becomes a gather
// in a fixed order, so results are bit-reproducible.
#pragma once

#include "rykov_dev.cuh"

namespace rk {

constexpr int ADJ_FPAR = 12;
// minimum resident blocks of the per-velocity adjoint kernels (register budget)
#ifndef ADJ_MINB
#define ADJ_MINB 1
#endif     // per boundary face: dR/dp^T v (6), J, force (3), 2 spare

struct AdjBufs {
    double *f0, *fbar;           // [2][F][Kp] phi(x_f - u s) and its adjoint
    const double *vphi;          // [2][N][Kp] weights v of R_phi
    double* ophi;                // [2][N][Kp] output (phi part)
    const double *vW, *vq;       // [N][6]
    double *oW, *oq;             // [N][6]
    double* nbg;                 // [2][4][N][Kp] gradient adjoint (3) and Delta adjoint per cell
    signed char* nbs;            // [2][N][Kp] local slot of the neighbour giving Delta_max/min
    const int* slot_mirg;        // [nnz] global slot of the same face in the neighbour's list (-1)
    const double* slot_AVn;      // [nnz] A_f / V_neighbour (0 at boundary faces)
    const double* tau;           // [N] tau(W_i)
    double* fpar;                // [Fb][ADJ_FPAR]
    const double* iterp;         // [4]: [1] reconstruction mode of the steady operator (0-3)
    double obj_scale;            // weight of the objective seed at wall faces (0: none)
    int objective;               // 0: heat to the wall, 1: drag
    double edrag[3];             // drag direction
    // FP32 arithmetic of a mixed context: its FP32 velocity set and distributions
    const float *uf, *wf, *phif;
    const float* f0f;            // [2][F][Kp] the FP32 reconstruction (phi0 at the faces)
    const float* vphif;          // [2][N][Kp] the phi block of v rounded to FP32
};

// per-velocity inputs in the arithmetic type S: FP32 arrays of a mixed context when S
// is float (no conversions), the FP64 arrays otherwise
template <typename S>
__device__ __forceinline__ S vel(const Dev<double>& c, const AdjBufs& a, int dim, int k) {
    if constexpr (sizeof(S) == 4) return a.uf[(size_t)dim * c.Kp + k];
    else return c.u[(size_t)dim * c.Kp + k];
}
template <typename S>
__device__ __forceinline__ S wgt(const Dev<double>& c, const AdjBufs& a, int k) {
    if constexpr (sizeof(S) == 4) return a.wf[k];
    else return c.w[k];
}
template <typename S>
__device__ __forceinline__ S vin(const AdjBufs& a, size_t o) {
    if constexpr (sizeof(S) == 4) return a.vphif[o];
    else return a.vphi[o];
}
template <typename S>
__device__ __forceinline__ S dist(const Dev<double>& c, const AdjBufs& a, size_t o) {
    if constexpr (sizeof(S) == 4) return a.phif[o];
    else return c.phi[o];
}

// ------------------------------------------------------------------------------------
// reverse mode of one Rykov equilibrium point (Eqs. eqdf_G* - eqdf_Rrot)
// ------------------------------------------------------------------------------------
// State in the variables of the formula: theta = R T, theta_tr = R T_tr,
// theta_rot = R T_rot.  With p = rho theta etc. the equilibrium reads
//   G^tr = M_tr (1 + (c.q_tr) A_tr),   A_tr = (|c|^2/theta_tr - 5) / (15 rho theta_tr^2)
//   G^rot = M (1 + w0 (c.q_tr) A),  A = (|c|^2/theta - 5) / (15 rho theta^2)
//   R^tr = theta_rot G^tr + (1 - delta)(c.q_rot) M_tr / (rho theta_tr)
//   R^rot = theta G^rot + w1 (1 - delta)(c.q_rot) M / (rho theta)
// (the same functions as the forward formula, with p_rot theta_tr / theta_rot = rho
// theta_tr simplified), G* = (1-1/Z) G^tr + G^rot/Z, R* likewise.
template <typename S>
struct EqS {
    S rho, U[3], th, thtr, throt, qtr[3], qrot[3];
    // derived constants (make_eqs): 1/rho, 1/theta_tr, 1/theta, the Maxwellian
    // prefactors rho (2 pi theta_tr)^-3/2 and rho (2 pi theta)^-3/2, 1/(15 rho)
    S irho, itr, it, ntr, nr, i15r;
};
template <typename S>
__device__ __forceinline__ EqS<S> make_eqs(S rho, const S* U, S th, S thtr, S throt, const S* qtr,
                                           const S* qrot) {
    EqS<S> e;
    e.rho = rho;
    for (int k = 0; k < 3; ++k) { e.U[k] = U[k]; e.qtr[k] = qtr[k]; e.qrot[k] = qrot[k]; }
    e.th = th; e.thtr = thtr; e.throt = throt;
    e.irho = S(1) / rho; e.itr = S(1) / thtr; e.it = S(1) / th;
    const S atr = S(2.0 * PI) * thtr, ar = S(2.0 * PI) * th;
    e.ntr = rho / (atr * sqrt(atr));
    e.nr = rho / (ar * sqrt(ar));
    e.i15r = S(1) / (S(15) * rho);
    return e;
}

// d[0] rho, [1-3] U, [4] theta, [5] theta_tr, [6] theta_rot, [7-9] q_tr, [10-12] q_rot
// = Gb dG*/dx + Hb dR*/dx at velocity u (written, not added); G, H receive G*(u), R*(u)
// themselves (the forward values come with the same exponentials).  S: the arithmetic
// type (FP64, or FP32 for the adjoint of a mixed-precision context).
template <typename S>
__device__ __forceinline__ void eq_vjp(const EqS<S>& s, S om0, S om1, S del, S Z, S ux, S uy, S uz,
                                       S Gb, S Hb, S (&d)[13], S& G, S& H) {
    const S c[3] = {ux - s.U[0], uy - s.U[1], uz - s.U[2]};
    const S c2 = c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
    const S cqt = c[0] * s.qtr[0] + c[1] * s.qtr[1] + c[2] * s.qtr[2];
    const S cqr = c[0] * s.qrot[0] + c[1] * s.qrot[1] + c[2] * s.qrot[2];
    const S irho = s.irho, itr = s.itr, it = s.it, i15r = s.i15r;
    const S Mtr = s.ntr * ex(S(-0.5) * c2 * itr);
    const S M = s.nr * ex(S(-0.5) * c2 * it);
    const S Atr = (c2 * itr - S(5)) * itr * itr * i15r;
    const S Ar = (c2 * it - S(5)) * it * it * i15r;
    const S Ptr = S(1) + cqt * Atr;
    const S Pr = S(1) + om0 * cqt * Ar;
    const S Gtr = Mtr * Ptr, Grot = M * Pr;
    const S Btr = (S(1) - del) * irho * itr;
    const S Br = om1 * (S(1) - del) * irho * it;
    const S a1 = S(1) - S(1) / Z, a2 = S(1) / Z;
    G = a1 * Gtr + a2 * Grot;
    H = a1 * (s.throt * Gtr + Btr * cqr * Mtr) + a2 * (s.th * Grot + Br * cqr * M);
    const S htb = a1 * Hb, hrb = a2 * Hb;
    const S gtb = a1 * Gb + htb * s.throt;
    const S grb = a2 * Gb + hrb * s.th;
    S rb = S(0), thb = S(0), thtrb = S(0), Ub[3] = {S(0), S(0), S(0)}, qtb[3] = {S(0), S(0), S(0)},
      qrb[3] = {S(0), S(0), S(0)}, Mtrb = S(0), Mb = S(0);
    d[6] = htb * Gtr;
    thb += hrb * Grot;
    {   // (1 - delta) (c.q_rot) M_tr / (rho theta_tr)
        const S X = Btr * cqr * Mtr;
        const S cqb = htb * Btr * Mtr;
        Mtrb += htb * Btr * cqr;
        rb -= htb * X * irho;
        thtrb -= htb * X * itr;
        for (int k = 0; k < 3; ++k) { qrb[k] += cqb * c[k]; Ub[k] -= cqb * s.qrot[k]; }
    }
    {   // w1 (1 - delta) (c.q_rot) M / (rho theta)
        const S X = Br * cqr * M;
        const S cqb = hrb * Br * M;
        Mb += hrb * Br * cqr;
        rb -= hrb * X * irho;
        thb -= hrb * X * it;
        for (int k = 0; k < 3; ++k) { qrb[k] += cqb * c[k]; Ub[k] -= cqb * s.qrot[k]; }
    }
    {   // G^tr = M_tr (1 + (c.q_tr) A_tr)
        Mtrb += gtb * Ptr;
        const S Pb = gtb * Mtr;
        const S cqb = Pb * Atr, Ab = Pb * cqt;
        const S c2b = Ab * itr * itr * itr * i15r;
        rb -= Ab * Atr * irho;
        thtrb += Ab * (S(10) - S(3) * c2 * itr) * itr * itr * itr * i15r;
        for (int k = 0; k < 3; ++k) { qtb[k] += cqb * c[k]; Ub[k] -= cqb * s.qtr[k] + S(2) * c2b * c[k]; }
    }
    {   // G^rot = M (1 + w0 (c.q_tr) A)
        Mb += grb * Pr;
        const S Pb = grb * M;
        const S cqb = Pb * om0 * Ar, Ab = Pb * om0 * cqt;
        const S c2b = Ab * it * it * it * i15r;
        rb -= Ab * Ar * irho;
        thb += Ab * (S(10) - S(3) * c2 * it) * it * it * it * i15r;
        for (int k = 0; k < 3; ++k) { qtb[k] += cqb * c[k]; Ub[k] -= cqb * s.qtr[k] + S(2) * c2b * c[k]; }
    }
    // Maxwellians rho (2 pi theta)^-3/2 exp(-|c|^2 / (2 theta))
    rb += Mtrb * Mtr * irho + Mb * M * irho;
    thtrb += Mtrb * Mtr * (S(0.5) * c2 * itr * itr - S(1.5) * itr);
    thb += Mb * M * (S(0.5) * c2 * it * it - S(1.5) * it);
    for (int k = 0; k < 3; ++k) Ub[k] += (Mtrb * Mtr * itr + Mb * M * it) * c[k];
    d[0] = rb;
    for (int k = 0; k < 3; ++k) { d[1 + k] = Ub[k]; d[7 + k] = qtb[k]; d[10 + k] = qrb[k]; }
    d[4] = thb;
    d[5] = thtrb;
}

// ------------------------------------------------------------------------------------
// cell terms: collision part of R_phi and the compensation rows R_W, R_q.
// mode bit 0: write ophi = the cell part of (dR/dphi)^T v (the face gathers add the
// flux part later); bit 1: write oW, oq.  One warp per cell.
// ------------------------------------------------------------------------------------
template <int WPB, typename S = double>
__global__ void __launch_bounds__(WPB * 32, sizeof(S) == 4 ? ADJ_MINB : 1) k_adj_cell(Dev<double> c, AdjBufs a, int mode) {
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * WPB + (threadIdx.x >> 5);
    if (i >= c.N) return;
    const double R = c.R, Z = c.Z;
    const double* W = c.W + 6 * (size_t)i;
    const double* q = c.q + 6 * (size_t)i;
    const Prim p = prim_from_W(W, R);
    const double tau = relax_time(c, p.rho, p.Ttr);
    const double itau = 1.0 / tau;
    // per-velocity arithmetic in S (FP64, or FP32 with compensated sums)
    const S Us[3] = {(S)p.U[0], (S)p.U[1], (S)p.U[2]};
    const S qs[6] = {(S)q[0], (S)q[1], (S)q[2], (S)q[3], (S)q[4], (S)q[5]};
    const EqS<S> st = make_eqs<S>((S)p.rho, Us, (S)(R * p.T), (S)(R * p.Ttr), (S)(R * p.Trot), qs, qs + 3);
    const S itS = (S)itau, om0 = (S)c.omega0, om1 = (S)c.omega1, del = (S)c.delta, ZS = (S)Z;
    double vW[6], vq[6];
    S vWs[6], vqs[6];
    for (int d = 0; d < 6; ++d) {
        vW[d] = a.vW[6 * (size_t)i + d]; vq[d] = a.vq[6 * (size_t)i + d];
        vWs[d] = (S)vW[d]; vqs[d] = (S)vq[d];
    }
    const size_t NK = (size_t)c.N * c.Kp;
    Acc<S> acc[17];
    for (int k = lane; k < c.K; k += 32) {
        const S ux = vel<S>(c, a, 0, k), uy = vel<S>(c, a, 1, k), uz = vel<S>(c, a, 2, k), w = wgt<S>(c, a, k);
        const size_t o = (size_t)i * c.Kp + k;
        const S g = dist<S>(c, a, o), h = dist<S>(c, a, NK + o);
        const S vg = vin<S>(a, o), vh = vin<S>(a, NK + o);
        const S cx = ux - Us[0], cy = uy - Us[1], cz = uz - Us[2];
        const S c2 = cx * cx + cy * cy + cz * cz;
        const S cvt = cx * vqs[0] + cy * vqs[1] + cz * vqs[2];
        const S cvr = cx * vqs[3] + cy * vqs[4] + cz * vqs[5];
        const S u2h = S(0.5) * (ux * ux + uy * uy + uz * uz);
        // weights of phi in the compensation rows (moments Psi and the heat fluxes)
        const S mg = w * (vWs[0] + ux * vWs[1] + uy * vWs[2] + uz * vWs[3] + u2h * vWs[4] + S(0.5) * c2 * cvt);
        const S mh = w * (vWs[4] + vWs[5] + cvr);
        if (mode & 1) {
            a.ophi[o] = (double)(-vg * itS + mg);
            a.ophi[NK + o] = (double)(-vh * itS + mh);
        }
        if (mode & 2) {
            S G, H, dd[13];
            eq_vjp<S>(st, om0, om1, del, ZS, ux, uy, uz, vg * itS - mg, vh * itS - mh, dd, G, H);
#pragma unroll
            for (int j = 0; j < 13; ++j) acc[j].add(dd[j]);
            acc[13].add(-((vg * (G - g) + vh * (H - h)) * itS * itS));
            const S dg = g - G, dh = h - H;
            const S t1 = S(-0.5) * w * dg, t2 = -w * dh;
            acc[14].add(t1 * (vqs[0] * c2 + S(2) * cx * cvt) + t2 * vqs[3]);
            acc[15].add(t1 * (vqs[1] * c2 + S(2) * cy * cvt) + t2 * vqs[4]);
            acc[16].add(t1 * (vqs[2] * c2 + S(2) * cz * cvt) + t2 * vqs[5]);
        }
    }
    if (!(mode & 2)) return;
    typename Red<S>::V v[17];
#pragma unroll
    for (int j = 0; j < 17; ++j) v[j] = Red<S>::from(acc[j]);
    warp_red<S, 17>(v);
    if (lane != 0) return;
    double t[17];
    for (int j = 0; j < 17; ++j) t[j] = Red<S>::to_d(v[j]);
    double rb = t[0], Ub[3] = {t[1] + t[14], t[2] + t[15], t[3] + t[16]};
    double Tb = R * t[4], Ttrb = R * t[5], Trotb = R * t[6], taub = t[13];
    double qb[6];
    for (int d = 0; d < 6; ++d) qb[d] = t[7 + d];
    double Wb[6] = {0.0, 0.0, 0.0, 0.0, 0.0, -vW[5]};
    // rotational-energy row: + rho R ((1 - 1/Z) T_rot + T/Z) - rho E_rot
    rb += vW[5] * R * ((1.0 - 1.0 / Z) * p.Trot + p.T / Z);
    Trotb += vW[5] * p.rho * R * (1.0 - 1.0 / Z);
    Tb += vW[5] * p.rho * R / Z;
    // heat-flux rows: + (a - 1) q
    const double atr = (1.0 / 3.0) * (1.0 - (1.0 - c.omega0) / Z);
    const double arot = (1.0 - c.delta) * (1.0 - (1.0 - c.omega1) / Z);
    for (int d = 0; d < 3; ++d) { qb[d] += vq[d] * (atr - 1.0); qb[3 + d] += vq[3 + d] * (arot - 1.0); }
    // tau = mu(T_tr) / (rho R T_tr); d ln mu / d ln T_tr from the viscosity law
    Ttrb += taub * tau * (viscosity_slope(c, p.Ttr) - 1.0) / p.Ttr;
    rb -= taub * tau / p.rho;
    // primitives from W
    const double k15 = 1.0 / (1.5 * p.rho * R), k25 = 1.0 / (2.5 * p.rho * R), kr = 1.0 / (p.rho * R);
    double keb = 0.0;
    Wb[4] += Ttrb * k15; keb -= Ttrb * k15; Wb[5] -= Ttrb * k15; rb -= Ttrb * p.Ttr / p.rho;
    Wb[5] += Trotb * kr; rb -= Trotb * p.Trot / p.rho;
    Wb[4] += Tb * k25; keb -= Tb * k25; rb -= Tb * p.T / p.rho;
    const double U2 = p.U[0] * p.U[0] + p.U[1] * p.U[1] + p.U[2] * p.U[2];
    rb += keb * 0.5 * U2;
    double UbU = 0.0;
    for (int d = 0; d < 3; ++d) {
        Ub[d] += keb * p.rho * p.U[d];
        Wb[1 + d] += Ub[d] / p.rho;
        UbU += Ub[d] * p.U[d];
    }
    rb -= UbU / p.rho;
    Wb[0] += rb;
    for (int d = 0; d < 6; ++d) { a.oW[6 * (size_t)i + d] = Wb[d]; a.oq[6 * (size_t)i + d] = qb[d]; }
}

// ------------------------------------------------------------------------------------
// steady residual R(X; p) from the face distributions phi_ij in c.face (forward face
// kernels run first): R_phi into a.ophi, R_W into a.oW, R_q into a.oq.  One warp per cell.
// ------------------------------------------------------------------------------------
template <int WPB>
__global__ void __launch_bounds__(WPB * 32) k_adj_residual(Dev<double> c, AdjBufs a) {
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * WPB + (threadIdx.x >> 5);
    if (i >= c.N) return;
    const double R = c.R, Z = c.Z;
    const double* W = c.W + 6 * (size_t)i;
    const double* q = c.q + 6 * (size_t)i;
    const Prim p = prim_from_W(W, R);
    const double itau = 1.0 / relax_time(c, p.rho, p.Ttr);
    double e[EQN];
    make_eq<double, double>(c, p.rho, p.U, p.T, p.Ttr, p.Trot, q, q + 3, e);
    const size_t NK = (size_t)c.N * c.Kp, FK = (size_t)c.F * c.Kp;
    const int s0 = c.slot_off[i], s1 = c.slot_off[i + 1];
    double S[12];
#pragma unroll
    for (int j = 0; j < 12; ++j) S[j] = 0.0;
    for (int k = lane; k < c.K; k += 32) {
        const double ux = c.u[k], uy = c.u[c.Kp + k], uz = c.u[2 * c.Kp + k], w = c.w[k];
        double Fg = 0.0, Fh = 0.0;
        for (int m = s0; m < s1; ++m) {
            const int f = c.slot_face[m];
            double un = dot_rn(ux, uy, uz, c.fn[f], c.fn[c.F + f], c.fn[2 * c.F + f]);
            if (!c.slot_left[m]) un = -un;
            Fg += c.slot_AV[m] * un * c.face[(size_t)f * c.Kp + k];
            Fh += c.slot_AV[m] * un * c.face[FK + (size_t)f * c.Kp + k];
        }
        double G, H;
        eval_eq(e, ux, uy, uz, G, H);
        const size_t o = (size_t)i * c.Kp + k;
        const double g = c.phi[o], h = c.phi[NK + o];
        a.ophi[o] = (G - g) * itau - Fg;
        a.ophi[NK + o] = (H - h) * itau - Fh;
        const double dg = g - G, dh = h - H;
        const double cx = ux - p.U[0], cy = uy - p.U[1], cz = uz - p.U[2];
        const double c2 = cx * cx + cy * cy + cz * cz;
        S[0] += w * dg;
        S[1] += w * ux * dg; S[2] += w * uy * dg; S[3] += w * uz * dg;
        S[4] += w * (0.5 * (ux * ux + uy * uy + uz * uz) * dg + dh);
        S[5] += w * dh;
        S[6] += w * cx * c2 * dg; S[7] += w * cy * c2 * dg; S[8] += w * cz * c2 * dg;
        S[9] += w * cx * dh; S[10] += w * cy * dh; S[11] += w * cz * dh;
    }
    warp_sum<12>(S);
    if (lane != 0) return;
    double* oW = a.oW + 6 * (size_t)i;
    double* oq = a.oq + 6 * (size_t)i;
    for (int d = 0; d < 5; ++d) oW[d] = S[d];
    oW[5] = S[5] + p.rho * R * ((1.0 - 1.0 / Z) * p.Trot + p.T / Z) - W[5];
    const double atr = (1.0 / 3.0) * (1.0 - (1.0 - c.omega0) / Z);
    const double arot = (1.0 - c.delta) * (1.0 - (1.0 - c.omega1) / Z);
    for (int d = 0; d < 3; ++d) {
        oq[d] = 0.5 * S[6 + d] + (atr - 1.0) * q[d];
        oq[3 + d] = S[9 + d] + (arot - 1.0) * q[3 + d];
    }
}

// ------------------------------------------------------------------------------------
// interior faces: reverse of Step 2 (b)-(d).  One warp per face.
//   pass 1, 2 : moments of phi0 = phi(x_f - u s) (rho, rho U, rho E, sum w h, then the
//               heat-flux sums and second moments about the interface velocity U)
//   state     : tau, rho E_rot, T_rot, T_tr, q_tr, q_rot as in the forward kernel
//   pass A    : adjoint of phi_ij, wb = -A (u.n)(v_L/V_L - v_R/V_R); reductions of
//               the blend's tau derivative and of phi*'s state derivatives
//   scalar    : reverse of the interface state down to the moments
//   pass B    : adjoint of phi0, written to fbar
// ------------------------------------------------------------------------------------
template <int WPB, typename S = double>
__global__ void __launch_bounds__(WPB * 32, sizeof(S) == 4 ? ADJ_MINB : 1) k_adj_face_interior(Dev<double> c, AdjBufs a) {
    const int lane = threadIdx.x & 31;
    const int fi = blockIdx.x * WPB + (threadIdx.x >> 5);
    if (fi >= c.Fi) return;
    const int f = c.face_int[fi];
    const int cl = c.fc[2 * f], cr = c.fc[2 * f + 1];
    const size_t FK = (size_t)c.F * c.Kp, NK = (size_t)c.N * c.Kp;
    // phi0 at this face in the arithmetic type (the FP32 reconstruction for S = float)
    const S* g0;
    if constexpr (sizeof(S) == 4) g0 = a.f0f + (size_t)f * c.Kp;
    else g0 = a.f0 + (size_t)f * c.Kp;
    const S* h0 = g0 + FK;
    const double Rg = c.R, Z = c.Z, s = c.fs[f];
    using RS = Red<S>;
    double m6[6];
    {
        Acc<S> am[6];
        for (int k = lane; k < c.K; k += 32) {
            const S ux = vel<S>(c, a, 0, k), uy = vel<S>(c, a, 1, k), uz = vel<S>(c, a, 2, k), w = wgt<S>(c, a, k);
            const S wg = w * (S)g0[k], wh = w * (S)h0[k];
            am[0].add(wg);
            am[1].add(wg * ux); am[2].add(wg * uy); am[3].add(wg * uz);
            am[4].add(S(0.5) * (ux * ux + uy * uy + uz * uz) * wg + wh);
            am[5].add(wh);
        }
        typename RS::V v[6];
#pragma unroll
        for (int j = 0; j < 6; ++j) v[j] = RS::from(am[j]);
        warp_red<S, 6>(v);
#pragma unroll
        for (int j = 0; j < 6; ++j) m6[j] = RS::to_d(v[j]);
    }
    const double rho = m6[0], E = m6[4], Er0 = m6[5];
    const double U[3] = {m6[1] / rho, m6[2] / rho, m6[3] / rho};
    const double U2 = U[0] * U[0] + U[1] * U[1] + U[2] * U[2];
    const double ke = 0.5 * rho * U2;
    const double T = (E - ke) / (2.5 * rho * Rg);
    const double Ttr0 = (E - ke - Er0) / (1.5 * rho * Rg);
    const double tau = relax_time(c, rho, Ttr0);
    const double den = Z * tau + s;
    const double Erot = (Z * tau * Er0 + s * rho * Rg * T) / den;
    const double Trot = Erot / (rho * Rg);
    const double Ttr = (E - ke - Erot) / (1.5 * rho * Rg);
    double m12[12];
    {
        const S Us[3] = {(S)U[0], (S)U[1], (S)U[2]};
        Acc<S> am[12];
        for (int k = lane; k < c.K; k += 32) {
            const S cx = vel<S>(c, a, 0, k) - Us[0], cy = vel<S>(c, a, 1, k) - Us[1], cz = vel<S>(c, a, 2, k) - Us[2];
            const S w = wgt<S>(c, a, k);
            const S wg = w * (S)g0[k], wh = w * (S)h0[k];
            const S wgc2 = wg * (cx * cx + cy * cy + cz * cz);
            am[0].add(wgc2 * cx); am[1].add(wgc2 * cy); am[2].add(wgc2 * cz);
            am[3].add(wh * cx); am[4].add(wh * cy); am[5].add(wh * cz);
            am[6].add(wg * cx * cx); am[7].add(wg * cy * cy); am[8].add(wg * cz * cz);
            am[9].add(wg * cx * cy); am[10].add(wg * cx * cz); am[11].add(wg * cy * cz);
        }
        typename RS::V v[12];
#pragma unroll
        for (int j = 0; j < 12; ++j) v[j] = RS::from(am[j]);
        warp_red<S, 12>(v);
#pragma unroll
        for (int j = 0; j < 12; ++j) m12[j] = RS::to_d(v[j]);
    }
    const double dtr = tau + s - s / 3.0 * (1.0 - 1.0 / Z + c.omega0 / Z);
    const double drot = tau + s - s * (1.0 - c.delta) * (1.0 - 1.0 / Z + c.omega1 / Z);
    double qtr[3], qrot[3];
    for (int d = 0; d < 3; ++d) {
        qtr[d] = tau * 0.5 * m12[d] / dtr;
        qrot[d] = tau * m12[3 + d] / drot;
    }
    const S Us[3] = {(S)U[0], (S)U[1], (S)U[2]};
    const S qts[3] = {(S)qtr[0], (S)qtr[1], (S)qtr[2]}, qrs[3] = {(S)qrot[0], (S)qrot[1], (S)qrot[2]};
    const EqS<S> st = make_eqs<S>((S)rho, Us, (S)(Rg * T), (S)(Rg * Ttr), (S)(Rg * Trot), qts, qrs);
    const S om0 = (S)c.omega0, om1 = (S)c.omega1, del = (S)c.delta, ZS = (S)Z;
    const double ab = tau / (tau + s), bb = s / (tau + s), db = s / ((tau + s) * (tau + s));
    const double nx = c.fn[f], ny = c.fn[c.F + f], nz = c.fn[2 * c.F + f], A = c.fa[f];
    const double iVl = 1.0 / c.vol[cl], iVr = 1.0 / c.vol[cr];
    const size_t ol = (size_t)cl * c.Kp, orr = (size_t)cr * c.Kp;   // rows of v at the two cells
    double acc[14];
    {
        const S nxs = (S)nx, nys = (S)ny, nzs = (S)nz, As = (S)A, iVls = (S)iVl, iVrs = (S)iVr;
        const S bbs = (S)bb, dbs = (S)db;
        Acc<S> am[14];
        for (int k = lane; k < c.K; k += 32) {
            const S ux = vel<S>(c, a, 0, k), uy = vel<S>(c, a, 1, k), uz = vel<S>(c, a, 2, k);
            const S wn = -As * dot_rn(ux, uy, uz, nxs, nys, nzs);
            const S wgb = wn * (vin<S>(a, ol + k) * iVls - vin<S>(a, orr + k) * iVrs);
            const S whb = wn * (vin<S>(a, NK + ol + k) * iVls - vin<S>(a, NK + orr + k) * iVrs);
            S G, H, dd[13];
            eq_vjp<S>(st, om0, om1, del, ZS, ux, uy, uz, bbs * wgb, bbs * whb, dd, G, H);
#pragma unroll
            for (int j = 0; j < 13; ++j) am[j].add(dd[j]);
            am[13].add((wgb * ((S)g0[k] - G) + whb * ((S)h0[k] - H)) * dbs);
        }
        typename RS::V v[14];
#pragma unroll
        for (int j = 0; j < 14; ++j) v[j] = RS::from(am[j]);
        warp_red<S, 14>(v);
#pragma unroll
        for (int j = 0; j < 14; ++j) acc[j] = RS::to_d(v[j]);
    }
    // reverse of the interface state
    double rb = acc[0], Ub[3] = {acc[1], acc[2], acc[3]};
    double Tb = Rg * acc[4], Ttrb = Rg * acc[5], Trotb = Rg * acc[6], taub = acc[13];
    double Qtb[3], Qrb[3];
    for (int d = 0; d < 3; ++d) {
        Qtb[d] = acc[7 + d] * tau * 0.5 / dtr;
        taub += acc[7 + d] * 0.5 * m12[d] * (dtr - tau) / (dtr * dtr);
        Qrb[d] = acc[10 + d] * tau / drot;
        taub += acc[10 + d] * m12[3 + d] * (drot - tau) / (drot * drot);
    }
    {   // heat-flux sums depend on U through c = u - U
        const double P2 = m12[6] + m12[7] + m12[8];
        const double S[3][3] = {{m12[6], m12[9], m12[10]}, {m12[9], m12[7], m12[11]}, {m12[10], m12[11], m12[8]}};
        for (int e2 = 0; e2 < 3; ++e2) {
            double t = Qtb[e2] * P2 + Qrb[e2] * Er0;
            for (int d = 0; d < 3; ++d) t += 2.0 * Qtb[d] * S[d][e2];
            Ub[e2] -= t;
        }
    }
    const double k15 = 1.0 / (1.5 * rho * Rg), k25 = 1.0 / (2.5 * rho * Rg);
    double Eb = Ttrb * k15, keb = -Ttrb * k15, Erotb = -Ttrb * k15;
    rb -= Ttrb * Ttr / rho;
    Erotb += Trotb / (rho * Rg);
    rb -= Trotb * Trot / rho;
    taub += Erotb * Z * (Er0 - Erot) / den;
    double Er0b = Erotb * Z * tau / den;
    rb += Erotb * s * Rg * T / den;
    Tb += Erotb * s * rho * Rg / den;
    const double Ttr0b = taub * tau * (viscosity_slope(c, Ttr0) - 1.0) / Ttr0;
    rb -= taub * tau / rho;
    Eb += Ttr0b * k15; keb -= Ttr0b * k15; Er0b -= Ttr0b * k15;
    rb -= Ttr0b * Ttr0 / rho;
    Eb += Tb * k25; keb -= Tb * k25;
    rb -= Tb * T / rho;
    rb += keb * 0.5 * U2;
    double mb[3], UbU = 0.0;
    for (int d = 0; d < 3; ++d) {
        Ub[d] += keb * rho * U[d];
        mb[d] = Ub[d] / rho;
        UbU += Ub[d] * U[d];
    }
    rb -= UbU / rho;
    double* gb = a.fbar + (size_t)f * c.Kp;
    double* hb = a.fbar + FK + (size_t)f * c.Kp;
    const S nxs = (S)nx, nys = (S)ny, nzs = (S)nz, As = (S)A, iVls = (S)iVl, iVrs = (S)iVr, abs_ = (S)ab;
    const S rbs = (S)rb, mbs[3] = {(S)mb[0], (S)mb[1], (S)mb[2]}, Ebs = (S)Eb, Eh = (S)(Eb + Er0b);
    const S Qts[3] = {(S)Qtb[0], (S)Qtb[1], (S)Qtb[2]}, Qrs[3] = {(S)Qrb[0], (S)Qrb[1], (S)Qrb[2]};
    for (int k = lane; k < c.K; k += 32) {
        const S ux = vel<S>(c, a, 0, k), uy = vel<S>(c, a, 1, k), uz = vel<S>(c, a, 2, k), w = wgt<S>(c, a, k);
        const S wn = -As * dot_rn(ux, uy, uz, nxs, nys, nzs);
        const S wgb = wn * (vin<S>(a, ol + k) * iVls - vin<S>(a, orr + k) * iVrs);
        const S whb = wn * (vin<S>(a, NK + ol + k) * iVls - vin<S>(a, NK + orr + k) * iVrs);
        const S cx = ux - Us[0], cy = uy - Us[1], cz = uz - Us[2];
        const S c2 = cx * cx + cy * cy + cz * cz;
        gb[k] = (double)(abs_ * wgb + w * (rbs + mbs[0] * ux + mbs[1] * uy + mbs[2] * uz +
                                         Ebs * S(0.5) * (ux * ux + uy * uy + uz * uz) +
                                         c2 * (Qts[0] * cx + Qts[1] * cy + Qts[2] * cz)));
        hb[k] = (double)(abs_ * whb + w * (Eh + Qrs[0] * cx + Qrs[1] * cy + Qrs[2] * cz));
    }
}

// ------------------------------------------------------------------------------------
// boundary faces: reverse of the wall / farfield treatment (no interface collision).
// Seeds: -A (u.n) v_i / V_i from R_phi, plus obj_scale times the derivative of the
// objective at wall faces (heat: A w (u.n)(|u|^2/2 g + h); drag: A w (u.n)(u.e) g).
// Writes fbar at outgoing velocities and per face fpar = (dT_w, drho_inf, dU_inf[3],
// dT_inf, J_f, force_f[3]).  One block per boundary face.
// ------------------------------------------------------------------------------------
template <int BS>
__global__ void __launch_bounds__(BS) k_adj_face_boundary(Dev<double> c, AdjBufs a) {
    __shared__ double red[12 * (BS / 32)];
    __shared__ double sh[4];
    const int b = blockIdx.x;
    const int f = c.face_bnd[b];
    const int bc = -1 - c.fc[2 * f + 1];
    const int kind = c.bck[bc];
    const int i = c.fc[2 * f];
    const size_t FK = (size_t)c.F * c.Kp, NK = (size_t)c.N * c.Kp;
    const double* g0 = a.f0 + (size_t)f * c.Kp;
    const double* h0 = a.f0 + FK + (size_t)f * c.Kp;
    double* gbar = a.fbar + (size_t)f * c.Kp;
    double* hbar = a.fbar + FK + (size_t)f * c.Kp;
    const double nx = c.fn[f], ny = c.fn[c.F + f], nz = c.fn[2 * c.F + f], A = c.fa[f];
    const double iV = 1.0 / c.vol[i];
    const double* bv = c.bcv + 5 * bc;
    const double Tb0 = bv[4], RT = c.R * Tb0;
    const double rho_b = (kind == 0) ? 1.0 : bv[0];
    const double an = 2.0 * PI * RT;
    const double Mn = rho_b / (an * sqrt(an)), Mx = 1.0 / (2.0 * RT);
    const bool wall = kind == 0;
    const double seed = wall ? a.obj_scale : 0.0;
    const double* vg = a.vphi + (size_t)i * c.Kp;
    double num = 0.0, dn = 0.0;
    if (wall) {
        double v[2] = {0.0, 0.0};
        for (int k = threadIdx.x; k < c.K; k += BS) {
            const double ux = c.u[k], uy = c.u[c.Kp + k], uz = c.u[2 * c.Kp + k], w = c.w[k];
            const double un = dot_rn(ux, uy, uz, nx, ny, nz);
            if (un > 0.0) {
                v[0] += w * un * g0[k];
            } else {
                const double cx = ux - bv[1], cy = uy - bv[2], cz = uz - bv[3];
                v[1] += -w * un * Mn * exp(-(cx * cx + cy * cy + cz * cz) * Mx);
            }
        }
        block_sum<2, BS>(v, red);
        num = v[0];
        dn = v[1];
    }
    const double rw = wall ? num / dn : 1.0;
    double acc[12];
#pragma unroll
    for (int j = 0; j < 12; ++j) acc[j] = 0.0;
    // acc: 0 rho_w adjoint, 1 T_w adjoint (direct), 2 d(den)/dT_w, 3 rho_inf, 4-6 U_inf,
    //      7 T_inf, 8 J_f, 9-11 force_f
    for (int k = threadIdx.x; k < c.K; k += BS) {
        const double ux = c.u[k], uy = c.u[c.Kp + k], uz = c.u[2 * c.Kp + k], w = c.w[k];
        const double un = dot_rn(ux, uy, uz, nx, ny, nz);
        const double u2h = 0.5 * (ux * ux + uy * uy + uz * uz);
        double wgb = -A * un * vg[k] * iV, whb = -A * un * vg[NK + k] * iV;
        if (seed != 0.0) {
            if (a.objective == 0) {
                wgb += seed * A * w * un * u2h;
                whb += seed * A * w * un;
            } else {
                wgb += seed * A * w * un * (ux * a.edrag[0] + uy * a.edrag[1] + uz * a.edrag[2]);
            }
        }
        double gf, hf;
        if (un > 0.0) {
            gf = g0[k];
            hf = h0[k];
            gbar[k] = wgb;
            hbar[k] = whb;
        } else {
            const double cx = ux - bv[1], cy = uy - bv[2], cz = uz - bv[3];
            const double c2 = cx * cx + cy * cy + cz * cz;
            const double M = Mn * exp(-c2 * Mx);
            const double dMdT = M * (c2 / (2.0 * c.R * Tb0 * Tb0) - 1.5 / Tb0);
            if (wall) {
                gf = rw * M;
                hf = RT * gf;
                acc[0] += wgb * M + whb * RT * M;
                acc[1] += wgb * rw * dMdT + whb * rw * c.R * (M + Tb0 * dMdT);
                acc[2] += -w * un * dMdT;
            } else {
                gf = M;
                hf = RT * M;
                const double X = wgb + whb * RT;
                acc[3] += X * M / rho_b;
                acc[4] += X * M * cx / RT;
                acc[5] += X * M * cy / RT;
                acc[6] += X * M * cz / RT;
                acc[7] += X * dMdT + whb * c.R * M;
            }
        }
        if (wall) {
            acc[8] += A * w * un * (u2h * gf + hf);
            acc[9] += A * w * un * ux * gf;
            acc[10] += A * w * un * uy * gf;
            acc[11] += A * w * un * uz * gf;
        }
    }
    block_sum<12, BS>(acc, red);
    if (threadIdx.x == 0) {
        double* o = a.fpar + (size_t)b * ADJ_FPAR;
        double numb = 0.0;
        for (int j = 0; j < ADJ_FPAR; ++j) o[j] = 0.0;
        if (wall) {
            numb = acc[0] / dn;
            o[0] = acc[1] - acc[0] * num / (dn * dn) * acc[2];
            o[6] = a.objective == 0 ? acc[8]
                                    : acc[9] * a.edrag[0] + acc[10] * a.edrag[1] + acc[11] * a.edrag[2];
            o[7] = acc[9]; o[8] = acc[10]; o[9] = acc[11];
        } else {
            for (int j = 0; j < 5; ++j) o[1 + j] = acc[3 + j];
        }
        sh[0] = numb;
    }
    __syncthreads();
    if (wall) {
        const double numb = sh[0];
        for (int k = threadIdx.x; k < c.K; k += BS) {
            const double un = dot_rn(c.u[k], c.u[c.Kp + k], c.u[2 * c.Kp + k], nx, ny, nz);
            if (un > 0.0) gbar[k] += numb * c.w[k] * un;
        }
    }
}

// ------------------------------------------------------------------------------------
// cell gather 1: adjoint of phi0 from the faces where the cell is upwind, then the
// reverse of phi0 = phi_c + (x_f - u s - x_c) . L g (Eq. flux_solve_phi_phi) through the
// Venkatakrishnan limiter (Sec. 3.3 readings: minimum over faces capped at 1, eps^2
// phi_c^2 threshold) and the least-squares gradient g = sum_j M^-1 d_j (phi_j - phi_c).
// Adds the cell's own terms to ophi and leaves, per (cell, velocity, field), the
// gradient adjoint and the Delta_max/min adjoint with the slot of the neighbour that
// gave it, for the neighbours to gather.  One warp per cell.
// ------------------------------------------------------------------------------------
template <int WPB, typename S = double>
__global__ void __launch_bounds__(WPB * 32, sizeof(S) == 4 ? ADJ_MINB : 1) k_adj_gather(Dev<double> c, AdjBufs a) {
    __shared__ int s_face[WPB][MAXF], s_nbr[WPB][MAXF], s_left[WPB][MAXF];
    __shared__ S s_lsq[WPB][3][MAXF], s_d[WPB][3][MAXF], s_n[WPB][3][MAXF], s_s[WPB][MAXF];
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const int i = blockIdx.x * WPB + wp;
    if (i >= c.N) return;
    const int s0 = c.slot_off[i], ns = c.slot_off[i + 1] - s0;
    if (lane < ns) {
        const int m = s0 + lane;
        const int f = c.slot_face[m];
        s_face[wp][lane] = f;
        s_nbr[wp][lane] = c.slot_nbr[m];
        s_left[wp][lane] = c.slot_left[m];
        s_s[wp][lane] = (S)c.fs[f];
        for (int r = 0; r < 3; ++r) {
            s_lsq[wp][r][lane] = (S)c.slot_lsq[r * c.nnz + m];
            s_d[wp][r][lane] = (S)c.slot_d[r * c.nnz + m];
            s_n[wp][r][lane] = (S)c.slot_n[r * c.nnz + m];
        }
    }
    __syncwarp();
    const S eps2 = (S)c.eps2[i];
    const int limiter = (int)a.iterp[1];
    const size_t NK = (size_t)c.N * c.Kp, FK = (size_t)c.F * c.Kp;
    for (int k = lane; k < c.K; k += 32) {
        const S ux = vel<S>(c, a, 0, k), uy = vel<S>(c, a, 1, k), uz = vel<S>(c, a, 2, k);
        for (int fd = 0; fd < 2; ++fd) {
            const size_t fo = fd * NK;
            const S pc = dist<S>(c, a, fo + (size_t)i * c.Kp + k);
            // forward: gradient, Delta_max/min with the slot that gave them
            S g[3] = {S(0), S(0), S(0)}, dmax = S(0), dmin = S(0);
            int amax = -1, amin = -1;
            for (int q = 0; q < ns; ++q) {
                const int j = s_nbr[wp][q];
                if (j < 0) continue;
                const S dp = dist<S>(c, a, fo + (size_t)j * c.Kp + k) - pc;
                g[0] += s_lsq[wp][0][q] * dp; g[1] += s_lsq[wp][1][q] * dp; g[2] += s_lsq[wp][2][q] * dp;
                if (dp > dmax) { dmax = dp; amax = q; }
                if (dp < dmin) { dmin = dp; amin = q; }
            }
            S L = (limiter == 2) ? S(0) : S(1);
            int lq = -1;
            if (limiter == 3) {
                L = (S)c.lstore[fd * NK + (size_t)i * c.Kp + k];  // frozen: a constant
            } else if (limiter == 1) {
                // the forward kernel's minimum: psi at the face of largest d2 (with
                // Delta_max) and at the face of smallest d2 (with Delta_min)
                S d2hi = S(0), d2lo = S(0);
                int qhi = -1, qlo = -1;
                for (int q = 0; q < ns; ++q) {
                    const S d2 = g[0] * s_d[wp][0][q] + g[1] * s_d[wp][1][q] + g[2] * s_d[wp][2][q];
                    if (d2 > d2hi) { d2hi = d2; qhi = q; }
                    if (d2 < d2lo) { d2lo = d2; qlo = q; }
                }
                const S ep = eps2 * pc * pc;
                if (qhi >= 0) {
                    const S d1 = dmax, d2 = d2hi;
                    const S nu = d1 * d1 + ep + S(2) * d1 * d2;
                    const S de = d1 * d1 + S(2) * d2 * d2 + d1 * d2 + ep;
                    if (nu < de) { L = lim_div(nu, de); lq = qhi; }
                }
                if (qlo >= 0) {
                    const S d1 = dmin, d2 = d2lo;
                    const S nu = d1 * d1 + ep + S(2) * d1 * d2;
                    const S de = d1 * d1 + S(2) * d2 * d2 + d1 * d2 + ep;
                    if (nu < L * de) { L = lim_div(nu, de); lq = qlo; }
                }
            }
            // adjoint of phi0 gathered over the faces where this cell is upwind
            S self = S(0), Gb[3] = {S(0), S(0), S(0)};
            const double* fb = a.fbar + fd * FK;
            for (int q = 0; q < ns; ++q) {
                const S un = dot_rn(ux, uy, uz, s_n[wp][0][q], s_n[wp][1][q], s_n[wp][2][q]);
                const bool up = s_left[wp][q] ? (un > S(0)) : (un <= S(0));
                if (!up) continue;
                const S x = (S)fb[(size_t)s_face[wp][q] * c.Kp + k];
                const S sq = s_s[wp][q];
                self += x;
                Gb[0] += (s_d[wp][0][q] - ux * sq) * x;
                Gb[1] += (s_d[wp][1][q] - uy * sq) * x;
                Gb[2] += (s_d[wp][2][q] - uz * sq) * x;
            }
            // reverse of L g
            const S Lb = Gb[0] * g[0] + Gb[1] * g[1] + Gb[2] * g[2];
            S gb[3] = {L * Gb[0], L * Gb[1], L * Gb[2]};
            S d1b = S(0);
            int slot = -1;
            if (limiter == 1 && lq >= 0) {
                const S dx = s_d[wp][0][lq], dy = s_d[wp][1][lq], dz = s_d[wp][2][lq];
                const S d2 = g[0] * dx + g[1] * dy + g[2] * dz;
                const S d1 = d2 > S(0) ? dmax : dmin;
                const S ep = eps2 * pc * pc;
                S Lp2, Lself, Lp1;          // Lb times the partial derivatives of psi
                if constexpr (sizeof(S) == 8) {
                    const S nu = d1 * d1 + ep + S(2) * d1 * d2;
                    const S de = d1 * d1 + S(2) * d2 * d2 + d1 * d2 + ep;
                    const S ide2 = S(1) / (de * de);
                    Lp1 = Lb * (((S(2) * d1 + S(2) * d2) * de - nu * (S(2) * d1 + d2)) * ide2);
                    Lp2 = Lb * ((S(2) * d1 * de - nu * (S(4) * d2 + d1)) * ide2);
                    Lself = Lb * ((de - nu) * ide2) * S(2) * eps2 * pc;    // through ep
                } else {
                    // FP32: psi is homogeneous of degree 0 in (d1, d2, sqrt(ep)); its
                    // derivatives are formed from the values scaled by
                    // sigma = max(|d1|, |d2|) and divided by sigma (sigma^2 for ep), which
                    // keeps them in range.  Below sigma = 1e-30 (the far tails of the
                    // distributions) the limiter is taken as constant.
                    const S sg = fmaxf(fabsf(d1), fabsf(d2));
                    Lp1 = Lp2 = Lself = S(0);
                    if (sg > S(1e-30)) {
                        const S is = S(1) / sg, a1 = d1 * is, a2 = d2 * is, e = (ep * is) * is;
                        const S nu = a1 * a1 + e + S(2) * a1 * a2;
                        const S de = a1 * a1 + S(2) * a2 * a2 + a1 * a2 + e;
                        const S ide2 = S(1) / (de * de);
                        const S Lbs = Lb * is;
                        Lp1 = Lbs * (((S(2) * a1 + S(2) * a2) * de - nu * (S(2) * a1 + a2)) * ide2);
                        Lp2 = Lbs * ((S(2) * a1 * de - nu * (S(4) * a2 + a1)) * ide2);
                        Lself = (Lbs * ((de - nu) * ide2)) * ((S(2) * eps2 * pc) * is);
                    }
                }
                gb[0] += Lp2 * dx; gb[1] += Lp2 * dy; gb[2] += Lp2 * dz;
                self += Lself;
                const int arg = d2 > S(0) ? amax : amin;
                if (arg >= 0) {
                    d1b = Lp1;
                    self -= d1b;
                    slot = arg;
                }
            }
            // reverse of the least-squares gradient: the cell's own part
            for (int q = 0; q < ns; ++q) {
                if (s_nbr[wp][q] < 0) continue;
                self -= s_lsq[wp][0][q] * gb[0] + s_lsq[wp][1][q] * gb[1] + s_lsq[wp][2][q] * gb[2];
            }
            const size_t o = (size_t)i * c.Kp + k;
            a.ophi[fd * NK + o] += (double)self;
            // the gradient and Delta adjoints, stored in the arithmetic type
            S* nb = reinterpret_cast<S*>(a.nbg) + (size_t)fd * 4 * NK;
            nb[o] = gb[0];
            nb[NK + o] = gb[1];
            nb[2 * NK + o] = gb[2];
            nb[3 * NK + o] = d1b;
            a.nbs[fd * NK + o] = (signed char)slot;
        }
    }
}

// cell gather 2: the neighbours' gradient and Delta terms that involve this cell's
// value: sum over neighbours c of  lsq_c(this) . gb_c  +  [c's Delta came from this
// cell] d1b_c.  One warp per cell.
template <int WPB, typename S = double>
__global__ void __launch_bounds__(WPB * 32) k_adj_gather2(Dev<double> c, AdjBufs a) {
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * WPB + (threadIdx.x >> 5);
    if (i >= c.N) return;
    const int s0 = c.slot_off[i], s1 = c.slot_off[i + 1];
    const size_t NK = (size_t)c.N * c.Kp;
    for (int k = lane; k < c.K; k += 32) {
        S acc[2] = {S(0), S(0)};
        for (int m = s0; m < s1; ++m) {
            const int j = c.slot_nbr[m];
            if (j < 0) continue;
            const int mm = a.slot_mirg[m];
            const int loc = mm - c.slot_off[j];
            const S lx = (S)c.slot_lsq[mm], ly = (S)c.slot_lsq[c.nnz + mm], lz = (S)c.slot_lsq[2 * c.nnz + mm];
            const size_t o = (size_t)j * c.Kp + k;
            for (int fd = 0; fd < 2; ++fd) {
                const S* nb = reinterpret_cast<const S*>(a.nbg) + (size_t)fd * 4 * NK;
                S t = lx * nb[o] + ly * nb[NK + o] + lz * nb[2 * NK + o];
                if (a.nbs[fd * NK + o] == loc) t += nb[3 * NK + o];
                acc[fd] += t;
            }
        }
        const size_t o = (size_t)i * c.Kp + k;
        a.ophi[o] += (double)acc[0];
        a.ophi[NK + o] += (double)acc[1];
    }
}

// Sum of the per-boundary-face records in face order (one block of 32 threads): out[0-5]
// (dR/dp)^T v or dJ/dp|_X, out[6] J, out[7-9] force.
__global__ void k_adj_params(const double* fpar, int Fb, double* out) {
    const int j = threadIdx.x;
    if (j >= 10) return;
    double s = 0.0;
    for (int b = 0; b < Fb; ++b) s += fpar[(size_t)b * ADJ_FPAR + j];
    out[j] = s;
}

// ------------------------------------------------------------------------------------
// preconditioner: transposed point Gauss-Seidel sweep of the first-order implicit
// operator of Eq. implicit_mic_final_equ for the cells of one colour,
//   y_i = (r_i + sum_j (A/V_j) max(u.n_ij, 0) y_j) / D_i,
//   D_i = 1/(cfl dt_i) + 1/tau_i + sum_f (A/V_i) max(u.n_if, 0)
// (the transpose of the micro PR-SGS operator: entry (i, j) is (A/V_j) min(u.n_ji, 0)).
// One warp per cell.
// ------------------------------------------------------------------------------------
template <int WPB, typename S = double>
__global__ void __launch_bounds__(WPB * 32) k_adj_sweep(Dev<double> c, AdjBufs a, const int* cells,
                                                        int n, const double* r, double* y) {
    const int lane = threadIdx.x & 31;
    const int t = blockIdx.x * WPB + (threadIdx.x >> 5);
    if (t >= n) return;
    const int i = cells[t];
    const int s0 = c.slot_off[i], s1 = c.slot_off[i + 1];
    const size_t NK = (size_t)c.N * c.Kp;
    const S base = (S)(1.0 / (c.cfl_imp * c.dt[i]) + 1.0 / a.tau[i]);
    for (int k = lane; k < c.K; k += 32) {
        const S ux = vel<S>(c, a, 0, k), uy = vel<S>(c, a, 1, k), uz = vel<S>(c, a, 2, k);
        S D = base, ag = S(0), ah = S(0);
        for (int m = s0; m < s1; ++m) {
            S un = dot_rn(ux, uy, uz, (S)c.slot_n[m], (S)c.slot_n[c.nnz + m], (S)c.slot_n[2 * c.nnz + m]);
            if (!c.slot_left[m]) un = -un;
            if (!(un > S(0))) continue;
            D += (S)c.slot_AV[m] * un;
            const int j = c.slot_nbr[m];
            if (j < 0) continue;
            const S cf = (S)a.slot_AVn[m] * un;
            ag += cf * (S)y[(size_t)j * c.Kp + k];
            ah += cf * (S)y[NK + (size_t)j * c.Kp + k];
        }
        const size_t o = (size_t)i * c.Kp + k;
        y[o] = (double)(((S)r[o] + ag) / D);
        y[NK + o] = (double)(((S)r[NK + o] + ah) / D);
    }
}

// tau(W_i) per cell
__global__ void k_adj_tau(Dev<double> c, double* tau) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= c.N) return;
    const Prim p = prim_from_W(c.W + 6 * (size_t)i, c.R);
    tau[i] = relax_time(c, p.rho, p.Ttr);
}

// ------------------------------------------------------------------------------------
// vectors X = (phi [2][N][K], W [N][6], q [N][6]) in the packed (unpadded) layout of the
// interface <-> padded internal arrays
// ------------------------------------------------------------------------------------
__global__ void k_adj_unpack(const double* x, int N, int K, int Kp, double* phi, double* W, double* q) {
    const size_t n1 = 2 * (size_t)N * K;
    const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (t < n1) {
        const size_t row = t / K, k = t % K;
        phi[row * Kp + k] = x[t];
    } else if (t < n1 + 6 * (size_t)N) {
        W[t - n1] = x[t];
    } else if (t < n1 + 12 * (size_t)N) {
        q[t - n1 - 6 * (size_t)N] = x[t];
    }
}

__global__ void k_adj_pack(const double* phi, const double* W, const double* q, int N, int K, int Kp, double* x) {
    const size_t n1 = 2 * (size_t)N * K;
    const size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (t < n1) {
        const size_t row = t / K, k = t % K;
        x[t] = phi[row * Kp + k];
    } else if (t < n1 + 6 * (size_t)N) {
        x[t] = W[t - n1];
    } else if (t < n1 + 12 * (size_t)N) {
        x[t] = q[t - n1 - 6 * (size_t)N];
    }
}

// per-velocity arrays of a mixed-precision context in FP64 and back, and s_ij per slot
__global__ void k_adj_upcast(const float* src, double* dst, size_t n) {
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
        dst[t] = (double)src[t];
}
__global__ void k_adj_downcast(const double* src, float* dst, size_t n) {
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
        dst[t] = (float)src[t];
}
__global__ void k_adj_slot_s(DevBase c, double* slot_s) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m < c.nnz) slot_s[m] = c.fs[c.slot_face[m]];
}

// ------------------------------------------------------------------------------------
// Krylov vector kernels on packed vectors of length n (deterministic: fixed grid, block
// partial sums combined in block order by k_vec_finish)
// ------------------------------------------------------------------------------------
constexpr int VEC_BS = 256, VEC_GRID = 1024;
constexpr int GM_MAX = 64;      // maximum Krylov dimension of one restart cycle

// part[b * m + j] = sum over the block's range of x . V_j, j < m (V_j = V + j * ld)
__global__ void __launch_bounds__(VEC_BS) k_vec_mdot(const double* x, const double* V, size_t ld, int m,
                                                      size_t n, double* part) {
    __shared__ double red[VEC_BS / 32];
    for (int j = 0; j < m; ++j) {
        const double* v = V + (size_t)j * ld;
        double s = 0.0;
        for (size_t t = blockIdx.x * (size_t)VEC_BS + threadIdx.x; t < n; t += (size_t)VEC_GRID * VEC_BS)
            s += x[t] * v[t];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double tsum = red[0];
            for (int q = 1; q < VEC_BS / 32; ++q) tsum += red[q];
            part[(size_t)blockIdx.x * m + j] = tsum;
        }
        __syncthreads();
    }
}

__global__ void k_vec_finish(const double* part, int m, double* out) {
    const int j = threadIdx.x;
    if (j >= m) return;
    double s = 0.0;
    for (int b = 0; b < VEC_GRID; ++b) s += part[(size_t)b * m + j];
    out[j] = s;
}

// x -= sum_j h[j] V_j  (h on the device)
__global__ void k_vec_msub(double* x, const double* V, size_t ld, int m, const double* h, size_t n) {
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
        double s = x[t];
        for (int j = 0; j < m; ++j) s -= h[j] * V[(size_t)j * ld + t];
        x[t] = s;
    }
}

// y = a x + b y (a term with a zero coefficient is not read)
__global__ void k_vec_axpby(double a, const double* x, double b, double* y, size_t n) {
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
        y[t] = (a == 0.0 ? 0.0 : a * x[t]) + (b == 0.0 ? 0.0 : b * y[t]);
}

// y += sum_j c[j] V_j  (c on the device)
__global__ void k_vec_madd(double* y, const double* V, size_t ld, int m, const double* cc, size_t n) {
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
        double s = y[t];
        for (int j = 0; j < m; ++j) s += cc[j] * V[(size_t)j * ld + t];
        y[t] = s;
    }
}


// ------------------------------------------------------------------------------------
// Macroscopic part of the adjoint preconditioner.  The forward iteration (Sec. 3.5)
// predicts W~ from the moments of the micro residual by the implicit macroscopic
// system (Eq. implicit_mac_equ_fin) before the micro sweeps use phi*(W~); linearised
// at a steady state it maps a residual r to
//   dW~ = L^-1 M_W r_phi,  dphi = S^-1 (r_phi + B_W dW~),  dY = M_Y dphi + r_Y,
// L the macro operator, S the micro PR-SGS operator, M_W / M_Y the moment rows of R_W /
// (R_W, R_q), B_W = dR_phi/dW.  Its transpose, applied by these kernels with the
// transposed micro sweeps, is the adjoint's preconditioner.
// ------------------------------------------------------------------------------------
// out = base + sgn * M_Y^T (yW, yq) per (cell, velocity): the weights of phi in the rows
// R_W (moments 1, u, |u|^2/2 of g; h in the energy rows) and R_q (c|c|^2/2 of g, c of h,
// c = u - U(W)); base may be null (zero).
__global__ void k_adj_momT(Dev<double> c, const double* base, const double* yW, const double* yq,
                           double sgn, double* out) {
    const size_t NK = (size_t)c.N * c.Kp;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < NK; t += (size_t)gridDim.x * blockDim.x) {
        const size_t i = t / c.Kp;
        const int k = (int)(t - i * c.Kp);
        double og = 0.0, oh = 0.0;
        if (k < c.K) {
            const double* W = c.W + 6 * i;
            const double rho = W[0], U[3] = {W[1] / rho, W[2] / rho, W[3] / rho};
            const double ux = c.u[k], uy = c.u[c.Kp + k], uz = c.u[2 * c.Kp + k], w = c.w[k];
            const double* a = yW + 6 * i;
            const double* b = yq + 6 * i;
            const double cx = ux - U[0], cy = uy - U[1], cz = uz - U[2];
            const double c2 = cx * cx + cy * cy + cz * cz;
            og = w * (a[0] + ux * a[1] + uy * a[2] + uz * a[3] + 0.5 * (ux * ux + uy * uy + uz * uz) * a[4] +
                      0.5 * c2 * (cx * b[0] + cy * b[1] + cz * b[2]));
            oh = w * (a[4] + a[5] + cx * b[3] + cy * b[4] + cz * b[5]);
        }
        out[t] = (base ? base[t] : 0.0) + sgn * og;
        out[NK + t] = (base ? base[NK + t] : 0.0) + sgn * oh;
    }
}

// Per cell: 1/D and 1/(D + 1/(Z tau)) of the macro operator, D = 1/(cfl dt) +
// sum_f (A_f / 2V) r_f (the forward macro solve's diagonal, Eq. implicit_mac_equ_fin)
__global__ void k_adj_macro_prep(Dev<double> c, const double* tau, double* dinv) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= c.N) return;
    double D = 1.0 / (c.cfl_imp * c.dt[i]);
    const double iv = 1.0 / c.vol[i];
    for (int m = c.slot_off[i]; m < c.slot_off[i + 1]; ++m) {
        const int f = c.slot_face[m];
        D += 0.5 * c.fa[f] * iv * c.rf[f];
    }
    dinv[2 * (size_t)i] = 1.0 / D;
    dinv[2 * (size_t)i + 1] = 1.0 / (D + 1.0 / (c.Z * tau[i]));
}

// J(W; n)^T y: the transposed Jacobian of the Euler flux G(W).n (Eq.
// implicit_mac_equ_euler_flux; p = (2/5)(rho E - rho |U|^2 / 2), rotational energy
// convected) applied to y, i.e. the gradient of y . G(W; n) in W
__device__ __forceinline__ void euler_jt(const double* W, double nx, double ny, double nz, const double* y,
                                         double* o) {
    const double rho = W[0], ir = 1.0 / rho;
    const double U[3] = {W[1] * ir, W[2] * ir, W[3] * ir};
    const double Un = U[0] * nx + U[1] * ny + U[2] * nz;
    const double U2 = U[0] * U[0] + U[1] * U[1] + U[2] * U[2];
    const double p = 0.4 * (W[4] - 0.5 * rho * U2);
    const double s = y[1] * W[1] + y[2] * W[2] + y[3] * W[3];
    const double yn = y[1] * nx + y[2] * ny + y[3] * nz;
    const double EpUn = (W[4] + p) * ir;          // (E + p) / rho
    o[0] = -s * Un * ir + yn * 0.2 * U2 + y[4] * (0.2 * U2 * Un - EpUn * Un) - y[5] * W[5] * Un * ir;
    const double n[3] = {nx, ny, nz};
    for (int k = 0; k < 3; ++k)
        o[1 + k] = y[0] * n[k] + y[1 + k] * Un + s * n[k] * ir - 0.4 * yn * U[k] +
                   y[4] * (-0.4 * U[k] * Un + EpUn * n[k]) + y[5] * W[5] * n[k] * ir;
    o[4] = 0.4 * yn + 1.4 * y[4] * Un;
    o[5] = y[5] * Un;
}

// One colour phase of a point Gauss-Seidel sweep on the transposed macro operator L^T:
// for every cell j of the colour, y_j = D_j^-1 (b_j - sum_i c_ij (J(W_j; n_ij)^T y_i -
// r_ij y_i)) over the interior neighbours i, c_ij = A_f / (2 V_i), n_ij the normal out
// of i (the forward operator's coefficient of dW_j in cell i's row, transposed).
__global__ void __launch_bounds__(128) k_adj_macro_sweepT(Dev<double> c, const int* cells, int n,
                                                          const double* dinv, const double* b, double* y) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int j = cells[t];
    const double* Wj = c.W + 6 * (size_t)j;
    double acc[6];
    for (int q = 0; q < 6; ++q) acc[q] = b[6 * (size_t)j + q];
    for (int m = c.slot_off[j]; m < c.slot_off[j + 1]; ++m) {
        const int i = c.slot_nbr[m];
        if (i < 0) continue;
        const int f = c.slot_face[m];
        // the normal out of j is sg n_f; out of i it is -sg n_f
        const double sg = c.slot_left[m] ? -1.0 : 1.0;
        const double cij = 0.5 * c.fa[f] / c.vol[i];
        double yi[6], jt[6];
        for (int q = 0; q < 6; ++q) yi[q] = y[6 * (size_t)i + q];
        euler_jt(Wj, sg * c.fn[f], sg * c.fn[c.F + f], sg * c.fn[2 * c.F + f], yi, jt);
        for (int q = 0; q < 6; ++q) acc[q] -= cij * (jt[q] - c.rf[f] * yi[q]);
    }
    const double d0 = dinv[2 * (size_t)j], d1 = dinv[2 * (size_t)j + 1];
    for (int q = 0; q < 5; ++q) y[6 * (size_t)j + q] = acc[q] * d0;
    y[6 * (size_t)j + 5] = acc[5] * d1;
}

}  // namespace rk
