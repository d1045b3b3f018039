/*
 * CPU oracle for the conservative implicit Rykov scheme (plain C, FP64).
 *
 * TEST INFRASTRUCTURE ONLY: a slow, direct restatement of the paper's Sec. 2-3
 * used to check the CUDA library; it shares no code with it.  Each function says
 * which equation or step it follows.  Where the paper leaves a choice open, the
 * reading taken is stated at the point of use (the same readings bind the CUDA
 * path).  Loops over independent cells/faces may run on OpenMP threads; every sum
 * over velocities or faces is sequential in a fixed order, so results do not depend
 * on the thread count.  Build with -ffp-contract=off so that products are rounded
 * as written (the upwind decisions u.n > 0 must be bit-reproducible).
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAX_BC 64
#define PI 3.14159265358979323846

struct orc_ctx {
    orc_params p;
    int64_t N, F, K;
    /* mesh (copies) */
    int64_t* fc;            /* [F][2] */
    double *fn, *fa, *fx;   /* [F][3], [F], [F][3] */
    double *cx, *cv;        /* [N][3], [N] */
    int32_t* col;
    int32_t ncol;
    /* DVS */
    double *u, *w;          /* [K][3], [K] */
    /* boundary conditions */
    int32_t bc_kind[ORC_MAX_BC];
    double bc_rho[ORC_MAX_BC], bc_U[ORC_MAX_BC][3], bc_T[ORC_MAX_BC];
    /* derived geometry */
    int64_t *cf_off, *cf_face;     /* cell -> faces, increasing face index */
    int64_t *col_off, *col_cell;   /* cells grouped by colour, increasing index */
    double *dt, *dtimp, *eps2;     /* [N] */
    double* Minv;                  /* [N][9] inverse LSQ normal matrix */
    double* s;                     /* [F] local physical step s_ij */
    /* state */
    double *phi, *W, *q;
    /* work */
    double *grad, *face0, *face, *fstate, *mface, *microF, *macroF, *Wt, *dW, *taut;
    double *res, *dphi, *rf;
    double* lstore;                /* [2][N][K] limiter values kept for freezing */
    int prepared;
    int64_t iter;       /* iterations since the last set_state */
};

/* ------------------------------------------------------------------------------ */
/* small helpers                                                                  */
/* ------------------------------------------------------------------------------ */
static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

#define PHI(buf, fd, i, k) (buf)[((size_t)(fd) * (size_t)c->N + (size_t)(i)) * (size_t)c->K + (size_t)(k)]
#define FACEV(buf, fd, f, k) (buf)[((size_t)(fd) * (size_t)c->F + (size_t)(f)) * (size_t)c->K + (size_t)(k)]
#define LSTORE(fd, i, k) c->lstore[((size_t)(fd) * (size_t)c->N + (size_t)(i)) * (size_t)c->K + (size_t)(k)]
#define GRAD(fd, d, i, k) c->grad[(((size_t)(fd) * 3 + (size_t)(d)) * (size_t)c->N + (size_t)(i)) * (size_t)c->K + (size_t)(k)]

/* Viscosity of the translational temperature: the power law of Eq. T_solve_mu, or
 * Sutherland's formula, Eq. T_solve_mu_Sut (chosen by viscosity_law). */
static double viscosity(const orc_params* P, double Ttr) {
    if (P->viscosity_law == 1)
        return P->mu_ref * pow(Ttr / P->T_ref, 1.5) * (P->T_ref + P->sutherland_c) / (Ttr + P->sutherland_c);
    return P->mu_ref * pow(Ttr / P->T_ref, P->omega_vis);
}

/* Relaxation time tau = mu(T_tr) / p_tr (Sec. 2.1, text after Eq. frot). */
static double relax_time(const orc_params* P, double rho, double Ttr) {
    return viscosity(P, Ttr) / (rho * P->R * Ttr);
}

/* Primitive variables from W = (rho, rho U, rho E, rho E_rot), Eqs. f_solve_rho -
 * f_solve_EnergyRot with K_tr = 3, K_rot = 2:
 *   rho E     = 1/2 rho |U|^2 + 5/2 rho R T
 *   rho E_rot = rho R T_rot
 *   rho E_tr  = 1/2 rho |U|^2 + 3/2 rho R T_tr                                 */
static void prim_from_W(const orc_params* P, const double* W, double* rho, double U[3],
                        double* T, double* Ttr, double* Trot) {
    double r = W[0];
    U[0] = W[1] / r; U[1] = W[2] / r; U[2] = W[3] / r;
    double ke = 0.5 * r * dot3(U, U);
    *rho = r;
    *T = (W[4] - ke) / (2.5 * r * P->R);
    *Trot = W[5] / (r * P->R);
    *Ttr = (W[4] - ke - W[5]) / (1.5 * r * P->R);
}

/* Maxwellian g^eq(u; rho, U, T), Eq. eqdf_Maxwellian. */
static double maxwellian(const orc_params* P, double rho, const double* U, double T, const double* u) {
    double RT = P->R * T;
    double c[3] = {u[0] - U[0], u[1] - U[1], u[2] - U[2]};
    return rho * pow(2.0 * PI * RT, -1.5) * exp(-dot3(c, c) / (2.0 * RT));
}

/* Rykov reduced equilibria at one velocity, Eqs. eqdf_G* - eqdf_Rrot:
 *   G^tr  = g^eq(T_tr) [1 + c.q_tr/(15 R T_tr p_tr) (|c|^2/(R T_tr) - 5)]
 *   G^rot = g^eq(T)    [1 + w0 c.q_tr/(15 R T p) (|c|^2/(R T) - 5)]
 *   R^tr  = R T_rot [G^tr + (1-delta) c.q_rot/(R T_tr p_rot) g^eq(T_tr)]
 *   R^rot = R T     [G^rot + w1 (1-delta) c.q_rot/(R T p) g^eq(T)]
 *   G* = (1 - 1/Z) G^tr + G^rot / Z,  R* likewise.
 * p = rho R T, p_tr = rho R T_tr, p_rot = rho R T_rot.  (The paper's f^rot writes
 * "p_2"; the reduced form uses p, which is the reading taken.) */
static void rykov_eq_point(const orc_params* P, const orc_state* s, const double* u,
                           double* G, double* H, double* parts) {
    const double R = P->R;
    double c[3] = {u[0] - s->U[0], u[1] - s->U[1], u[2] - s->U[2]};
    double c2 = dot3(c, c);
    double RTtr = R * s->Ttr, RT = R * s->T, RTrot = R * s->Trot;
    double ptr = s->rho * RTtr, p = s->rho * RT, prot = s->rho * RTrot;
    double geq_tr = s->rho * pow(2.0 * PI * RTtr, -1.5) * exp(-c2 / (2.0 * RTtr));
    double geq = s->rho * pow(2.0 * PI * RT, -1.5) * exp(-c2 / (2.0 * RT));
    double cqtr = dot3(c, s->qtr), cqrot = dot3(c, s->qrot);
    double Gtr = geq_tr * (1.0 + cqtr / (15.0 * RTtr * ptr) * (c2 / RTtr - 5.0));
    double Grot = geq * (1.0 + P->omega0 * cqtr / (15.0 * RT * p) * (c2 / RT - 5.0));
    double Htr = RTrot * (Gtr + (1.0 - P->delta) * cqrot / (RTtr * prot) * geq_tr);
    double Hrot = RT * (Grot + P->omega1 * (1.0 - P->delta) * cqrot / (RT * p) * geq);
    double iz = 1.0 / P->Z_rot;
    *G = (1.0 - iz) * Gtr + iz * Grot;
    *H = (1.0 - iz) * Htr + iz * Hrot;
    if (parts) { parts[0] = Gtr; parts[1] = Grot; parts[2] = Htr; parts[3] = Hrot; }
}

void orc_equilibrium(const orc_params* p, const orc_state* s, int64_t K, const double* u,
                     double* G, double* H) {
    for (int64_t k = 0; k < K; ++k) rykov_eq_point(p, s, u + 3 * k, G + k, H + k, NULL);
}

void orc_equilibrium_parts(const orc_params* p, const orc_state* s, int64_t K, const double* u,
                           double* Gtr, double* Grot, double* Htr, double* Hrot) {
    double G, H, parts[4];
    for (int64_t k = 0; k < K; ++k) {
        rykov_eq_point(p, s, u + 3 * k, &G, &H, parts);
        Gtr[k] = parts[0]; Grot[k] = parts[1]; Htr[k] = parts[2]; Hrot[k] = parts[3];
    }
}

/* Equilibrium state of a cell from W (predicted or current) and its heat flux. */
static void state_from_W(const orc_params* P, const double* W, const double* q, orc_state* s) {
    prim_from_W(P, W, &s->rho, s->U, &s->T, &s->Ttr, &s->Trot);
    for (int d = 0; d < 3; ++d) { s->qtr[d] = q[d]; s->qrot[d] = q[3 + d]; }
}

/* Venkatakrishnan's smooth limiter function (Sec. 3.3, text after Eq.
 * flux_solve_phi_phi; Venkatakrishnan 1995):
 *   psi = (d1^2 + eps2 + 2 d1 d2) / (d1^2 + 2 d2^2 + d1 d2 + eps2),  psi = 1 if d2 = 0,
 * with d1 = Delta_max (d2 > 0) or Delta_min (d2 < 0). */
double orc_venkat(double d1, double d2, double eps2) {
    if (d2 == 0.0) return 1.0;
    return (d1 * d1 + eps2 + 2.0 * d1 * d2) / (d1 * d1 + 2.0 * d2 * d2 + d1 * d2 + eps2);
}

/* Euler flux G_ij(W) along n, Eq. implicit_mac_equ_euler_flux, with
 * p = rho R T = (2/5)(rho E - 1/2 rho |U|^2) (5 degrees of freedom). */
void orc_euler_flux(const orc_params* P, const double* W, const double* n, double* G) {
    (void)P;
    double rho = W[0];
    double U[3] = {W[1] / rho, W[2] / rho, W[3] / rho};
    double p = 0.4 * (W[4] - 0.5 * rho * dot3(U, U));
    double Un = dot3(U, n);
    G[0] = rho * Un;
    for (int d = 0; d < 3; ++d) G[1 + d] = W[1 + d] * Un + p * n[d];
    G[4] = (W[4] + p) * Un;
    G[5] = W[5] * Un;
}

/* Spectral radius r_ij = |U.n| + a + 2 mu/(rho dl), Eq.
 * implicit_mac_equ_spectral_radius, evaluated at the face state Wm (reading: the
 * arithmetic mean of the two cells' W^n), a = sqrt(gamma R T), gamma = 7/5,
 * mu = mu(T_tr) of that state. */
double orc_spectral_radius(const orc_params* P, const double* Wm, const double* n, double dl) {
    double rho, U[3], T, Ttr, Trot;
    prim_from_W(P, Wm, &rho, U, &T, &Ttr, &Trot);
    double a = sqrt(1.4 * P->R * T);
    return fabs(dot3(U, n)) + a + 2.0 * viscosity(P, Ttr) / (rho * dl);
}

/* ------------------------------------------------------------------------------ */
/* Step 2 (b)-(d) for one interior face                                           */
/* ------------------------------------------------------------------------------ */
/* Face state layout (16 doubles): rho, U[3], T, T_tr, T_rot, tau, q_tr[3],
 * q_rot[3], s, rho_w (wall faces only). */
static void interface_state(const orc_params* P, int64_t K, const double* u, const double* w,
                            const double* g0, const double* h0, double s, double* st) {
    const double R = P->R, Z = P->Z_rot;
    /* Eqs. halftime_solve_rho, _U, _E: conserved moments of the free-transport
     * distribution phi(x_ij - u s) (collisions conserve them). */
    double rho = 0.0, m[3] = {0.0, 0.0, 0.0}, E = 0.0, Er0 = 0.0;
    for (int64_t k = 0; k < K; ++k) {
        const double* uk = u + 3 * k;
        rho += w[k] * g0[k];
        for (int d = 0; d < 3; ++d) m[d] += w[k] * uk[d] * g0[k];
        E += w[k] * (0.5 * dot3(uk, uk) * g0[k] + h0[k]);
        Er0 += w[k] * h0[k];
    }
    double U[3] = {m[0] / rho, m[1] / rho, m[2] / rho};
    double ke = 0.5 * rho * dot3(U, U);
    double T = (E - ke) / (2.5 * rho * R);
    /* tau(x_ij, t_n + s): the paper evaluates it at the interface after collision,
     * which needs E_rot, which in turn needs tau.  Reading: one explicit evaluation
     * with the translational temperature of the free-transport moments. */
    double Ttr0 = (E - ke - Er0) / (1.5 * rho * R);
    double tau = relax_time(P, rho, Ttr0);
    /* Eq. halftime_solve_Erot */
    double Erot = (Z * tau * Er0 + s * rho * R * T) / (Z * tau + s);
    double Trot = Erot / (rho * R);
    double Ttr = (E - ke - Erot) / (1.5 * rho * R);
    /* Eqs. halftime_solve_qtra / halftime_solve_qrot with c = u - U */
    double Qtr[3] = {0.0, 0.0, 0.0}, Qrot[3] = {0.0, 0.0, 0.0};
    for (int64_t k = 0; k < K; ++k) {
        const double* uk = u + 3 * k;
        double c[3] = {uk[0] - U[0], uk[1] - U[1], uk[2] - U[2]};
        double c2 = dot3(c, c);
        for (int d = 0; d < 3; ++d) {
            Qtr[d] += w[k] * c[d] * c2 * g0[k];
            Qrot[d] += w[k] * c[d] * h0[k];
        }
    }
    double dtr = tau + s - s / 3.0 * (1.0 - 1.0 / Z + P->omega0 / Z);
    double drot = tau + s - s * (1.0 - P->delta) * (1.0 - 1.0 / Z + P->omega1 / Z);
    st[0] = rho; st[1] = U[0]; st[2] = U[1]; st[3] = U[2];
    st[4] = T; st[5] = Ttr; st[6] = Trot; st[7] = tau;
    for (int d = 0; d < 3; ++d) {
        st[8 + d] = tau * 0.5 * Qtr[d] / dtr;
        st[11 + d] = tau * Qrot[d] / drot;
    }
    st[14] = s; st[15] = 0.0;
}

static void st_to_state(const double* st, orc_state* s) {
    s->rho = st[0]; s->U[0] = st[1]; s->U[1] = st[2]; s->U[2] = st[3];
    s->T = st[4]; s->Ttr = st[5]; s->Trot = st[6];
    for (int d = 0; d < 3; ++d) { s->qtr[d] = st[8 + d]; s->qrot[d] = st[11 + d]; }
}

/* Eq. flux_solve_phi: phi_ij = tau/(tau+s) phi(x_ij - u s) + s/(tau+s) phi*(x_ij). */
static void interface_blend(const orc_params* P, int64_t K, const double* u, const double* st,
                            const double* g0, const double* h0, double* gf, double* hf) {
    orc_state s;
    st_to_state(st, &s);
    double tau = st[7], sl = st[14];
    for (int64_t k = 0; k < K; ++k) {
        double G, H;
        rykov_eq_point(P, &s, u + 3 * k, &G, &H, NULL);
        gf[k] = (tau * g0[k] + sl * G) / (tau + sl);
        hf[k] = (tau * h0[k] + sl * H) / (tau + sl);
    }
}

void orc_interface(const orc_params* p, int64_t K, const double* u, const double* w,
                   const double* g0, const double* h0, double s, double* state16,
                   double* gf, double* hf) {
    interface_state(p, K, u, w, g0, h0, s, state16);
    interface_blend(p, K, u, state16, g0, h0, gf, hf);
}

/* ------------------------------------------------------------------------------ */
/* context management                                                             */
/* ------------------------------------------------------------------------------ */
static void* xcalloc(size_t n, size_t sz) { return n ? calloc(n, sz) : calloc(1, sz); }

orc_ctx* orc_create(const orc_params* p) {
    orc_ctx* c = (orc_ctx*)calloc(1, sizeof(orc_ctx));
    if (!c) return NULL;
    c->p = *p;
    for (int b = 0; b < ORC_MAX_BC; ++b) c->bc_kind[b] = -1;
    return c;
}

static void free_work(orc_ctx* c) {
    double** bufs[] = {&c->dt, &c->dtimp, &c->eps2, &c->Minv, &c->s, &c->phi, &c->W, &c->q,
                       &c->grad, &c->face0, &c->face, &c->fstate, &c->mface, &c->microF,
                       &c->macroF, &c->Wt, &c->dW, &c->taut, &c->res, &c->dphi, &c->rf, &c->lstore};
    for (size_t b = 0; b < sizeof(bufs) / sizeof(bufs[0]); ++b) { free(*bufs[b]); *bufs[b] = NULL; }
    free(c->cf_off); free(c->cf_face); free(c->col_off); free(c->col_cell);
    c->cf_off = c->cf_face = c->col_off = c->col_cell = NULL;
    c->prepared = 0;
}

void orc_destroy(orc_ctx* c) {
    if (!c) return;
    free_work(c);
    free(c->fc); free(c->fn); free(c->fa); free(c->fx); free(c->cx); free(c->cv); free(c->col);
    free(c->u); free(c->w);
    free(c);
}

int orc_set_params(orc_ctx* c, const orc_params* p) {
    c->p = *p;
    if (c->prepared) return orc_prepare(c);
    return 0;
}

int orc_set_mesh(orc_ctx* c, int64_t n_cell, int64_t n_face, const int64_t* face_cell,
                 const double* face_normal, const double* face_area, const double* face_center,
                 const double* cell_center, const double* cell_volume, const int32_t* cell_colour) {
    if (n_cell <= 0 || n_face <= 0 || !cell_colour) return -1;
    free_work(c);
    free(c->fc); free(c->fn); free(c->fa); free(c->fx); free(c->cx); free(c->cv); free(c->col);
    c->N = n_cell; c->F = n_face;
    c->fc = (int64_t*)malloc(sizeof(int64_t) * 2 * n_face);
    c->fn = (double*)malloc(sizeof(double) * 3 * n_face);
    c->fa = (double*)malloc(sizeof(double) * n_face);
    c->fx = (double*)malloc(sizeof(double) * 3 * n_face);
    c->cx = (double*)malloc(sizeof(double) * 3 * n_cell);
    c->cv = (double*)malloc(sizeof(double) * n_cell);
    c->col = (int32_t*)malloc(sizeof(int32_t) * n_cell);
    memcpy(c->fc, face_cell, sizeof(int64_t) * 2 * n_face);
    memcpy(c->fn, face_normal, sizeof(double) * 3 * n_face);
    memcpy(c->fa, face_area, sizeof(double) * n_face);
    memcpy(c->fx, face_center, sizeof(double) * 3 * n_face);
    memcpy(c->cx, cell_center, sizeof(double) * 3 * n_cell);
    memcpy(c->cv, cell_volume, sizeof(double) * n_cell);
    memcpy(c->col, cell_colour, sizeof(int32_t) * n_cell);
    return 0;
}

int orc_set_dvs(orc_ctx* c, int64_t K, const double* u, const double* w) {
    if (K <= 0) return -1;
    free_work(c);
    free(c->u); free(c->w);
    c->K = K;
    c->u = (double*)malloc(sizeof(double) * 3 * K);
    c->w = (double*)malloc(sizeof(double) * K);
    memcpy(c->u, u, sizeof(double) * 3 * K);
    memcpy(c->w, w, sizeof(double) * K);
    return 0;
}

int orc_set_bc(orc_ctx* c, int32_t bc_id, int32_t kind, double rho, const double* U, double T) {
    if (bc_id < 0 || bc_id >= ORC_MAX_BC) return -1;
    c->bc_kind[bc_id] = kind;
    c->bc_rho[bc_id] = rho;
    for (int d = 0; d < 3; ++d) c->bc_U[bc_id][d] = U[d];
    c->bc_T[bc_id] = T;
    return 0;
}

/* Implicit step factor of iteration n.  The paper only says the implicit step is
 * not limited by the CFL condition; reading: a geometric ramp from cfl_imp0 to
 * cfl_imp (a common start-up device for implicit steady solvers). */
static double implicit_cfl(const orc_params* P, int64_t n) {
    if (P->cfl_imp0 <= 0.0 || P->cfl_ramp <= 1.0) return P->cfl_imp;
    double c = P->cfl_imp0 * pow(P->cfl_ramp, (double)n);
    return c < P->cfl_imp ? c : P->cfl_imp;
}

static void set_implicit_step(orc_ctx* c) {
    double cfl = implicit_cfl(&c->p, c->iter);
    for (int64_t i = 0; i < c->N; ++i) c->dtimp[i] = cfl * c->dt[i];
}

/* Set-up (Step 1 ingredients): cell->face lists, colour groups, the CFL step
 * Delta t_i, the local physical step s_ij = min(Delta t_i, Delta t_j) (Sec. 3.3,
 * text after Eq. flux_dis_equ), the implicit step, and the least-squares normal
 * matrices.  The paper gives neither the CFL formula nor the implicit step; the
 * readings are
 *   Delta t_i = cfl_s V_i / max_k sum_f A_f max(u_k . n_f,out, 0)
 *   (the positivity bound of explicit upwind transport), s = Delta t_i at
 *   boundary faces, and an implicit step cfl_imp * Delta t_i. */
int orc_prepare(orc_ctx* c) {
    const int64_t N = c->N, F = c->F, K = c->K;
    if (!c->fc || !c->u) return -1;
    free_work(c);
    /* CSR */
    c->cf_off = (int64_t*)calloc((size_t)N + 1, sizeof(int64_t));
    for (int64_t f = 0; f < F; ++f) {
        int64_t a = c->fc[2 * f], b = c->fc[2 * f + 1];
        if (a < 0 || a >= N || b >= N) return -1;
        c->cf_off[a + 1]++;
        if (b >= 0) c->cf_off[b + 1]++;
        else if (c->bc_kind[-1 - b] < 0) return -2;   /* bc id without a condition */
    }
    for (int64_t i = 0; i < N; ++i) c->cf_off[i + 1] += c->cf_off[i];
    c->cf_face = (int64_t*)malloc(sizeof(int64_t) * (size_t)c->cf_off[N]);
    int64_t* fill = (int64_t*)calloc((size_t)N, sizeof(int64_t));
    for (int64_t f = 0; f < F; ++f) {
        int64_t a = c->fc[2 * f], b = c->fc[2 * f + 1];
        c->cf_face[c->cf_off[a] + fill[a]++] = f;
        if (b >= 0) c->cf_face[c->cf_off[b] + fill[b]++] = f;
    }
    free(fill);
    /* colour groups */
    int32_t nc = 0;
    for (int64_t i = 0; i < N; ++i) {
        if (c->col[i] < 0) return -3;
        if (c->col[i] + 1 > nc) nc = c->col[i] + 1;
    }
    for (int64_t f = 0; f < F; ++f) {
        int64_t a = c->fc[2 * f], b = c->fc[2 * f + 1];
        if (b >= 0 && c->col[a] == c->col[b]) return -3;     /* not a proper colouring */
    }
    c->ncol = nc;
    c->col_off = (int64_t*)calloc((size_t)nc + 1, sizeof(int64_t));
    for (int64_t i = 0; i < N; ++i) c->col_off[c->col[i] + 1]++;
    for (int32_t k = 0; k < nc; ++k) c->col_off[k + 1] += c->col_off[k];
    c->col_cell = (int64_t*)malloc(sizeof(int64_t) * (size_t)N);
    int64_t* cfill = (int64_t*)calloc((size_t)nc, sizeof(int64_t));
    for (int64_t i = 0; i < N; ++i) c->col_cell[c->col_off[c->col[i]] + cfill[c->col[i]]++] = i;
    free(cfill);
    /* allocations */
    size_t NK = (size_t)N * (size_t)K, FK = (size_t)F * (size_t)K;
    c->dt = (double*)xcalloc((size_t)N, sizeof(double));
    c->dtimp = (double*)xcalloc((size_t)N, sizeof(double));
    c->eps2 = (double*)xcalloc((size_t)N, sizeof(double));
    c->Minv = (double*)xcalloc((size_t)N * 9, sizeof(double));
    c->s = (double*)xcalloc((size_t)F, sizeof(double));
    c->phi = (double*)xcalloc(2 * NK, sizeof(double));
    c->W = (double*)xcalloc((size_t)N * 6, sizeof(double));
    c->q = (double*)xcalloc((size_t)N * 6, sizeof(double));
    c->grad = (double*)xcalloc(6 * NK, sizeof(double));
    c->face0 = (double*)xcalloc(2 * FK, sizeof(double));
    c->face = (double*)xcalloc(2 * FK, sizeof(double));
    c->fstate = (double*)xcalloc((size_t)F * 16, sizeof(double));
    c->mface = (double*)xcalloc((size_t)F * 6, sizeof(double));
    c->microF = (double*)xcalloc(2 * NK, sizeof(double));
    c->macroF = (double*)xcalloc((size_t)N * 6, sizeof(double));
    c->Wt = (double*)xcalloc((size_t)N * 6, sizeof(double));
    c->dW = (double*)xcalloc((size_t)N * 6, sizeof(double));
    c->taut = (double*)xcalloc((size_t)N, sizeof(double));
    c->res = (double*)xcalloc(2 * NK, sizeof(double));
    c->dphi = (double*)xcalloc(2 * NK, sizeof(double));
    c->rf = (double*)xcalloc((size_t)F, sizeof(double));
    c->lstore = (double*)xcalloc(2 * NK, sizeof(double));
    if (!c->dphi || !c->res || !c->grad || !c->face || !c->face0) return -4;

    /* CFL step per cell */
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        double vmax = 0.0;
        for (int64_t k = 0; k < K; ++k) {
            double sum = 0.0;
            for (int64_t m = c->cf_off[i]; m < c->cf_off[i + 1]; ++m) {
                int64_t f = c->cf_face[m];
                double un = dot3(c->u + 3 * k, c->fn + 3 * f);
                if (c->fc[2 * f] != i) un = -un;      /* outward from i */
                if (un > 0.0) sum += c->fa[f] * un;
            }
            if (sum > vmax) vmax = sum;
        }
        c->dt[i] = c->p.cfl_s * c->cv[i] / vmax;
        c->dtimp[i] = implicit_cfl(&c->p, 0) * c->dt[i];
        double h = cbrt(c->cv[i]) * c->p.lim_k;
        c->eps2[i] = h * h * h;
    }
    for (int64_t f = 0; f < F; ++f) {
        int64_t a = c->fc[2 * f], b = c->fc[2 * f + 1];
        c->s[f] = (b >= 0) ? fmin(c->dt[a], c->dt[b]) : c->dt[a];
    }
    /* Least-squares normal matrix M_i = sum_m d_m d_m^T over face neighbours
     * (d = x_j - x_i) and, reading for boundaries, the boundary face centroids
     * (d = x_f - x_i) as pseudo-neighbours holding the cell's own value. */
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        double M[9] = {0};
        for (int64_t m = c->cf_off[i]; m < c->cf_off[i + 1]; ++m) {
            int64_t f = c->cf_face[m];
            int64_t a = c->fc[2 * f], b = c->fc[2 * f + 1];
            int64_t j = (a == i) ? b : a;
            const double* xo = (j >= 0) ? c->cx + 3 * j : c->fx + 3 * f;
            double d[3] = {xo[0] - c->cx[3 * i], xo[1] - c->cx[3 * i + 1], xo[2] - c->cx[3 * i + 2]};
            for (int r = 0; r < 3; ++r)
                for (int s2 = 0; s2 < 3; ++s2) M[3 * r + s2] += d[r] * d[s2];
        }
        /* inverse by the adjugate */
        double A = M[4] * M[8] - M[5] * M[7], B = M[5] * M[6] - M[3] * M[8], C = M[3] * M[7] - M[4] * M[6];
        double det = M[0] * A + M[1] * B + M[2] * C;
        double* Mi = c->Minv + 9 * i;
        Mi[0] = A / det; Mi[1] = (M[2] * M[7] - M[1] * M[8]) / det; Mi[2] = (M[1] * M[5] - M[2] * M[4]) / det;
        Mi[3] = B / det; Mi[4] = (M[0] * M[8] - M[2] * M[6]) / det; Mi[5] = (M[2] * M[3] - M[0] * M[5]) / det;
        Mi[6] = C / det; Mi[7] = (M[1] * M[6] - M[0] * M[7]) / det; Mi[8] = (M[0] * M[4] - M[1] * M[3]) / det;
    }
    c->prepared = 1;
    return 0;
}

/* ------------------------------------------------------------------------------ */
/* state                                                                          */
/* ------------------------------------------------------------------------------ */
int orc_set_state_prim(orc_ctx* c, const double* prim, const double* q) {
    if (!c->prepared) return -1;
    c->iter = 0;
    const orc_params* P = &c->p;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < c->N; ++i) {
        const double* pr = prim + 6 * i;
        double rho = pr[0], U[3] = {pr[1], pr[2], pr[3]}, Ttr = pr[4], Trot = pr[5];
        double* W = c->W + 6 * i;
        W[0] = rho;
        for (int d = 0; d < 3; ++d) W[1 + d] = rho * U[d];
        W[4] = 0.5 * rho * dot3(U, U) + 1.5 * rho * P->R * Ttr + rho * P->R * Trot;
        W[5] = rho * P->R * Trot;
        for (int d = 0; d < 6; ++d) c->q[6 * i + d] = q ? q[6 * i + d] : 0.0;
        orc_state s;
        state_from_W(P, W, c->q + 6 * i, &s);
        for (int64_t k = 0; k < c->K; ++k)
            rykov_eq_point(P, &s, c->u + 3 * k, &PHI(c->phi, 0, i, k), &PHI(c->phi, 1, i, k), NULL);
    }
    return 0;
}

int orc_set_state(orc_ctx* c, const double* W, const double* q, const double* phi) {
    if (!c->prepared) return -1;
    c->iter = 0;
    memcpy(c->W, W, sizeof(double) * 6 * (size_t)c->N);
    if (q) memcpy(c->q, q, sizeof(double) * 6 * (size_t)c->N);
    else memset(c->q, 0, sizeof(double) * 6 * (size_t)c->N);
    if (phi) memcpy(c->phi, phi, sizeof(double) * 2 * (size_t)c->N * (size_t)c->K);
    return 0;
}

/* ------------------------------------------------------------------------------ */
/* Step 2 (a) ingredients: least-squares gradient and Venkatakrishnan limiter     */
/* ------------------------------------------------------------------------------ */
void orc_step_gradient(orc_ctx* c) {
    const int64_t N = c->N, K = c->K;
    /* reading: an optional first-order start (gradient zero) before the limited
     * second-order reconstruction */
    const int lim = (c->iter < c->p.first_order_iters) ? 2 : c->p.limiter;
    /* reading (no counterpart in the paper): the limiter values may be frozen once
     * the iteration is close to its fixed point, because the min/max selections of
     * the limiter otherwise keep switching and stall the residual; iteration
     * limiter_freeze - 1 stores them, later iterations reuse them */
    const int freeze = (lim == 1 && c->p.limiter_freeze > 0);
    const int frozen = freeze && c->iter >= c->p.limiter_freeze;
    const int store = freeze && c->iter == c->p.limiter_freeze - 1;
    set_implicit_step(c);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        const double* xi = c->cx + 3 * i;
        const double* Mi = c->Minv + 9 * i;
        for (int fd = 0; fd < 2; ++fd) {
            for (int64_t k = 0; k < K; ++k) {
                double phii = PHI(c->phi, fd, i, k);
                double b[3] = {0.0, 0.0, 0.0}, dmax = 0.0, dmin = 0.0;
                for (int64_t m = c->cf_off[i]; m < c->cf_off[i + 1]; ++m) {
                    int64_t f = c->cf_face[m];
                    int64_t a = c->fc[2 * f], bb = c->fc[2 * f + 1];
                    int64_t j = (a == i) ? bb : a;
                    if (j < 0) continue;        /* boundary pseudo-neighbour: zero difference */
                    double dphi = PHI(c->phi, fd, j, k) - phii;
                    const double* xj = c->cx + 3 * j;
                    double d[3] = {xj[0] - xi[0], xj[1] - xi[1], xj[2] - xi[2]};
                    for (int r = 0; r < 3; ++r) b[r] += d[r] * dphi;
                    if (dphi > dmax) dmax = dphi;
                    if (dphi < dmin) dmin = dphi;
                }
                double g[3];
                for (int r = 0; r < 3; ++r) g[r] = Mi[3 * r] * b[0] + Mi[3 * r + 1] * b[1] + Mi[3 * r + 2] * b[2];
                double L = 1.0;
                if (lim == 2) {
                    L = 0.0;
                } else if (frozen) {
                    L = LSTORE(fd, i, k);
                } else if (lim == 1) {
                    /* limiter at each face centroid, minimum over faces; readings: capped
                     * at 1 so that it only ever reduces the gradient, and the threshold
                     * eps^2 = (K V^{1/3})^3 taken relative to the cell value,
                     * eps^2 phi_i^2, because the distribution spans many orders of
                     * magnitude (an absolute threshold switches the limiter off in
                     * near-vacuum cells) */
                    for (int64_t m = c->cf_off[i]; m < c->cf_off[i + 1]; ++m) {
                        int64_t f = c->cf_face[m];
                        const double* xf = c->fx + 3 * f;
                        double r[3] = {xf[0] - xi[0], xf[1] - xi[1], xf[2] - xi[2]};
                        double d2 = dot3(g, r);
                        double psi = orc_venkat(d2 > 0.0 ? dmax : dmin, d2, c->eps2[i] * phii * phii);
                        if (psi < L) L = psi;
                    }
                    if (store) LSTORE(fd, i, k) = L;
                }
                for (int r = 0; r < 3; ++r) GRAD(fd, r, i, k) = L * g[r];
            }
        }
    }
}

/* ------------------------------------------------------------------------------ */
/* Step 2 (a)-(d): face distributions                                             */
/* ------------------------------------------------------------------------------ */
/* Eq. flux_solve_phi_phi: phi(x_ij - u s) = phi(x_c) + (x_ij - u s - x_c) . L grad phi(x_c)
 * with x_c = x_i if u.n_ij > 0, else x_j. */
static double reconstruct(const orc_ctx* c, int fd, int64_t cell, int64_t k, const double* xf,
                          double s) {
    const double* uk = c->u + 3 * k;
    const double* xc = c->cx + 3 * cell;
    double r[3] = {xf[0] - uk[0] * s - xc[0], xf[1] - uk[1] * s - xc[1], xf[2] - uk[2] * s - xc[2]};
    double g[3] = {GRAD(fd, 0, cell, k), GRAD(fd, 1, cell, k), GRAD(fd, 2, cell, k)};
    return PHI(c->phi, fd, cell, k) + dot3(r, g);
}

void orc_step_faces(orc_ctx* c) {
    const int64_t F = c->F, K = c->K;
    const orc_params* P = &c->p;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t f = 0; f < F; ++f) {
        int64_t i = c->fc[2 * f], j = c->fc[2 * f + 1];
        const double* n = c->fn + 3 * f;
        const double* xf = c->fx + 3 * f;
        double s = c->s[f];
        double* g0 = &FACEV(c->face0, 0, f, 0);
        double* h0 = &FACEV(c->face0, 1, f, 0);
        double* gf = &FACEV(c->face, 0, f, 0);
        double* hf = &FACEV(c->face, 1, f, 0);
        double* st = c->fstate + 16 * f;
        if (j >= 0) {
            for (int64_t k = 0; k < K; ++k) {
                double un = dot3(c->u + 3 * k, n);
                int64_t up = (un > 0.0) ? i : j;
                g0[k] = reconstruct(c, 0, up, k, xf, s);
                h0[k] = reconstruct(c, 1, up, k, xf, s);
            }
            interface_state(P, K, c->u, c->w, g0, h0, s, st);
            interface_blend(P, K, c->u, st, g0, h0, gf, hf);
            continue;
        }
        /* Boundary faces (the paper names diffuse reflection with full accommodation
         * but gives no formula; reading): particles leaving the fluid carry the
         * reconstructed interior value; incoming particles follow the boundary
         * distribution.  Wall: rho_w g^eq(u; 1, U_w, T_w), h = R T_w g, with rho_w set
         * so that the discrete mass flux through the face vanishes.  Farfield:
         * freestream Maxwellian, h = R T_inf g.  No interface collision. */
        int32_t bc = (int32_t)(-1 - j);
        int kind = c->bc_kind[bc];
        double one = 1.0;
        double num = 0.0, den = 0.0;
        for (int64_t k = 0; k < K; ++k) {
            const double* uk = c->u + 3 * k;
            double un = dot3(uk, n);
            if (un > 0.0) {
                g0[k] = reconstruct(c, 0, i, k, xf, s);
                h0[k] = reconstruct(c, 1, i, k, xf, s);
                num += c->w[k] * un * g0[k];
            } else if (kind == ORC_WALL) {
                double M = maxwellian(P, one, c->bc_U[bc], c->bc_T[bc], uk);
                g0[k] = M;
                h0[k] = P->R * c->bc_T[bc] * M;
                den += c->w[k] * (-un) * M;
            } else {
                double M = maxwellian(P, c->bc_rho[bc], c->bc_U[bc], c->bc_T[bc], uk);
                g0[k] = M;
                h0[k] = P->R * c->bc_T[bc] * M;
            }
        }
        double rho_w = (kind == ORC_WALL) ? num / den : 0.0;
        for (int64_t k = 0; k < K; ++k) {
            double un = dot3(c->u + 3 * k, n);
            if (un <= 0.0 && kind == ORC_WALL) { gf[k] = rho_w * g0[k]; hf[k] = rho_w * h0[k]; }
            else { gf[k] = g0[k]; hf[k] = h0[k]; }
        }
        memset(st, 0, 16 * sizeof(double));
        st[14] = s;
        st[15] = rho_w;
    }
}

/* ------------------------------------------------------------------------------ */
/* Step 2 (e) and Step 3: micro flux F_{i,k} and macro flux F_i                   */
/* ------------------------------------------------------------------------------ */
void orc_step_fluxes(orc_ctx* c) {
    const int64_t N = c->N, F = c->F, K = c->K;
    /* per-face DVS quadrature of Eq. implicit_mac_equ_mac_flux (without A/V):
     * sum_k w_k (u_k . n) (g, u g, 1/2|u|^2 g + h, h) */
#pragma omp parallel for schedule(static)
    for (int64_t f = 0; f < F; ++f) {
        const double* n = c->fn + 3 * f;
        double M[6] = {0};
        for (int64_t k = 0; k < K; ++k) {
            const double* uk = c->u + 3 * k;
            double un = dot3(uk, n);
            double g = FACEV(c->face, 0, f, k), h = FACEV(c->face, 1, f, k);
            double wu = c->w[k] * un;
            M[0] += wu * g;
            M[1] += wu * uk[0] * g;
            M[2] += wu * uk[1] * g;
            M[3] += wu * uk[2] * g;
            M[4] += wu * (0.5 * dot3(uk, uk) * g + h);
            M[5] += wu * h;
        }
        for (int m = 0; m < 6; ++m) c->mface[6 * f + m] = M[m];
    }
    /* Eq. implicit_mic_flux: F_{i,k} = (1/V_i) sum_j A_ij (u_k . n_ij) phi_ij,k with
     * n_ij pointing out of cell i; macro flux F_i likewise from the face sums. */
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        double iv = 1.0 / c->cv[i];
        for (int fd = 0; fd < 2; ++fd) {
            for (int64_t k = 0; k < K; ++k) {
                double sum = 0.0;
                for (int64_t m = c->cf_off[i]; m < c->cf_off[i + 1]; ++m) {
                    int64_t f = c->cf_face[m];
                    double un = dot3(c->u + 3 * k, c->fn + 3 * f);
                    if (c->fc[2 * f] != i) un = -un;
                    sum += c->fa[f] * un * FACEV(c->face, fd, f, k);
                }
                PHI(c->microF, fd, i, k) = sum * iv;
            }
        }
        double Mi[6] = {0};
        for (int64_t m = c->cf_off[i]; m < c->cf_off[i + 1]; ++m) {
            int64_t f = c->cf_face[m];
            double sg = (c->fc[2 * f] == i) ? 1.0 : -1.0;
            for (int q2 = 0; q2 < 6; ++q2) Mi[q2] += sg * c->fa[f] * c->mface[6 * f + q2];
        }
        for (int q2 = 0; q2 < 6; ++q2) c->macroF[6 * i + q2] = Mi[q2] * iv;
    }
}

/* ------------------------------------------------------------------------------ */
/* Step 4: implicit macroscopic prediction, Eq. implicit_mac_equ_fin, PR-SGS     */
/* ------------------------------------------------------------------------------ */
static void macro_point_update(orc_ctx* c, int64_t i, int first_forward, int32_t colour) {
    const orc_params* P = &c->p;
    const double Z = P->Z_rot;
    double iv = 1.0 / c->cv[i];
    /* rotational source (Eq. implicit_mac_equ_source_term): reading for the tilde
     * quantities, which are unknown until the prediction is done: rho~ R T~ from the
     * current iterate of cell i just before this update, tau~ frozen at its W^n
     * value for the whole macro solve (c->taut holds it during the sweeps) */
    double Wc[6];
    for (int m = 0; m < 6; ++m) Wc[m] = c->W[6 * i + m] + c->dW[6 * i + m];
    double rho, U[3], T, Ttr, Trot;
    prim_from_W(P, Wc, &rho, U, &T, &Ttr, &Trot);
    double tau = c->taut[i];
    double D = 1.0 / c->dtimp[i];
    double off[6] = {0};
    for (int64_t m = c->cf_off[i]; m < c->cf_off[i + 1]; ++m) {
        int64_t f = c->cf_face[m];
        int64_t a = c->fc[2 * f], b = c->fc[2 * f + 1];
        int64_t j = (a == i) ? b : a;
        double A = c->fa[f] * iv;
        D += 0.5 * A * c->rf[f];
        if (j < 0) continue;                       /* ghost increment is zero */
        if (first_forward && c->col[j] > colour) continue;   /* not yet updated: zero */
        double n[3] = {c->fn[3 * f], c->fn[3 * f + 1], c->fn[3 * f + 2]};
        if (a != i) { n[0] = -n[0]; n[1] = -n[1]; n[2] = -n[2]; }
        const double* Wj = c->W + 6 * j;
        const double* dWj = c->dW + 6 * j;
        double Wn[6], G1[6], G0[6];
        for (int q2 = 0; q2 < 6; ++q2) Wn[q2] = Wj[q2] + dWj[q2];
        /* matrix-free product dG/dW dW~_j = G(W_j + dW~_j) - G(W_j) */
        orc_euler_flux(P, Wn, n, G1);
        orc_euler_flux(P, Wj, n, G0);
        for (int q2 = 0; q2 < 6; ++q2) off[q2] += 0.5 * A * ((G1[q2] - G0[q2]) - c->rf[f] * dWj[q2]);
    }
    double cand[6];
    for (int q2 = 0; q2 < 5; ++q2) cand[q2] = (-c->macroF[6 * i + q2] - off[q2]) / D;
    double src = (rho * P->R * T - c->W[6 * i + 5]) / (Z * tau);
    cand[5] = (src - c->macroF[6 * i + 5] - off[5]) / (D + 1.0 / (Z * tau));
    /* Reading (the paper gives no safeguard): a point update whose predicted state
     * is not physically admissible (rho, T_tr or T_rot not positive) is skipped and
     * the cell keeps its previous iterate, which is admissible. */
    double Wn[6];
    for (int q2 = 0; q2 < 6; ++q2) Wn[q2] = c->W[6 * i + q2] + cand[q2];
    double r2, U2[3], T2, Ttr2, Trot2;
    prim_from_W(P, Wn, &r2, U2, &T2, &Ttr2, &Trot2);
    if (!(r2 > 0.0 && Ttr2 > 0.0 && Trot2 > 0.0)) return;
    for (int q2 = 0; q2 < 6; ++q2) c->dW[6 * i + q2] = cand[q2];
}

void orc_step_macro(orc_ctx* c) {
    const int64_t N = c->N, F = c->F;
    const orc_params* P = &c->p;
    /* spectral radius per face from the arithmetic mean of W^n (boundary: W_i and
     * dl = 2 |x_f - x_i|) */
#pragma omp parallel for schedule(static)
    for (int64_t f = 0; f < F; ++f) {
        int64_t a = c->fc[2 * f], b = c->fc[2 * f + 1];
        double Wm[6], dl;
        if (b >= 0) {
            for (int m = 0; m < 6; ++m) Wm[m] = 0.5 * (c->W[6 * a + m] + c->W[6 * b + m]);
            double d[3] = {c->cx[3 * b] - c->cx[3 * a], c->cx[3 * b + 1] - c->cx[3 * a + 1],
                           c->cx[3 * b + 2] - c->cx[3 * a + 2]};
            dl = sqrt(dot3(d, d));
        } else {
            for (int m = 0; m < 6; ++m) Wm[m] = c->W[6 * a + m];
            double d[3] = {c->fx[3 * f] - c->cx[3 * a], c->fx[3 * f + 1] - c->cx[3 * a + 1],
                           c->fx[3 * f + 2] - c->cx[3 * a + 2]};
            dl = 2.0 * sqrt(dot3(d, d));
        }
        c->rf[f] = orc_spectral_radius(P, Wm, c->fn + 3 * f, dl);
    }
    memset(c->dW, 0, sizeof(double) * 6 * (size_t)N);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        double rho, U[3], T, Ttr, Trot;
        prim_from_W(P, c->W + 6 * i, &rho, U, &T, &Ttr, &Trot);
        c->taut[i] = relax_time(P, rho, Ttr);
    }
    /* n_macro_sgs x (forward colour sweep, backward colour sweep) */
    for (int32_t it = 0; it < P->n_macro_sgs; ++it) {
        for (int dir = 0; dir < 2; ++dir) {
            for (int32_t cc = 0; cc < c->ncol; ++cc) {
                int32_t colour = dir == 0 ? cc : c->ncol - 1 - cc;
                int first_forward = (it == 0 && dir == 0);
                int64_t lo = c->col_off[colour], hi = c->col_off[colour + 1];
#pragma omp parallel for schedule(static)
                for (int64_t t = lo; t < hi; ++t) macro_point_update(c, c->col_cell[t], first_forward, colour);
            }
        }
    }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        for (int m = 0; m < 6; ++m) c->Wt[6 * i + m] = c->W[6 * i + m] + c->dW[6 * i + m];
        double rho, U[3], T, Ttr, Trot;
        prim_from_W(P, c->Wt + 6 * i, &rho, U, &T, &Ttr, &Trot);
        c->taut[i] = relax_time(P, rho, Ttr);
    }
}

/* ------------------------------------------------------------------------------ */
/* Step 5: implicit microscopic equation, Eq. implicit_mic_final_equ, PR-SGS      */
/* ------------------------------------------------------------------------------ */
/* D_{i,k} = 1/dt + 1/tau~ + sum_j (A/V) u.n [1 + sign(u.n)] / 2 (all faces,
 * including boundary faces);  off-diagonal (A/V) u.n [1 - sign(u.n)] / 2 acting on
 * the neighbour's increment; boundary ghost increments are zero. */
static void micro_point_update(orc_ctx* c, int64_t i, int first_forward, int32_t colour) {
    const int64_t K = c->K;
    double iv = 1.0 / c->cv[i];
    double base = 1.0 / c->dtimp[i] + 1.0 / c->taut[i];
    for (int64_t k = 0; k < K; ++k) {
        const double* uk = c->u + 3 * k;
        double D = base, off0 = 0.0, off1 = 0.0;
        for (int64_t m = c->cf_off[i]; m < c->cf_off[i + 1]; ++m) {
            int64_t f = c->cf_face[m];
            int64_t a = c->fc[2 * f], b = c->fc[2 * f + 1];
            int64_t j = (a == i) ? b : a;
            double un = dot3(uk, c->fn + 3 * f);
            if (a != i) un = -un;
            double A = c->fa[f] * iv;
            if (un > 0.0) {
                D += A * un;
            } else if (j >= 0 && !(first_forward && c->col[j] > colour)) {
                off0 += A * un * PHI(c->dphi, 0, j, k);
                off1 += A * un * PHI(c->dphi, 1, j, k);
            }
        }
        PHI(c->dphi, 0, i, k) = (PHI(c->res, 0, i, k) - off0) / D;
        PHI(c->dphi, 1, i, k) = (PHI(c->res, 1, i, k) - off1) / D;
    }
}

void orc_step_micro(orc_ctx* c) {
    const int64_t N = c->N, K = c->K;
    const orc_params* P = &c->p;
    /* predicted equilibrium phi~* from W~ and the heat flux q^n (reading: the macro
     * prediction gives no heat flux, so the last Step-6 value is used), then
     * Res_{i,k} = (phi~* - phi^n)/tau~ - F_{i,k} */
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        orc_state s;
        state_from_W(P, c->Wt + 6 * i, c->q + 6 * i, &s);
        double it = 1.0 / c->taut[i];
        for (int64_t k = 0; k < K; ++k) {
            double G, H;
            rykov_eq_point(P, &s, c->u + 3 * k, &G, &H, NULL);
            PHI(c->res, 0, i, k) = (G - PHI(c->phi, 0, i, k)) * it - PHI(c->microF, 0, i, k);
            PHI(c->res, 1, i, k) = (H - PHI(c->phi, 1, i, k)) * it - PHI(c->microF, 1, i, k);
        }
    }
    for (int32_t sw = 0; sw < P->n_micro_sgs; ++sw) {
        for (int dir = 0; dir < 2; ++dir) {
            for (int32_t cc = 0; cc < c->ncol; ++cc) {
                int32_t colour = dir == 0 ? cc : c->ncol - 1 - cc;
                int first_forward = (sw == 0 && dir == 0);
                int64_t lo = c->col_off[colour], hi = c->col_off[colour + 1];
#pragma omp parallel for schedule(static)
                for (int64_t t = lo; t < hi; ++t) micro_point_update(c, c->col_cell[t], first_forward, colour);
            }
        }
    }
}

/* ------------------------------------------------------------------------------ */
/* Step 6: update and integral error compensation, Eqs. solve_rho - solve_qrot    */
/* ------------------------------------------------------------------------------ */
static void update_cell(orc_ctx* c, int64_t i) {
    const int64_t K = c->K;
    const orc_params* P = &c->p;
    const double Z = P->Z_rot;
    {
        orc_state s;
        state_from_W(P, c->Wt + 6 * i, c->q + 6 * i, &s);
        double S[12] = {0};
        for (int64_t k = 0; k < K; ++k) {
            const double* uk = c->u + 3 * k;
            double g1 = PHI(c->phi, 0, i, k) + PHI(c->dphi, 0, i, k);
            double h1 = PHI(c->phi, 1, i, k) + PHI(c->dphi, 1, i, k);
            PHI(c->phi, 0, i, k) = g1;
            PHI(c->phi, 1, i, k) = h1;
            double G, H;
            rykov_eq_point(P, &s, uk, &G, &H, NULL);
            double dg = g1 - G, dh = h1 - H;
            double cv[3] = {uk[0] - s.U[0], uk[1] - s.U[1], uk[2] - s.U[2]};   /* c = u - U~ */
            double c2 = dot3(cv, cv);
            double wk = c->w[k];
            S[0] += wk * dg;
            S[1] += wk * uk[0] * dg;
            S[2] += wk * uk[1] * dg;
            S[3] += wk * uk[2] * dg;
            S[4] += wk * (0.5 * dot3(uk, uk) * dg + dh);
            S[5] += wk * dh;
            for (int d = 0; d < 3; ++d) {
                S[6 + d] += wk * cv[d] * c2 * dg;
                S[9 + d] += wk * cv[d] * dh;
            }
        }
        const double* Wt = c->Wt + 6 * i;
        double* W = c->W + 6 * i;
        double* q = c->q + 6 * i;
        double rho_t = s.rho;
        W[0] = S[0] + Wt[0];
        W[1] = S[1] + Wt[1];
        W[2] = S[2] + Wt[2];
        W[3] = S[3] + Wt[3];
        W[4] = S[4] + Wt[4];
        /* K_rot/2 = 1: exact rotational energy of R~* */
        W[5] = S[5] + rho_t * P->R * ((1.0 - 1.0 / Z) * s.Trot + s.T / Z);
        double atr = (1.0 / 3.0) * (1.0 - (1.0 - P->omega0) / Z);
        double arot = (1.0 - P->delta) * (1.0 - (1.0 - P->omega1) / Z);
        for (int d = 0; d < 3; ++d) {
            double qtr_t = q[d], qrot_t = q[3 + d];
            q[d] = 0.5 * S[6 + d] + qtr_t * atr;
            q[3 + d] = S[9 + d] + qrot_t * arot;
        }
    }
}

void orc_update_cell(orc_ctx* c, int64_t cell) { update_cell(c, cell); }

void orc_micro_point(orc_ctx* c, int64_t cell, int first_forward, int32_t colour) {
    micro_point_update(c, cell, first_forward, colour);
}

void orc_step_update(orc_ctx* c, double res_out[6]) {
    const int64_t N = c->N;
    double* Wold = (double*)malloc(sizeof(double) * 6 * (size_t)N);
    memcpy(Wold, c->W, sizeof(double) * 6 * (size_t)N);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) update_cell(c, i);
    /* residual: global average relative change of each macroscopic variable
     * (Sec. 4.1 names "the global average residual of macroscopic variables";
     * reading: sum_i |W^{n+1} - W^n| / sum_i |W^n| per component, the three
     * momentum components sharing the denominator sum_i |rho U|_i) */
    double num[6] = {0}, den[6] = {0};
    for (int64_t i = 0; i < N; ++i) {
        const double* Wn = c->W + 6 * i;
        const double* Wo = Wold + 6 * i;
        for (int m = 0; m < 6; ++m) num[m] += fabs(Wn[m] - Wo[m]);
        den[0] += fabs(Wo[0]);
        double mom = sqrt(Wo[1] * Wo[1] + Wo[2] * Wo[2] + Wo[3] * Wo[3]);
        den[1] += mom; den[2] += mom; den[3] += mom;
        den[4] += fabs(Wo[4]);
        den[5] += fabs(Wo[5]);
    }
    for (int m = 0; m < 6; ++m) res_out[m] = num[m] / (den[m] > 1e-300 ? den[m] : 1e-300);
    free(Wold);
    c->iter++;
}

int orc_iterate(orc_ctx* c, int32_t n_iter, double tol, int32_t* iters_done, double res_out[6]) {
    if (!c->prepared) return -1;
    double res[6] = {0};
    int32_t it;
    for (it = 0; it < n_iter; ++it) {
        orc_step_gradient(c);
        orc_step_faces(c);
        orc_step_fluxes(c);
        orc_step_macro(c);
        orc_step_micro(c);
        orc_step_update(c, res);
        double mx = 0.0;
        int bad = 0;
        for (int m = 0; m < 6; ++m) {
            if (!(res[m] == res[m]) || isinf(res[m])) bad = 1;
            if (res[m] > mx) mx = res[m];
        }
        if (bad) {
            if (iters_done) *iters_done = it + 1;
            if (res_out) memcpy(res_out, res, sizeof(res));
            return -5;
        }
        if (tol > 0.0 && mx < tol) { ++it; break; }
    }
    if (iters_done) *iters_done = it;
    if (res_out) memcpy(res_out, res, sizeof(res));
    return 0;
}

/* ------------------------------------------------------------------------------ */
/* buffers                                                                        */
/* ------------------------------------------------------------------------------ */
static double* buffer_ptr(const orc_ctx* c, int which, int64_t* len) {
    int64_t NK = c->N * c->K, FK = c->F * c->K;
    switch (which) {
        case ORC_BUF_PHI: *len = 2 * NK; return c->phi;
        case ORC_BUF_W: *len = 6 * c->N; return c->W;
        case ORC_BUF_Q: *len = 6 * c->N; return c->q;
        case ORC_BUF_GRAD: *len = 6 * NK; return c->grad;
        case ORC_BUF_FACE: *len = 2 * FK; return c->face;
        case ORC_BUF_FACE0: *len = 2 * FK; return c->face0;
        case ORC_BUF_FSTATE: *len = 16 * c->F; return c->fstate;
        case ORC_BUF_MICRO_F: *len = 2 * NK; return c->microF;
        case ORC_BUF_MACRO_F: *len = 6 * c->N; return c->macroF;
        case ORC_BUF_WT: *len = 6 * c->N; return c->Wt;
        case ORC_BUF_RES: *len = 2 * NK; return c->res;
        case ORC_BUF_DPHI: *len = 2 * NK; return c->dphi;
        case ORC_BUF_S: *len = c->F; return c->s;
        case ORC_BUF_TAUT: *len = c->N; return c->taut;
        case ORC_BUF_LSTORE: *len = 2 * NK; return c->lstore;
        default: *len = 0; return NULL;
    }
}

int64_t orc_buffer_len(const orc_ctx* c, int which) {
    int64_t len = 0;
    if (which == ORC_BUF_DT) return 3 * c->N;
    buffer_ptr(c, which, &len);
    return len;
}

int orc_get(const orc_ctx* c, int which, double* out) {
    if (!c->prepared) return -1;
    if (which == ORC_BUF_DT) {
        for (int64_t i = 0; i < c->N; ++i) {
            out[3 * i] = c->dt[i]; out[3 * i + 1] = c->dtimp[i]; out[3 * i + 2] = c->eps2[i];
        }
        return 0;
    }
    int64_t len;
    double* p = buffer_ptr(c, which, &len);
    if (!p) return -1;
    memcpy(out, p, sizeof(double) * (size_t)len);
    return 0;
}

int orc_put(orc_ctx* c, int which, const double* in) {
    if (!c->prepared || which == ORC_BUF_DT) return -1;
    int64_t len;
    double* p = buffer_ptr(c, which, &len);
    if (!p) return -1;
    memcpy(p, in, sizeof(double) * (size_t)len);
    return 0;
}

/* ------------------------------------------------------------------------------ */
/* wall quantities, Eqs. cp, cf, ch                                               */
/* ------------------------------------------------------------------------------ */
int64_t orc_n_wall_faces(const orc_ctx* c) {
    int64_t n = 0;
    for (int64_t f = 0; f < c->F; ++f) {
        int64_t b = c->fc[2 * f + 1];
        if (b < 0 && c->bc_kind[-1 - b] == ORC_WALL) ++n;
    }
    return n;
}

/* The wall distribution G_w, R_w is the face distribution of Step 2 at the wall
 * faces, evaluated from the current phi.  n_w is the face normal (pointing from
 * the fluid into the wall).  Force on the body = sum_f A_f sum_k w (u.n) u G_w;
 * heat to the wall = sum_f A_f q_w. */
int orc_surface(orc_ctx* c, double rho_inf, const double* U_inf, double T_inf, double* per_face,
                double force[3], double* heat) {
    if (!c->prepared) return -1;
    orc_step_gradient(c);
    orc_step_faces(c);
    const int64_t K = c->K;
    double U2 = dot3(U_inf, U_inf);
    double qd = 0.5 * rho_inf * U2;
    double p_inf = rho_inf * c->p.R * T_inf;
    double Umag = sqrt(U2);
    int64_t nw = 0;
    force[0] = force[1] = force[2] = 0.0;
    *heat = 0.0;
    for (int64_t f = 0; f < c->F; ++f) {
        int64_t b = c->fc[2 * f + 1];
        if (!(b < 0 && c->bc_kind[-1 - b] == ORC_WALL)) continue;
        const double* n = c->fn + 3 * f;
        double pw = 0.0, mf[3] = {0.0, 0.0, 0.0}, qw = 0.0;
        for (int64_t k = 0; k < K; ++k) {
            const double* uk = c->u + 3 * k;
            double un = dot3(uk, n);
            double g = FACEV(c->face, 0, f, k), h = FACEV(c->face, 1, f, k);
            double wk = c->w[k];
            pw += wk * un * un * g;
            for (int d = 0; d < 3; ++d) mf[d] += wk * un * uk[d] * g;
            qw += wk * un * (0.5 * dot3(uk, uk) * g + h);
        }
        double tw[3] = {mf[0] - n[0] * pw, mf[1] - n[1] * pw, mf[2] - n[2] * pw};
        double* o = per_face + 8 * nw;
        o[0] = pw; o[1] = tw[0]; o[2] = tw[1]; o[3] = tw[2]; o[4] = qw;
        o[5] = (pw - p_inf) / qd;
        o[6] = sqrt(dot3(tw, tw)) / qd;
        o[7] = qw / (qd * Umag);
        for (int d = 0; d < 3; ++d) force[d] += c->fa[f] * mf[d];
        *heat += c->fa[f] * qw;
        ++nw;
    }
    return 0;
}

/* Integrated loads and coefficients (Sec. 4, lift / drag / pitching moment); the
 * force per unit area m_f is the wall momentum flux of Eq. cf's integrand. */
int orc_aero(orc_ctx* c, double rho_inf, const double* U_inf, const double* x_ref,
             double S_ref, double L_ref, const double* lift_dir, double out[10]) {
    if (!c->prepared) return -1;
    const double U2 = dot3(U_inf, U_inf);
    const double q = 0.5 * rho_inf * U2;
    if (!(q > 0.0) || !(S_ref > 0.0) || !(L_ref > 0.0)) return -2;
    const double Um = sqrt(U2);
    const double eD[3] = {U_inf[0] / Um, U_inf[1] / Um, U_inf[2] / Um};
    const double a = dot3(lift_dir, eD);
    double eL[3] = {lift_dir[0] - a * eD[0], lift_dir[1] - a * eD[1], lift_dir[2] - a * eD[2]};
    const double nl = sqrt(dot3(eL, eL));
    if (!(nl > 1e-12 * sqrt(dot3(lift_dir, lift_dir)))) return -2;
    for (int d = 0; d < 3; ++d) eL[d] /= nl;
    const double eP[3] = {eL[1] * eD[2] - eL[2] * eD[1], eL[2] * eD[0] - eL[0] * eD[2],
                          eL[0] * eD[1] - eL[1] * eD[0]};
    orc_step_gradient(c);
    orc_step_faces(c);
    double F[3] = {0.0, 0.0, 0.0}, M[3] = {0.0, 0.0, 0.0};
    for (int64_t f = 0; f < c->F; ++f) {
        int64_t b = c->fc[2 * f + 1];
        if (!(b < 0 && c->bc_kind[-1 - b] == ORC_WALL)) continue;
        const double* n = c->fn + 3 * f;
        double m[3] = {0.0, 0.0, 0.0};
        for (int64_t k = 0; k < c->K; ++k) {
            const double* uk = c->u + 3 * k;
            const double wg = c->w[k] * dot3(uk, n) * FACEV(c->face, 0, f, k);
            for (int d = 0; d < 3; ++d) m[d] += wg * uk[d];
        }
        const double A = c->fa[f];
        const double r[3] = {c->fx[3 * f] - x_ref[0], c->fx[3 * f + 1] - x_ref[1], c->fx[3 * f + 2] - x_ref[2]};
        for (int d = 0; d < 3; ++d) F[d] += A * m[d];
        M[0] += A * (r[1] * m[2] - r[2] * m[1]);
        M[1] += A * (r[2] * m[0] - r[0] * m[2]);
        M[2] += A * (r[0] * m[1] - r[1] * m[0]);
    }
    for (int d = 0; d < 3; ++d) { out[d] = F[d]; out[3 + d] = M[d]; }
    out[6] = dot3(F, eD) / (q * S_ref);
    out[7] = dot3(F, eL) / (q * S_ref);
    out[8] = dot3(M, eP) / (q * S_ref * L_ref);
    out[9] = out[7] / out[6];
    return 0;
}
