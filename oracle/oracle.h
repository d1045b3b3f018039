/*
 * CPU oracle for the conservative implicit Rykov scheme (Zhang, Liu, Chen, Zhong,
 * Zhuo, "A conservative implicit scheme for three-dimensional steady flows of
 * diatomic gases in all flow regimes using unstructured meshes in the physical and
 * velocity spaces").
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, FP64 restatement of Steps 1-7
 * of Sec. 3.5, used to check the CUDA library.  It shares no code with the CUDA
 * path.  Only the tests, the smoke check and the CPU-baseline leg of the benchmark
 * may load it.
 *
 * Array conventions (all host memory, all owned by the caller unless stated):
 *   phi[field][cell][k]  field 0 = G (translational reduced distribution, called g),
 *                        field 1 = R (rotational reduced distribution, called h).
 *   W[cell][6]           (rho, rho U_x, rho U_y, rho U_z, rho E, rho E_rot)
 *   q[cell][6]           (q_tr x,y,z, q_rot x,y,z)
 */
#ifndef RYKOV_ORACLE_H
#define RYKOV_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    double R;           /* specific gas constant (1/2 in the paper's units)         */
    double Z_rot;       /* rotational collision number                              */
    double omega_vis;   /* VHS viscosity index, Eq. T_solve_mu                      */
    double mu_ref;      /* reference viscosity at T_ref                             */
    double T_ref;
    double omega0, omega1, delta;   /* Rykov constants, Eqs. eqdf_Grot, eqdf_Rtra   */
    double cfl_s;       /* CFL number of the local physical step s_ij (Sec. 3.3)    */
    double cfl_imp;     /* implicit step = cfl * CFL step (Sec. 3.1): the largest cfl */
    double cfl_imp0;    /* cfl of the first iteration after set_state (<= 0: cfl_imp) */
    double cfl_ramp;    /* growth factor of cfl per iteration, capped at cfl_imp      */
    double lim_k;       /* Venkatakrishnan constant K                               */
    int32_t n_micro_sgs;   /* PR-SGS iterations of the micro system (2, Sec. 3.1)  */
    int32_t n_macro_sgs;   /* PR-SGS iterations of the macro system (40, Sec. 3.2) */
    int32_t limiter;       /* 0 unlimited, 1 Venkatakrishnan, 2 first order        */
    int32_t first_order_iters; /* iterations run first order after set_state      */
    int32_t limiter_freeze;    /* > 0: from this iteration on the limiter values of
                                  iteration limiter_freeze - 1 are reused (0: never) */
    int32_t viscosity_law;     /* 0: power law (omega_vis), Eq. T_solve_mu;
                                  1: Sutherland's law (sutherland_c), Eq. T_solve_mu_Sut */
    double sutherland_c;       /* Sutherland constant C_s in units of temperature  */
} orc_params;

enum { ORC_WALL = 0, ORC_FARFIELD = 1 };

typedef struct orc_ctx orc_ctx;

/* Primitive state used to evaluate the Rykov equilibria (Eqs. eqdf_G* - eqdf_Rrot). */
typedef struct {
    double rho, U[3], T, Ttr, Trot, qtr[3], qrot[3];
} orc_state;

/* ---- set-up ------------------------------------------------------------------ */
orc_ctx* orc_create(const orc_params* p);
void     orc_destroy(orc_ctx* c);
int      orc_set_mesh(orc_ctx* c, int64_t n_cell, int64_t n_face, const int64_t* face_cell,
                      const double* face_normal, const double* face_area,
                      const double* face_center, const double* cell_center,
                      const double* cell_volume, const int32_t* cell_colour);
int      orc_set_dvs(orc_ctx* c, int64_t K, const double* u, const double* w);
int      orc_set_bc(orc_ctx* c, int32_t bc_id, int32_t kind, double rho, const double* U,
                    double T);
int      orc_set_params(orc_ctx* c, const orc_params* p);
/* Builds CSR, CFL steps, LSQ matrices.  Must follow set_mesh/set_dvs. */
int      orc_prepare(orc_ctx* c);

/* ---- state ---------------------------------------------------------------------*/
/* Step 1: prim[N][6] = (rho, U, T_tr, T_rot); q may be NULL (zero).  Sets W, q and
 * phi = Rykov equilibrium of that state. */
int      orc_set_state_prim(orc_ctx* c, const double* prim, const double* q);
int      orc_set_state(orc_ctx* c, const double* W, const double* q, const double* phi);

/* ---- the iteration (Steps 2-7) --------------------------------------------------*/
int      orc_iterate(orc_ctx* c, int32_t n_iter, double tol, int32_t* iters_done,
                     double res_out[6]);
/* the individual steps, in order, for step-by-step checks */
void     orc_step_gradient(orc_ctx* c);   /* Eq. flux_solve_phi_phi ingredients   */
void     orc_step_faces(orc_ctx* c);      /* Step 2 (a)-(d)                        */
void     orc_step_fluxes(orc_ctx* c);     /* Step 2 (e) and Step 3                 */
void     orc_step_macro(orc_ctx* c);      /* Step 4                                */
void     orc_step_micro(orc_ctx* c);      /* Step 5                                */
void     orc_step_update(orc_ctx* c, double res_out[6]);   /* Step 6 + residual    */
/* The units of Steps 5 and 6 for one cell, on the context's current buffers:
 * one point update of the micro PR-SGS (Eq. implicit_mic_final_equ: Delta phi_i from
 * Res_i, the neighbours' Delta phi, tau~_i and the implicit step of the current
 * iteration), and the update phi += Delta phi with the compensated W, q of Eqs.
 * solve_rho - solve_qrot from W~_i and q_i (no residual). */
void     orc_micro_point(orc_ctx* c, int64_t cell, int first_forward, int32_t colour);
void     orc_update_cell(orc_ctx* c, int64_t cell);

/* ---- read-back -----------------------------------------------------------------*/
enum {
    ORC_BUF_PHI = 0,      /* [2][N][K]                                          */
    ORC_BUF_W = 1,        /* [N][6]                                             */
    ORC_BUF_Q = 2,        /* [N][6]                                             */
    ORC_BUF_GRAD = 3,     /* limited gradient [2][3][N][K]                      */
    ORC_BUF_FACE = 4,     /* face distribution phi_ij [2][F][K] (after step 2)  */
    ORC_BUF_FACE0 = 5,    /* reconstructed phi(x_ij - u s) [2][F][K]            */
    ORC_BUF_FSTATE = 6,   /* face state [F][16]                                 */
    ORC_BUF_MICRO_F = 7,  /* micro flux F_{i,k} [2][N][K]                       */
    ORC_BUF_MACRO_F = 8,  /* macro flux F_i [N][6]                              */
    ORC_BUF_WT = 9,       /* predicted W~ [N][6]                                */
    ORC_BUF_RES = 10,     /* micro residual Res_{i,k} [2][N][K]                 */
    ORC_BUF_DPHI = 11,    /* Delta phi [2][N][K]                                */
    ORC_BUF_DT = 12,      /* [N][3]: CFL step, implicit step, eps^2             */
    ORC_BUF_S = 13,       /* [F] local physical step s_ij                       */
    ORC_BUF_TAUT = 14,    /* [N] predicted relaxation time tau~                  */
    ORC_BUF_LSTORE = 15   /* [2][N][K] frozen limiter values                      */
};
int64_t  orc_buffer_len(const orc_ctx* c, int which);
int      orc_get(const orc_ctx* c, int which, double* out);
int      orc_put(orc_ctx* c, int which, const double* in);

/* Wall quantities of the current state (Eqs. cp, cf, ch): per wall face
 * [p_w, tau_x, tau_y, tau_z, q_w, Cp, Ctau, Ch]; totals force[3], heat. */
int64_t  orc_n_wall_faces(const orc_ctx* c);
int      orc_surface(orc_ctx* c, double rho_inf, const double* U_inf, double T_inf,
                     double* per_face, double force[3], double* heat);
/* Aerodynamic loads of the current state (the lift, drag, lift-to-drag and pitching
 * moment results of Sec. 4): force F = sum_f A_f m_f and moment M = sum_f A_f
 * (x_f - x_ref) x m_f over the wall faces, m_f = sum_k w (u.n) u g_f; with
 * q = rho_inf |U_inf|^2 / 2, e_D = U_inf/|U_inf|, e_L = lift_dir with its e_D part
 * removed, normalised, and e_P = e_L x e_D:
 * out = [F(3), M(3), C_D = F.e_D/(q S), C_L = F.e_L/(q S), C_m = M.e_P/(q S L), C_L/C_D].
 * Returns -2 for a lift direction parallel to U_inf or a non-positive S, L, q. */
int      orc_aero(orc_ctx* c, double rho_inf, const double* U_inf, const double* x_ref,
                  double S_ref, double L_ref, const double* lift_dir, double out[10]);

/* ---- pure functions for the pins -----------------------------------------------*/
void     orc_equilibrium(const orc_params* p, const orc_state* s, int64_t K,
                         const double* u, double* G, double* H);
void     orc_equilibrium_parts(const orc_params* p, const orc_state* s, int64_t K,
                               const double* u, double* Gtr, double* Grot,
                               double* Htr, double* Hrot);
/* Step 2 (b)-(d) for one interior face: reconstructed g0,h0 -> face state (16
 * doubles, layout of ORC_BUF_FSTATE) and face distribution g_f,h_f. */
void     orc_interface(const orc_params* p, int64_t K, const double* u, const double* w,
                       const double* g0, const double* h0, double s, double* state16,
                       double* gf, double* hf);
void     orc_euler_flux(const orc_params* p, const double* W, const double* n, double* G);
double   orc_spectral_radius(const orc_params* p, const double* Wm, const double* n,
                             double dl);
double   orc_venkat(double d1, double d2, double eps2);

#ifdef __cplusplus
}
#endif
#endif
