/*
 * librykov -- GB300 (sm_103a) implementation of the per-iteration hot path of the
 * conservative implicit scheme for steady diatomic-gas flows of Zhang, Liu, Chen,
 * Zhong and Zhuo (Rykov model, unstructured physical mesh, unstructured discrete
 * velocity space).  One call of rk_implicit_iterate performs Steps 2-7 of the
 * paper's Sec. 3.5 for every (cell, discrete velocity) pair on the device.
 *
 * Conventions for every entry point
 *   - Return value: RK_OK (0) or a negative RK_E* code; rk_last_error() gives a
 *     message.  No C++ exception crosses this boundary.
 *   - All device work is enqueued on the CUDA stream given to rk_create (the
 *     caller's stream).  Calls that return data to host memory synchronise that
 *     stream before returning.
 *   - The library never allocates device memory: the caller allocates one
 *     workspace of rk_workspace_size() bytes and binds it; the library carves all
 *     device arrays from it and never frees it.  Host pointers passed in are only
 *     read during the call (their contents are copied); the caller keeps ownership.
 *   - A context is not thread safe; use one context per stream.
 *
 * Array layouts (row-major, C order):
 *   face_cell[F][2]   (left cell, right cell); right < 0 marks a boundary face whose
 *                     boundary-condition id is -1-right.
 *   face_normal[F][3] unit normal from left to right (outward at boundary faces).
 *   W[N][6]           (rho, rho U_x, rho U_y, rho U_z, rho E, rho E_rot), Eq.
 *                     phi_solve_mac; prim[N][6] = (rho, U_x, U_y, U_z, T_tr, T_rot).
 *   q[N][6]           (q_tr x,y,z, q_rot x,y,z), Eqs. phi_solve_qtra / qrot.
 *   distribution      [2][N][K_pad] in the context precision (double for RK_FP64,
 *                     float for RK_MIXED); field 0 = G (called g), 1 = R (called h);
 *                     K_pad = K rounded up to a multiple of 32 (rk_dims).
 * All quantities are dimensionless as in the paper's Sec. 4 (U_ref = sqrt(2 R T_ref)).
 */
#ifndef RYKOV_H
#define RYKOV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RK_VERSION 102

enum {
    RK_OK = 0,
    RK_EINVAL = -1,     /* bad argument or inconsistent input                    */
    RK_ENOMEM = -2,     /* workspace missing or too small                        */
    RK_ECUDA = -3,      /* a CUDA runtime call failed                            */
    RK_EDEVICE = -4,    /* a kernel raised its device status flag                */
    RK_EDIVERGED = -5,  /* non-finite residual                                   */
    RK_ETIMEOUT = -6,   /* a bounded device wait gave up (cooperative solve)     */
    RK_ESTATE = -7      /* call out of order (e.g. iterate before set_state)     */
};

enum { RK_FP64 = 0, RK_MIXED = 1 };         /* context precision                 */
/* Flags or-ed into the precision argument of rk_create:
 *   RK_DEBUG_FLAG     reserve the verification buffers of rk_debug_get/rows;
 *   RK_MACRO_FP32     RK_MIXED only: solve the macro PR-SGS of Step 4 in FP32 in
 *                     delta form instead of FP64 (faster; its iterates differ from
 *                     the FP64 solve's by ~1e-6 of the increment, and its converged
 *                     state is the same).  FP64 contexts ignore it. */
enum { RK_DEBUG_FLAG = 0x100, RK_MACRO_FP32 = 0x200 };
enum { RK_WALL = 0, RK_FARFIELD = 1 };      /* boundary-condition kinds          */

/* Scheme parameters.  Field order and meaning are part of the ABI. */
typedef struct rk_params {
    double R;           /* specific gas constant (1/2 in the paper's units)       */
    double Z_rot;       /* rotational collision number, Eq. model_equ_f           */
    double omega_vis;   /* VHS index, Eq. T_solve_mu                              */
    double mu_ref;      /* viscosity at T_ref                                     */
    double T_ref;
    double omega0, omega1, delta;   /* Rykov constants, Eqs. eqdf_Grot - Rrot     */
    double cfl_s;       /* CFL number of Delta t_i that sets s_ij (Sec. 3.3)      */
    double cfl_imp;     /* implicit step = cfl * Delta t_i: the largest cfl       */
    double cfl_imp0;    /* cfl of the first iteration after set_state (<=0: none) */
    double cfl_ramp;    /* geometric growth of cfl per iteration                  */
    double lim_k;       /* Venkatakrishnan K: eps^2 = (K V^{1/3})^3 phi_i^2 (relative) */
    int32_t n_micro_sgs;   /* PR-SGS iterations of Eq. implicit_mic_final_equ (2) */
    int32_t n_macro_sgs;   /* PR-SGS iterations of Eq. implicit_mac_equ_fin (40)  */
    int32_t limiter;       /* 0 unlimited, 1 Venkatakrishnan, 2 first order       */
    int32_t first_order_iters; /* first-order iterations after set_state          */
    int32_t limiter_freeze;    /* > 0 (and > first_order_iters): iterations from this
                                  one on reuse the limiter values of iteration
                                  limiter_freeze - 1 (no counterpart in the paper: the
                                  limiter's switching otherwise stalls the residual);
                                  0: never                                        */
    int32_t viscosity_law;     /* 0: power law mu_ref (T_tr/T_ref)^omega_vis,
                                  Eq. T_solve_mu; 1: Sutherland's law with constant
                                  sutherland_c, Eq. T_solve_mu_Sut                 */
    double sutherland_c;       /* C_s >= 0 in the units of T (111 K for nitrogen) */
} rk_params;

typedef struct rk_ctx rk_ctx;

int rk_version(void);

/* Create a context of the given precision whose work goes to `cuda_stream`
 * (a cudaStream_t cast to uintptr_t; 0 = legacy default stream).
 * Arithmetic: RK_FP64 computes everything in FP64.  RK_MIXED stores the
 * distributions in FP32 and computes per velocity in FP32, with compensated sums
 * over the velocities combined in FP64, FP64 moments, interface states and
 * compensation (Step 6), and the macro PR-SGS of Step 4 in FP64.  With the
 * RK_MACRO_FP32 flag the macro PR-SGS runs in FP32 in delta form instead: its
 * constant part is formed in FP64 and every FP32 rounding is relative to the
 * increment, so the converged state is the FP64 solve's.
 * Environment switches read here (results unchanged unless noted):
 *   RYKOV_GRAPH=0       no CUDA graph of an iteration;
 *   RYKOV_COOP=1        cooperative launch of the FP64 macro PR-SGS (grid barriers
 *                       between colour phases, each wait bounded by 1 s; a wait that
 *                       runs out makes rk_implicit_iterate return RK_ETIMEOUT, once);
 *   RYKOV_COOP_UNREACHABLE=1  tests of that bound only: the barriers wait for one
 *                       arrival more than the grid makes, with a 50 ms bound;
 *   RYKOV_STAGED=b      micro sweeps with staged row loads (bit mask, default 4;
 *                       + 8: the cell's own rows by bulk copies with mbarrier
 *                       completion in the packed kernels, same results);
 *   RYKOV_PRIO=0        no stream priorities in the graph;
 *   RYKOV_PDL=1         macro phases with programmatic serialisation (default off:
 *                       the plain launches overlap better with the micro flux);
 *   RYKOV_PACKED=0      RK_MIXED per-velocity kernels with scalar FP32 arithmetic
 *                       instead of packed FP32 pairs (rounding-level differences);
 *   RYKOV_MACRO_LANES=L threads per cell of the FP32 macro phases, 1, 2 or 4 (default
 *                       4; another order of the face sums, ~1e-6 of the increment);
 *   RYKOV_ADJ_FP64=1    RK_MIXED adjoint in FP64 (see the adjoint section). */
int rk_create(rk_ctx** out, int precision, uintptr_t cuda_stream);
int rk_destroy(rk_ctx* ctx);
const char* rk_last_error(const rk_ctx* ctx);

/* Mesh (Sec. 3.1: cells V_i, faces A_ij, n_ij, neighbour sets N(i)).  Host
 * pointers.  cell_colour must be a proper colouring of the face-neighbour graph
 * (it fixes the Gauss-Seidel order: colours ascending forward, descending
 * backward).  Validates: indices, positive volumes and areas, geometric closure
 * (sum_f A_f n_f = 0 per cell, relative 1e-8), colouring, at most 8 faces per cell.
 * Invalidates any bound workspace. */
int rk_upload_mesh(rk_ctx* ctx, int64_t n_cell, int64_t n_face, const int64_t* face_cell,
                   const double* face_normal, const double* face_area,
                   const double* face_center, const double* cell_center,
                   const double* cell_volume, const int32_t* cell_colour);

/* Discrete velocity space: points u[K][3] (DVS-cell centroids) and weights w[K]
 * (DVS-cell volumes), Sec. 3.2 text after Eq. implicit_mac_equ_mac_flux.  Host
 * pointers.  Invalidates any bound workspace. */
int rk_upload_dvs(rk_ctx* ctx, int64_t K, const double* u, const double* w);

int rk_set_params(rk_ctx* ctx, const rk_params* p);

/* Boundary condition for faces with bc id `bc_id` (0..63).  RK_WALL: diffuse
 * reflection with full accommodation at wall velocity U and temperature T (rho
 * unused).  RK_FARFIELD: incoming freestream Maxwellian (rho, U, T). */
int rk_set_bc(rk_ctx* ctx, int32_t bc_id, int32_t kind, double rho, const double* U, double T);

/* Dimensions after upload: N, F, K, K_pad, number of colours, wall faces. */
int rk_dims(const rk_ctx* ctx, int64_t out[6]);

/* Bytes of device workspace needed for the uploaded mesh/DVS and precision. */
int rk_workspace_size(rk_ctx* ctx, size_t* bytes);
/* Bind a caller-owned device buffer (at least rk_workspace_size bytes, 256-byte
 * aligned) and run the set-up kernels (CFL steps, s_ij, least-squares weights). */
int rk_bind_workspace(rk_ctx* ctx, void* dev_ptr, size_t bytes);

/* Step 1 of Sec. 3.5: W from primitives, q (NULL = 0), and each cell's
 * distributions set to the Rykov equilibrium of (W, q).  Host or device
 * (on_device != 0) pointers to doubles.  Resets the iteration counter. */
int rk_set_state_prim(rk_ctx* ctx, const double* prim, const double* q, int on_device);
/* Restore W, q and the distribution (context precision layout above). */
int rk_set_state(rk_ctx* ctx, const double* W, const double* q, const void* dist, int on_device);
int rk_get_distribution(rk_ctx* ctx, void* dist, int on_device);

/* Steps 2-7 repeated n_iter times; stops early once max residual < tol (tol <= 0:
 * fixed count).  iters_done and res_out (6 doubles: rho, rho U x,y,z, rho E,
 * rho E_rot; may be NULL) are written on return.  Residual: sum_i |W^{n+1}-W^n|
 * / sum_i |W^n| per component (momentum normalised by sum_i |rho U|_i).
 * Returns RK_EDIVERGED when a residual is not finite. */
int rk_implicit_iterate(rk_ctx* ctx, int32_t n_iter, double tol, int32_t* iters_done,
                        double res_out[6]);
/* Residual of the last iteration. */
int rk_residual(rk_ctx* ctx, double res_out[6]);

/* Macroscopic state: W[N][6], q[N][6], T3[N][3] = (T, T_tr, T_rot); any pointer
 * may be NULL.  Host or device doubles. */
int rk_moments(rk_ctx* ctx, double* W, double* q, double* T3, int on_device);

/* Wall quantities of the current state, Eqs. cp, cf, ch: per wall face (in face
 * order) 8 doubles [p_w, tau_x, tau_y, tau_z, q_w, Cp, C_tau, C_h] with freestream
 * (rho_inf, U_inf, T_inf); force[3] = sum_f A_f sum_k w (u.n) u G_w (force of the
 * gas on the walls) and heat = sum_f A_f q_w.  Host pointers. */
int rk_surface(rk_ctx* ctx, double rho_inf, const double* U_inf, double T_inf,
               double* per_wall_face, double force[3], double* heat);

/* Aerodynamic loads of the current state: the lift, drag, lift-to-drag ratio and
 * pitching moment that Sec. 4 reports for the blunted cone and the capsule (the
 * paper gives no formulas; these are the standard definitions).  Over the wall
 * faces, with m_f = sum_k w (u.n) u g_f the momentum flux into the wall (Eq. cf's
 * integrand): force F = sum_f A_f m_f, moment M = sum_f A_f (x_f - x_ref) x m_f.
 * With q = rho_inf |U_inf|^2 / 2, e_D = U_inf/|U_inf|, e_L = lift_dir minus its
 * e_D component, normalised, and the pitch axis e_P = e_L x e_D (a positive C_m
 * turns the upstream nose towards e_L):
 *   out[10] = [F_x, F_y, F_z, M_x, M_y, M_z, C_D = F.e_D/(q S_ref),
 *              C_L = F.e_L/(q S_ref), C_m = M.e_P/(q S_ref L_ref), L/D = C_L/C_D].
 * Host pointers (U_inf, x_ref, lift_dir: 3 doubles).  RK_EINVAL for a null pointer,
 * non-positive rho_inf, |U_inf|, S_ref or L_ref, or lift_dir parallel to U_inf;
 * RK_ESTATE before a state is set.  Recomputes the face values of the current
 * state (as rk_surface does); the state itself is not changed. */
int rk_aero(rk_ctx* ctx, double rho_inf, const double* U_inf, const double* x_ref, double S_ref,
            double L_ref, const double* lift_dir, double out[10]);

/* ---- step access for verification ------------------------------------------ */
enum {
    RK_STEP_RECON = 0,   /* LSQ gradient, limiter, reconstruction (Eq. flux_solve_phi_phi) */
    RK_STEP_FACES = 1,   /* Step 2 (b)-(d): interface state and face distribution         */
    RK_STEP_FLUXES = 2,  /* Step 3: macro flux per cell, spectral radii                    */
    RK_STEP_MACRO = 3,   /* Step 4: implicit macroscopic prediction                        */
    RK_STEP_MICRO = 4    /* Steps 5-6: micro PR-SGS, update, compensation, residual        */
};
/* Run one step of the iteration (in order RECON..MICRO; MICRO advances the
 * iteration counter). */
int rk_step(rk_ctx* ctx, int step);

enum {
    RK_BUF_PHI = 0, RK_BUF_W = 1, RK_BUF_Q = 2, RK_BUF_FACE = 4, RK_BUF_FSTATE = 6,
    RK_BUF_MICRO_F = 7, RK_BUF_MACRO_F = 8, RK_BUF_WT = 9, RK_BUF_RES = 10,
    RK_BUF_DPHI = 11, RK_BUF_DT = 12, RK_BUF_S = 13, RK_BUF_TAUT = 14
};
/* Copy an internal buffer to host memory as doubles, without K padding:
 * PHI/MICRO_F/RES/DPHI [2][N][K], FACE [2][F][K], FSTATE [F][16], W/Q/MACRO_F/WT
 * [N][6], DT [N][3] (CFL step, implicit step, eps^2), S [F], TAUT [N].
 * `count` is the number of doubles the caller's buffer holds. */
int rk_debug_get(rk_ctx* ctx, int which, double* host_out, int64_t count);
/* Selected rows of a distribution-shaped verification buffer, for checks of large
 * cases one cell or face at a time: which = RK_BUF_PHI, RK_BUF_RES, RK_BUF_DPHI,
 * RK_BUF_MICRO_F (rows = cell indices) or RK_BUF_FACE (rows = face indices);
 * host_out[2][n_rows][K] doubles (field, row, velocity).  RK_BUF_MICRO_F needs a
 * context created with RK_DEBUG.  RK_EINVAL for a row out of range. */
int rk_debug_rows(rk_ctx* ctx, int which, const int64_t* rows, int64_t n_rows, double* host_out);

/* ---- per-kernel timing ----------------------------------------------------------
 * rk_profile(ctx, 1) makes the library bracket each kernel class below with CUDA
 * events on its stream (an event pair per launch); rk_profile_get returns, per
 * class, the summed device milliseconds and the launch count since the last
 * rk_profile call, plus in counts[RK_PROF_N] the total number of kernels launched
 * by this context since creation (with or without profiling).  Reading the
 * events synchronises the stream. */
enum {
    RK_PROF_RECON = 0, RK_PROF_FACE_INT = 1, RK_PROF_FACE_BND = 2, RK_PROF_FLUXES = 3,
    RK_PROF_MACRO = 4, RK_PROF_MICRO_FIRST = 5, RK_PROF_MICRO_MID = 6,
    RK_PROF_MICRO_LAST = 7, RK_PROF_UPDATE = 8, RK_PROF_N = 9
};
int rk_profile(rk_ctx* ctx, int enable);
/* ms[RK_PROF_N], counts[RK_PROF_N + 1] */
int rk_profile_get(rk_ctx* ctx, double* ms, int64_t* counts);

/* ---- residual without device allocation ------------------------------------------
 * The paper has no counterpart: this entry point exists for callers that cannot
 * allocate device memory -- for example a convergence monitor or plug-in that runs
 * inside another framework whose caching allocator owns the device memory (a raw
 * cudaMalloc there can fail or force a synchronising release), or a check made
 * every iteration that must not add an allocation or its failure path.
 *
 * Computes, on `cuda_stream`, the residual of one implicit step from two states:
 * res_out[m] = sum_i |W_new[i][m] - W_old[i][m]| / sum_i |W_old[i][m]| for m = rho,
 * rho E, rho E_rot, and with sum_i |rho U|_i as the denominator of the three
 * momentum rows -- the same definition as rk_implicit_iterate's res_out.
 *   W_new, W_old : device pointers, [n_cell][6] doubles (caller-owned inputs)
 *   res_out      : device pointer, 6 doubles (caller-owned output, written)
 *   n_cell       : 1 .. RK_NOALLOC_MAX_CELLS, larger sizes return RK_EINVAL
 * It allocates nothing: its scratch (per-block partial sums, 12 doubles per 256
 * cells) is one fixed array of RK_NOALLOC_MAX_CELLS / 256 * 12 doubles (384 KiB)
 * in the library's device memory, which every GPU that loads the library holds
 * until the process exits.  All calls on one device share that array: calls whose
 * work overlaps on that GPU (for instance on two streams) race on it and give wrong
 * results; calls on different devices do not, each device having its own copy.
 * Each call overwrites every part of the array it reads, so nothing carries over
 * from one call to the next.  Every call made outside stream capture looks the
 * array's device address up on the current device (so the address stays valid after
 * a device reset); a call during capture reuses the address of the last uncaptured
 * call on that device, so make one call on each device before any stream capture.
 * Returns RK_OK, RK_EINVAL (null pointer, bad size) or RK_ECUDA;
 * rk_noalloc_last_error() gives the message of the calling thread's last call (empty
 * after a call that succeeded).  Asynchronous: the result is ready when the stream
 * reaches it. */
#define RK_NOALLOC_MAX_CELLS 1048576
int rk_residual_noalloc(const double* W_new, const double* W_old, int64_t n_cell,
                        double* res_out, uintptr_t cuda_stream);
const char* rk_noalloc_last_error(void);


/* ---- adjoint of the steady residual operator -------------------------------------
 * A steady state of the implicit iteration (Sec. 3.5 with a zero micro increment and
 * a zero macro increment) is a zero of R(X; p), X = (phi, W, q):
 *   R_phi = (phi*(W, q) - phi)/tau(W) - F(phi; p)            Eq. implicit_mic_final_equ
 *   R_W   = sum_k w Psi (phi - phi*(W, q)), with rho R((1 - 1/Z) T_rot + T/Z) - rho E_rot
 *           added in the rho E_rot row                        Eqs. solve_rho - solve_Erot
 *   R_q   = 1/2 sum_k w c|c|^2 (g - g*) + (a_tr - 1) q_tr,  sum_k w c (h - h*) +
 *           (a_rot - 1) q_rot, c = u - U(W)                    Eqs. solve_qtr, solve_qrot
 * with F the micro flux of Eq. implicit_mic_flux (interface distribution of Eq.
 * flux_solve_phi, limited reconstruction of Eq. flux_solve_phi_phi, the boundary
 * treatment of the iteration) and the limiter of rk_params (the start-up order switch
 * does not apply).  Parameters p[RK_NPARAM] = (T_w, rho_inf, U_inf x/y/z, T_inf):
 * p[0] shifts the temperature of every wall boundary, p[1..5] set the state of every
 * farfield boundary; derivatives are with respect to these shifts.
 * Objectives (Eqs. cp, cf, ch): RK_OBJ_HEAT = sum over wall faces of A_f q_w,
 * q_w = sum_k w (u.n)(|u|^2/2 g_f + h_f); RK_OBJ_DRAG = (sum over wall faces of
 * A_f sum_k w (u.n) u g_f) . e, e = U_inf/|U_inf| of the first farfield boundary
 * (the x axis if there is none).
 *
 * State vectors ("packed", rk_state_len doubles): phi as [2][N][K] (no K padding),
 * then W[N][6], then q[N][6].  on_device = 1: the pointers are device pointers of that
 * size; 0: host pointers.  Every call evaluates at the context's current state.
 *
 * The adjoint needs a second caller-owned device workspace of
 * rk_adjoint_workspace_size(ctx, krylov_dim) bytes (256-byte aligned), bound with
 * rk_bind_adjoint_workspace after rk_bind_workspace; krylov_dim (1..64) is the
 * dimension of one GMRES restart cycle.  Rebinding the main workspace unbinds it.
 * Arithmetic: FP64 for RK_FP64 contexts.  RK_MIXED contexts evaluate at their own
 * state (FP32 distributions; rk_put_state rounds phi to FP32) with the per-velocity
 * work of rk_vjp, rk_objective and the GMRES preconditioner in FP32 (velocity sums
 * compensated and combined in FP64; vectors, per-cell and per-face scalars and the
 * Krylov arithmetic in FP64); relative accuracy ~1e-6, except that the limiter's
 * derivative is dropped where the limited differences are below 1e-30 (far tails).
 * The environment variable RYKOV_ADJ_FP64=1 makes mixed contexts use FP64 there too.
 *
 *   rk_steady_residual(ctx, r, on_device): r = R(X; p).
 *   rk_vjp(ctx, v, out, out_params, on_device): out = (dR/dX)^T v, out_params[6] =
 *       (dR/dp)^T v (out_params may be NULL).  Reverse mode of the kernels: exact up
 *       to round-off wherever R is differentiable (the limiter's min/max choices are
 *       held at the ones taken at X).
 *   rk_objective(ctx, objective, J, dJdX, dJdp, on_device): J(X; p), its gradient
 *       with respect to X (packed, may be NULL) and its explicit p-derivative dJdp[6].
 *   rk_adjoint_solve(ctx, objective, max_iter, tol, iters_done, rel_res, J, dJdp):
 *       solves (dR/dX)^T lam = -dJ/dX by restarted GMRES, right-preconditioned with
 *       the transpose of the forward iteration's linearised step: the transposed
 *       point Gauss-Seidel sweeps of the micro PR-SGS operator (n_micro_sgs x forward
 *       + backward colour sweeps; implicit CFL cfl_imp), coupled through the collision
 *       term's W derivative to n_macro_sgs transposed colour sweeps of the macro
 *       operator of Eq. implicit_mac_equ_fin and back through the moments (the
 *       environment variable RYKOV_ADJ_PC=micro keeps the micro sweeps alone, with -1
 *       on the (W, q) block); stops when ||(dR/dX)^T lam + dJ/dX||_2 <=
 *       tol ||dJ/dX||_2 or after max_iter Krylov iterations, starting from the last
 *       solution of the same objective at the same state (0 otherwise).  Returns the
 *       iterations done, the final relative residual (recomputed, not estimated),
 *       J, and the total derivative dJdp[6] = dJ/dp + lam^T dR/dp.  RK_EDIVERGED if
 *       the residual becomes non-finite.
 *   rk_adjoint_get(ctx, lam, on_device): the last adjoint solution (packed). */
/* Fused multiply-add throughput of the current device (a measurement utility with
 * no counterpart in the paper): the ALU ceiling of the FP64 form, whose per-velocity
 * FP64 arithmetic (GB300 issues FP64 at 1/64 of its FP32 rate) rather than HBM bounds
 * it.  kind: RK_PEAK_FP64 (DFMA) or RK_PEAK_FP32 (FFMA).  Launches a kernel of
 * independent FMA chains (~0.1-0.3 s) four times on `cuda_stream` (the first is a
 * warm-up), times each with CUDA events, and returns the best rate in TFLOP/s
 * (2 flops per FMA) in *tflops.  dev_sink: caller-owned device memory of at least 8
 * bytes, written only to keep the chains live.  Synchronises the stream.
 * RK_EINVAL for a bad kind or null pointer, RK_ECUDA if a launch fails. */
enum { RK_PEAK_FP64 = 0, RK_PEAK_FP32 = 1 };
int rk_peak_flops(int kind, uintptr_t cuda_stream, void* dev_sink, double* tflops);

#define RK_NPARAM 6
enum { RK_OBJ_HEAT = 0, RK_OBJ_DRAG = 1 };
int rk_state_len(const rk_ctx* ctx, int64_t* n);
int rk_adjoint_workspace_size(rk_ctx* ctx, int32_t krylov_dim, size_t* bytes);
int rk_bind_adjoint_workspace(rk_ctx* ctx, int32_t krylov_dim, void* dev_ptr, size_t bytes);
/* X as a packed state vector, and setting X from one (sets phi, W, q as given) */
int rk_get_state(rk_ctx* ctx, double* x, int on_device);
int rk_put_state(rk_ctx* ctx, const double* x, int on_device);
int rk_steady_residual(rk_ctx* ctx, double* r, int on_device);
int rk_vjp(rk_ctx* ctx, const double* v, double* out, double* out_params, int on_device);
int rk_objective(rk_ctx* ctx, int objective, double* J, double* dJdX, double* dJdp, int on_device);
int rk_adjoint_solve(rk_ctx* ctx, int objective, int32_t max_iter, double tol, int32_t* iters_done,
                     double* rel_res, double* J, double* dJdp);
int rk_adjoint_get(rk_ctx* ctx, double* lam, int on_device);

#ifdef __cplusplus
}
#endif
#endif
