/*
 * lrbms.h - C ABI of the GB300 library for the online time step of the
 * Localized Reduced Basis Multiscale (LRBMS) method for incompressible
 * two-phase flow (Kaulmann, Flemisch, Haasdonk, Lie, Ohlberger,
 * arXiv 1405.2810).
 *
 * One online step (Algorithm 3, step 5) advances the wetting saturation s^n
 * of every listed simulation to s^{n+1}:
 *   (a) least-squares fit of the mobility coefficients theta(s^n)
 *       (Eq. leastSquaresFit) and assembly of the reduced system
 *       (c + sum_q theta_q b_q) x = e + sum_q theta_q d_q   (Eq. reducedSystem);
 *   (b) solve of that symmetric positive definite block-sparse system;
 *   (c) reconstruction of the fine P1 pressure p = sum_i x_i phi_i
 *       (Algorithm 3, step 5(b)) and of the conservative face fluxes of
 *       Definition 2 (Eq. velocityDG) with the mobility lambda(s^n);
 *   (d) explicit upwind finite-volume saturation update (Definition 3 with
 *       piecewise-constant saturation, Eq. upwind) with a CFL time step.
 * All arithmetic runs in CUDA kernels on one GPU; there is no CPU fallback.
 *
 * Conventions shared by every call
 * --------------------------------
 * Fine grid: nx x ny rectangles on [0,Lx] x [0,Ly]; cell (i,j) -> j*nx + i.
 * Faces: x-faces (normal +x) (i,j), i=0..nx, j=0..ny-1 -> j*(nx+1)+i, then
 * y-faces (normal +y) (i,j), i=0..nx-1, j=0..ny -> (nx+1)*ny + j*nx + i.
 * Every face flux is the integral of u.n over the face with n = +x or +y.
 * Boundary faces, 2*nx + 2*ny of them: left side (j = 0..ny-1), right side
 * (j), bottom side (i = 0..nx-1), top side (i).
 * Local P1 basis on a cell with centre (xc,yc): psi0 = 1,
 * psi1 = 2(x-xc)/hx, psi2 = 2(y-yc)/hy; a pressure field is three arrays
 * p0[n_cells], p1[n_cells], p2[n_cells] (structure of arrays).
 * Coarse grid (Section 4.2): Sx x Sy subdomains of (nx/Sx) x (ny/Sy) cells,
 * subdomain (I,J) -> J*Sx + I; local cell (li,lj) -> lj*(nx/Sx) + li.
 * Coarse faces: x-interfaces between (I,J) and (I+1,J), index J*(Sx-1)+I,
 * then y-interfaces between (I,J) and (I,J+1), index Sy*(Sx-1) + J*Sx + I.
 *
 * Ownership: every pointer passed in is owned by the caller, may be host or
 * device memory (the library copies with unified addressing) and may be
 * freed when the call returns. The library owns all device memory it uses;
 * it is taken from one arena allocated at lrbms_create.
 *
 * Errors: every call returns LRBMS_OK (0) or a negative lrbms_status; the
 * message of the last error is available from lrbms_last_error. No call
 * aborts, traps or prints. A simulation whose step fails (non-SPD reduced
 * matrix, non-finite state) is frozen with its status word set; the other
 * simulations continue.
 *
 * Threads: a context is used by one host thread at a time.
 */
#ifndef LRBMS_H
#define LRBMS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lrbms_ctx lrbms_ctx;

typedef enum {
  LRBMS_OK = 0,
  LRBMS_E_ARG = -1,       /* invalid argument or shape                       */
  LRBMS_E_BUDGET = -2,    /* device-memory budget or slot table exhausted    */
  LRBMS_E_CUDA = -3,      /* a CUDA runtime call failed                       */
  LRBMS_E_NOT_SPD = -4,   /* reduced matrix not positive definite (Cholesky) */
  LRBMS_E_NONFINITE = -5, /* NaN or Inf in the saturation or time step       */
  LRBMS_E_TIMEOUT = -6,   /* a bounded device-side wait gave up              */
  LRBMS_E_FORMAT = -7,    /* offline data inconsistent with the problem      */
  LRBMS_E_CFL = -8,       /* a fixed time step beyond the CFL bound: some
                             cell would see dt L_f outflow/(phi|e|) > 1 (the
                             upwind update of Definition 3 could then leave
                             [0,1]); the simulation is frozen before its
                             saturation changes                            */
  LRBMS_E_STATE = -9      /* unknown or released simulation id               */
} lrbms_status;

enum { LRBMS_FP64 = 0, LRBMS_MIXED = 1 };
enum { LRBMS_SOLVE_FP64 = 0, LRBMS_SOLVE_MIXED = 1 };
enum { LRBMS_COREY = 0, LRBMS_LINEAR = 1 };
enum { LRBMS_DT_CFL = 0, LRBMS_DT_FIXED = 1 };
enum { LRBMS_VELOCITY_STATE = 0, LRBMS_VELOCITY_FITTED = 1 };
enum { LRBMS_TRANSPORT_FV = 0, LRBMS_TRANSPORT_DG1 = 1 };

typedef struct {
  int precision;     /* LRBMS_FP64: every phase in FP64. LRBMS_MIXED: basis
                        and component streams in FP32 with FP32 accumulation;
                        fit, solve, fluxes and saturation in FP64.          */
  int max_slots;     /* maximum number of resident simulations (>= 1)       */
  size_t hbm_budget; /* bytes of device memory for simulation data; the
                        arena is allocated once, at lrbms_create           */
  void* stream;      /* cudaStream_t for all work, or NULL for a stream
                        owned by the context                                */
  int device;        /* CUDA device ordinal                                 */
  int solver;        /* reduced solve: LRBMS_SOLVE_FP64 (FP64 block Cholesky
                        every step, FP64 substitutions) or LRBMS_SOLVE_MIXED
                        (FP32 block Cholesky and substitutions; conjugate
                        gradients in FP64 preconditioned by the FP32
                        factor, warm-started from the previous steps'
                        solutions; the FP32 factor of an earlier step is
                        reused for refactor_period steps, or until a step
                        needs more than 10 passes; a reused factor that has
                        not converged after 12 passes is recomputed at once
                        and the solve repeated with FP64-residual
                        refinement; a solve whose fresh FP32 factorisation
                        meets a non-positive pivot, or whose iteration stops
                        converging, is redone in FP64)                     */
  int refine_iters;  /* FP64: most refinement steps after the first solve;
                        MIXED: most passes of a step minus one (at least
                        11). 0: default (1 for FP64, 6 for MIXED); at most
                        16. The iteration stops early once the next
                        correction, predicted from the last two, is below
                        2.5e-13 (conjugate gradients) or 1e-12 (refinement)
                        of the solution (max norms); the refinement also
                        once a correction no longer halves                 */
  int refactor_period; /* MIXED: steps one FP32 factor serves before the
                        simulation refactors (1: every step); 0: default 8.
                        The first guess of each solve is the quadratic
                        extrapolation of the last three solutions          */
  int refactor_stages; /* MIXED: steps over which each next FP32 factor is
                        built, 1..refactor_period (0: default 1, the whole
                        factorisation in one step). With R > 1 the next
                        factor is computed in the idle one of two FP32
                        buffers during the last R steps of the current
                        factor's period, about n_sub / R block rows per
                        step from that step's matrix, and serves from the
                        solve of its last stage on. No step then carries a
                        whole factorisation (lower tail latency); the
                        factor is up to R - 1 steps older (more passes).
                        A first factor, and one forced by a slow or failed
                        solve, is still computed in one step. Larger than
                        refactor_period: LRBMS_E_ARG                     */
} lrbms_config;

/* The model problem of Section 2 (Eqs. mainPressure..mainInitialData) with
 * gravity and sources set to zero, on the grids described above. */
typedef struct {
  int nx, ny, Sx, Sy;
  double Lx, Ly;
  const double* perm;    /* [nx*ny] permeability kappa (P0)                  */
  const double* poro;    /* [nx*ny] porosity phi (P0)                        */
  double eta_w, eta_o;   /* viscosities                                      */
  int relperm;           /* LRBMS_COREY (k_rw=s^2, k_ro=(1-s)^2) or LRBMS_LINEAR */
  const int8_t* bc_type; /* [2nx+2ny] 1: Dirichlet pressure p_D; 0: Neumann,
                            outward flux density v_N (0 = no flow)          */
  const double* p_D;     /* [2nx+2ny]                                        */
  const double* v_N;     /* [2nx+2ny]                                        */
  const double* s_D;     /* [2nx+2ny] saturation entering through an inflow face */
  const double* s0;      /* [nx*ny] initial saturation                       */
  double cfl;            /* CFL number of the time step (dt_mode = CFL)      */
  int dt_mode;           /* LRBMS_DT_CFL or LRBMS_DT_FIXED                   */
  double dt_fixed;       /* time step for LRBMS_DT_FIXED; a step beyond the
                            CFL bound with CFL number 1 is refused with
                            LRBMS_E_CFL (checked every step, needs Lf > 0) */
  double dt_max;         /* upper bound on the CFL step; <= 0: none          */
  int mean_weights;      /* face mean weights: 0 tau_l = a_l/(a1+a2) (as
                            printed, Section 3.1); 1 the swapped weights     */
  int velocity;          /* mobility in the face fluxes of Definition 2:
                            LRBMS_VELOCITY_STATE lambda(s^n), as Definition 2
                            and Algorithm 3 step 5 state; LRBMS_VELOCITY_FITTED
                            the fitted mobility sum_q theta_q Lambda^q that
                            the reduced pressure system uses (Section 4.4) */
  int transport;         /* saturation scheme (Definition 3): LRBMS_TRANSPORT_FV
                            piecewise constant (finite-volume upwind);
                            LRBMS_TRANSPORT_DG1 piecewise linear (P1 DG,
                            explicit Euler, Raviart-Thomas velocity of the
                            face fluxes, 3x3 Gauss points in a cell and 3 on
                            a face, CFL step divided by 3) followed by the
                            slope limiter of Section 3.4 (Eq. limiterMain).
                            The saturation penalty term is dropped in both;
                            the fit, the reduced system and the fluxes take
                            the mobility at the cell means. s0 is a cell mean
                            (slopes start at zero)                          */
} lrbms_problem;

/* Offline data of the offline/online decomposition (Section 4.4) for M
 * mobility profiles and local bases of sizes N_E. Component index q = 0
 * holds the parameter-independent part (c for the matrix, e for the right
 * hand side); q = 1..M hold b_q and d_q. */
typedef struct {
  int M;
  const int* N_E;          /* [Sx*Sy] local basis sizes, 1..32               */
  const uint8_t* prof_idx; /* [nx*ny] first profile index q (2..M) whose value
                              is lambda(1) (profiles of Algorithm 2, step 1(c)),
                              or NULL                                       */
  const double* prof;      /* [M][nx*ny] total-mobility profiles, or NULL;
                              exactly one of prof_idx and prof is given     */
  const double* Gpinv;     /* [M*M] pseudo-inverse of the profile Gram matrix
                              (normal equations of Eq. leastSquaresFit)     */
  const double* Phi;       /* per subdomain E, concatenated: [N_E][3*cells_E],
                              row k*cells_E + c = coefficient of psi_k on
                              local cell c                                  */
  const double* Dblk;      /* per subdomain E: [M+1][N_E][N_E]               */
  const double* Fblk;      /* per coarse face (E-, E+): [M+1][N_E-][N_E+]    */
  const double* rhs;       /* per subdomain E: [M+1][N_E]                    */
  double c_pen;            /* penalty scale c_f / max(eta_w, eta_o), Remark 1:
                              sigma_f = c_pen * 2 k1 k2/(k1+k2) inside,
                              c_pen * k_e on a boundary face                */
  double Lf;               /* max over [0,1] of f_w'(s) for the CFL step     */
} lrbms_offline;

/* Create a context on cfg->device with an arena of cfg->hbm_budget bytes. */
int lrbms_create(lrbms_ctx** ctx, const lrbms_config* cfg);
/* Free every device buffer and the context. */
int lrbms_destroy(lrbms_ctx* ctx);

/* Admit one simulation: validate shapes, charge the arena, copy the problem
 * and offline data to the device and set s = s0, t = 0. On success *sim_id
 * receives the slot. LRBMS_E_BUDGET if the arena or slot table is full. The
 * copies and set-up kernels run on the context's admission stream, so they
 * overlap steps in flight on the context stream; the call returns once they
 * are done. */
int lrbms_offline_load(lrbms_ctx* ctx, const lrbms_problem* prob,
                       const lrbms_offline* off, int* sim_id);
/* Release a simulation's slot and arena memory. */
int lrbms_release(lrbms_ctx* ctx, int sim_id);

/* Enqueue n_steps online steps (Algorithm 3, step 5) for the n_sims listed
 * simulations on the context stream, all simulations in each launch (one
 * captured CUDA graph per step while the list and its launch shape stay the
 * same). With status == NULL the call returns once the work is enqueued;
 * otherwise it waits for the stream and writes one lrbms_status per
 * simulation (n_steps = 0: the current statuses). */
int lrbms_step(lrbms_ctx* ctx, int n_sims, const int* sim_ids, int n_steps,
               int* status);

/* After an lrbms_step with n_steps >= 1 and status == NULL: wait for the
 * context stream and write the statuses of the first n_sims simulations of
 * that call's list (one device-to-host copy for the whole batch). Work
 * enqueued meanwhile on the admission stream (lrbms_offline_load and
 * lrbms_clone of simulations outside the batch) is not waited for, so a
 * serving loop can admit new simulations while a step runs. */
int lrbms_step_status(lrbms_ctx* ctx, int n_sims, int* status);

/* Run n_steps steps of one simulation, wait, and copy the saturation
 * [n_cells], pressure [3][n_cells] and face fluxes [n_faces] of the last step
 * into the caller's buffers (NULL buffers are skipped). */
int lrbms_run(lrbms_ctx* ctx, int sim_id, int n_steps, double* s_out,
              double* p_out, double* flux_out);

/* Wait and copy the saturation [n_cells], simulated time and the cumulative
 * water volume that left through the boundary (NULL skipped). */
int lrbms_get_state(lrbms_ctx* ctx, int sim_id, double* s, double* t,
                    double* mass_out);
/* Overwrite a simulation's saturation (host or device pointer): the cell
 * values (finite volume) or cell means (P1 DG, whose slopes are reset to 0). */
int lrbms_set_saturation(lrbms_ctx* ctx, int sim_id, const double* s);
/* Overwrite the slopes [2][n_cells] (c1 then c2, see LRBMS_FIELD_SLOPES) of a
 * simulation with the P1-DG transport; LRBMS_E_ARG for the finite-volume one. */
int lrbms_set_slopes(lrbms_ctx* ctx, int sim_id, const double* slopes);

/* Intermediate fields of the last step, for inspection and parity tests. */
enum {
  LRBMS_FIELD_THETA = 0, /* [M] fit coefficients                              */
  LRBMS_FIELD_A = 1,     /* assembled blocks: per E [N_E][N_E], then per coarse
                            face [N_E-][N_E+]                                   */
  LRBMS_FIELD_RHS = 2,   /* [N] assembled right-hand side                       */
  LRBMS_FIELD_X = 3,     /* [N] reduced solution, subdomain-major               */
  LRBMS_FIELD_P = 4,     /* [3][n_cells] reconstructed pressure                 */
  LRBMS_FIELD_FLUX = 5,  /* [n_faces] face fluxes                               */
  LRBMS_FIELD_S = 6,     /* [n_cells] saturation                                */
  LRBMS_FIELD_DT = 7,    /* [1] last time step                                  */
  LRBMS_FIELD_STATUS = 8,/* [1] int status word                                 */
  LRBMS_FIELD_SLOPES = 10, /* [2][n_cells] slopes c1, c2 of the piecewise-linear
                            saturation s = c0 + c1 psi1 + c2 psi2 (c0 is
                            LRBMS_FIELD_S); zeros for LRBMS_TRANSPORT_FV      */
  LRBMS_FIELD_PHI = 11,  /* [N][3*cells_E] the local reduced bases (FP64), in
                            the layout of lrbms_offline.Phi (Algorithm 2 step
                            4: the union of the local bases)                  */
  LRBMS_FIELD_SOLVE_INFO = 9 /* [6] int: correction passes of the last reduced
                            solve; then, counted since load: reduced solves
                            redone in FP64 after the FP32 factorisation or
                            refinement failed; FP32 factorisations; steps
                            whose reused (stale) FP32 factor did not converge
                            and was recomputed at once; substitution passes;
                            reduced solves                                      */
};
/* Wait and copy a field (bytes must equal the field's size). */
int lrbms_get_field(lrbms_ctx* ctx, int sim_id, int field, void* dst, size_t bytes);

/* Size in bytes of a field for a resident simulation (0 if unknown). */
size_t lrbms_field_bytes(lrbms_ctx* ctx, int sim_id, int field);

/* Offline phase on the GPU (Algorithm 2 with a given list of snapshot
 * parameters instead of the greedy selection, then Section 4.4): initial
 * pressure and velocity with lambda(s0), time-of-flight, threshold profiles,
 * pseudo-inverse of the profile Gram matrix, fine snapshots at the parameters
 * mu, local bases (unit function first, FP64 Gram-Schmidt in L2(E)) and the
 * projected components. Fine systems are solved with the same block
 * Cholesky as the reduced ones. */
typedef struct {
  int M;             /* number of mobility profiles, 3..16                     */
  int n_steps_T;     /* profile thresholds use T = n_steps_T * dt0, dt0 the CFL
                        step of the initial velocity                          */
  const int* N_E;    /* [Sx*Sy] local basis sizes to build                     */
  int n_snap;        /* number of snapshot parameters                          */
  const double* mu;  /* [n_snap][M] snapshot parameters (drawn by the caller)  */
  double c_pen;      /* penalty scale c_f / max(eta_w, eta_o)                  */
  int allow_fewer;   /* 0: fail with LRBMS_E_FORMAT when a subdomain's snapshots
                        give fewer than N_E independent functions; 1: keep the
                        functions obtained (smaller N_E)                       */
  int greedy;        /* 0: the local bases are the unit function and the
                        snapshots at mu, in order (Gram-Schmidt, truncated to
                        N_E); 1: Algorithm 2 step 2, greedy selection over the
                        training set mu with the true error of Section 6 in
                        the energy norm of the fine SWIP matrix at mu_bar:
                        every subdomain below its cap N_E grows by the
                        orthonormalised restriction of the worst-approximated
                        snapshot until that error is at most greedy_tol      */
  double greedy_tol; /* greedy stopping tolerance                              */
  const double* mu_bar;  /* [M] energy-norm parameter; NULL: uniform 1/M        */
  double* history;   /* greedy: the worst error of every iteration (host or
                        device, at most max_history entries), or NULL          */
  int max_history;
  int* n_history;    /* greedy: number of iterations (host), or NULL           */
  double pca_eps;    /* greedy: > 0 applies the compression of Algorithm 2 step
                        3 to the snapshots the greedy selected (at most 256):
                        per subdomain the uncentred principal components of
                        their restrictions in L2(E), the fewest modes (at most
                        N_E) whose discarded energy is at most pca_eps^2 of the
                        total, singular values at most n eps_64 sigma_1 counted
                        as 0; 0: no compression. LRBMS_E_FORMAT if a subdomain
                        keeps no mode                                          */
  const double* prof_s; /* [M][n_cells] saturations s_1..s_M (host or device), or
                        NULL. Given, the mobility profiles are Lambda^q =
                        lambda(s_q), stored dense, instead of the
                        time-of-flight thresholds of Algorithm 2 step 1(c):
                        the variant of Section 6 with high-dimensional
                        saturation snapshots (for example states advanced by
                        lrbms_fine_step). n_steps_T is then unused          */
} lrbms_build_opts;

/* Build the offline data of n_prob problems (same grids, one options entry
 * each) and admit n_copies simulations per problem. Copy r of problem p uses
 * local bases rotated by the orthogonal matrices rot[p*n_copies + r]
 * (concatenated row-major N_E x N_E per subdomain; NULL entry or NULL rot: no
 * rotation), which changes the stored bytes but not the online results.
 * sim_ids receives n_prob*n_copies slots; achieved (optional, [n_prob][Sx*Sy])
 * the local basis sizes built. Scratch device memory is taken with cudaMalloc
 * and released before return. LRBMS_E_FORMAT if the snapshots do not span the
 * requested local basis sizes and allow_fewer is 0. */
int lrbms_offline_build(lrbms_ctx* ctx, int n_prob, const lrbms_problem* probs,
                        const lrbms_build_opts* opts, int n_copies,
                        const double* const* rot, int* sim_ids, int* achieved);

/* Admit a copy of resident simulation src whose local bases are rotated by
 * the orthogonal matrices in rot (concatenated row-major N_E x N_E per
 * subdomain, host or device; NULL: an unrotated copy): Phi_E Q_E, and
 * Q_E^T (.) Q_E' for every component block and right-hand side. The online
 * results are unchanged up to round-off; the stored bytes differ. The copy
 * starts from src's current saturation, at time 0. It runs on the admission
 * stream; if src was in the last stepped batch the call first waits for the
 * context stream. Warm admission (mixed solver, rot == NULL, src never
 * stepped): the copy has src's matrix, so it starts with src's FP32 factor.
 * The first such call computes that factor once for src (fit, theta,
 * assembly and factorisation of src alone, as its own first step would);
 * later calls only copy it. The results are bitwise those of a cold start;
 * only the first step's factorisation is saved. lrbms_set_saturation on src
 * drops the precomputed factor. */
int lrbms_clone(lrbms_ctx* ctx, int src, const double* rot, int* sim_id);

/* Like lrbms_step, with the saturation exchanged with caller memory: before
 * the first step each simulation's saturation is read from s_in[i], after the
 * last step it is written to s_out[i] (n_cells doubles each; pinned host or
 * device memory, read and written by kernels through unified addressing;
 * NULL arrays skip the exchange). Waits for completion. */
int lrbms_step_io(lrbms_ctx* ctx, int n_sims, const int* sim_ids, int n_steps,
                  const double* const* s_in, double* const* s_out, int* status);

/* Phases of one step, in launch order. FIT runs only in the first step after
 * the saturation was set from outside (load, lrbms_set_saturation,
 * lrbms_step_io input); otherwise TRANSPORT has already fitted the new
 * saturation. FLUX includes the per-tile CFL bound. */
enum {
  LRBMS_PHASE_FIT = 0, LRBMS_PHASE_ASSEMBLE, LRBMS_PHASE_SOLVE, LRBMS_PHASE_RECONSTRUCT,
  LRBMS_PHASE_FLUX, LRBMS_PHASE_TRANSPORT, LRBMS_PHASE_FINALIZE,
  LRBMS_N_PHASES
};
/* Profiling of live steps: with max_steps > 0 the next max_steps steps record
 * a CUDA event before the first phase and after every phase, on the context
 * stream (max_steps = 0 turns it off). */
int lrbms_profile_start(lrbms_ctx* ctx, int max_steps);
/* Wait, then report for the recorded steps the mean time of each phase
 * (phase_ms[LRBMS_N_PHASES], milliseconds) and each step's time
 * (step_ms[max_steps]); *n_recorded receives the number of steps recorded. */
int lrbms_profile_read(lrbms_ctx* ctx, double* phase_ms, double* step_ms, int* n_recorded);

/* Solve one reduced system (c + sum_q theta_q b_q) x = rhs, already
 * assembled, without allocating anything. The paper has no counterpart: it is
 * for callers that cannot call cudaMalloc, for example a host process whose
 * device memory belongs to another allocator, or a time-critical loop in
 * which the synchronisation and possible failure of an allocation are not
 * allowed. No context is needed and nothing is allocated on the host or the
 * device; all working memory (factor panels, diagonal inverses, work vectors,
 * offset tables, the substitutions' copy schedule) is a fixed 32 MiB array in
 * device memory that every GPU
 * loading the library holds until the process exits.
 *   Sx, Sy  coarse grid; N_E [Sx*Sy] local basis sizes (host memory, 1..32)
 *   A       device, assembled blocks in the layout of LRBMS_FIELD_A
 *           (per subdomain [N_E][N_E], then per coarse face [N_E-][N_E+])
 *   rhs     device, [N]; x: device, [N] output
 *   solver  LRBMS_SOLVE_FP64 or LRBMS_SOLVE_MIXED; refine_iters as in
 *           lrbms_config (0: default)
 *   stream  cudaStream_t (NULL: the legacy default stream)
 * A, rhs and x must be device (or managed) memory of exactly the sizes the
 * basis sizes give; pointers the runtime does not report as device memory are
 * refused with LRBMS_E_ARG (the sizes themselves cannot be checked here).
 * Returns LRBMS_E_BUDGET if the system needs more than the 32 MiB array or
 * more shared memory than one CTA has, LRBMS_E_NOT_SPD if a pivot is not
 * positive, LRBMS_E_NONFINITE if the solution holds a NaN or Inf (for
 * example from a non-finite right-hand side), LRBMS_E_ARG on bad arguments.
 * An error left pending by the caller's earlier CUDA work is cleared on entry
 * and not reported by this call. Every call copies the basis sizes from host
 * memory and waits for the stream. The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current;
 * make that first call before any stream capture. Every call uses the same
 * array: calls that overlap on the GPU (other streams, other host threads)
 * race and must be serialised by the caller. */
int lrbms_solve_noalloc(int Sx, int Sy, const int* N_E, const double* A, const double* rhs,
                        double* x, int solver, int refine_iters, void* stream);

/* Advance the listed resident simulations by n_steps steps of the
 * high-dimensional scheme instead of the reduced one (Algorithm 1, with the
 * piecewise-constant saturation of Definition 3): per step the fine SWIP-DG
 * pressure of Definition 1 with the mobility lambda(s^n) (Eqs. swipBilP,
 * penaltyParam; 3 unknowns per cell, FP64 assembly and an FP64 envelope block
 * Cholesky with one refinement step, one CTA per simulation), then the face
 * fluxes of Definition 2, the CFL step and the upwind update exactly as in
 * lrbms_step. The reduced offline data of the simulations are not used; the
 * simulations keep their state, so reduced and fine steps can alternate.
 * All listed simulations must share the fine grid (nx, ny) and use
 * LRBMS_VELOCITY_STATE (LRBMS_E_ARG otherwise). Scratch device memory for the
 * fine factors (about 8 * 3 nx ny * 3 (nx + 1) bytes per simulation) is taken
 * with cudaMalloc and released before return. Waits for completion; status
 * (optional) receives one lrbms_status per simulation (LRBMS_E_NOT_SPD for a
 * fine system that is not positive definite). */
int lrbms_fine_step(lrbms_ctx* ctx, int n_sims, const int* sim_ids, int n_steps, int* status);

/* CTA sizes the autotuner picked for the assembly and reconstruction kernels
 * of the shape class of these simulations (largest basis size in classes of
 * 8, cells per subdomain, component precision). The first lrbms_step of a new
 * class times each candidate on the live data and keeps the fastest; the
 * results do not depend on the choice. LRBMS_E_STATE before that step. */
int lrbms_tuned_threads(lrbms_ctx* ctx, int n_sims, const int* sim_ids, int* assemble, int* reconstruct);

/* Test hook for the failure detection of the bounded device-side waits; the
 * paper has no counterpart. The next reduced solve of sim_id withholds the
 * last bulk copy of its forward/backward substitution (every earlier copy has
 * been awaited by then, so nothing is left in flight); the wait for it gives
 * up after its limit (about 2 s), and the simulation stops with
 * LRBMS_E_TIMEOUT while the others in the launch continue unchanged. The hook
 * fires once. */
int lrbms_test_withhold_copy(lrbms_ctx* ctx, int sim_id);

/* Test hook (host only, no device work; the paper has no counterpart): the
 * mixed solver's factorisation plan for one step of a simulation with n_sub
 * block rows, the given refactor period and stages (1 <= stages <= period)
 * and solver state info[12] (the kernels' internal counters: [6] factor age,
 * [7] forced refactorisation, [8] current FP32 buffer). out[5] receives the
 * block rows [out[0], out[1]) that the step's factor kernel computes, the
 * buffer it writes (out[2]), whether it is a whole factorisation (out[3])
 * and whether it completes a staged build (out[4]). LRBMS_E_ARG on invalid
 * sizes. */
int lrbms_test_factor_plan(int n_sub, int refactor_period, int refactor_stages, const int* info, int* out);

/* Wait for all enqueued work. */
int lrbms_sync(lrbms_ctx* ctx);

/* Device bytes in use by resident simulations, and the arena size. */
int lrbms_memory(lrbms_ctx* ctx, size_t* used, size_t* capacity);

/* Number of kernel launches enqueued by this context so far. */
long long lrbms_launch_count(const lrbms_ctx* ctx);

const char* lrbms_last_error(const lrbms_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* LRBMS_H */
