/*
 * mofem.h -- C ABI of libmofem: matrix-oriented FEM (MO-FEM) and the
 * matrix-oriented preconditioned conjugate gradient (MO-PCG) on one GB300 GPU.
 *
 * Method: Frittelli & Sgura, "Matrix-oriented FEM formulation for stationary
 * and time-dependent PDEs on x-normal domains" (arXiv 2109.01173).
 *
 * Problem (Sec. 5, Eq. laplace_equation_xnormal):  -Lap u + gamma u = f on the
 * x-normal domain {0 <= x <= 1, g1(x) <= y <= g2(x)}, with homogeneous Dirichlet
 * (gamma >= 0) or Neumann (gamma > 0) boundary conditions, discretised by
 * degree-k tensor Lagrange elements (k = 1..4) or lumped P1 (k = 0) on the
 * curvilinear mesh mapped from the unit square (Sec. 2.2, Eq. transformation,
 * generalised to two profiles).  The unknown is a q x q matrix U[a][b]
 * (a = node along x, b = node along the mapped y direction), q = n - 2 for
 * Dirichlet and q = n for Neumann (Eq. variable_dimension), n = nodes per
 * direction.  The discrete system is the multiterm Sylvester equation
 *     L(U) = sum_i S_i U T_i^T = B          (Sec. 5, Eq. laplace_cap-shaped-domain_sylvester)
 * with banded 1D factors S_i, T_i (Sec. 3.2, Eq. kronecker_mass_distorted).
 *
 * Conventions (all entry points):
 *  - Matrix arguments are DEVICE pointers owned by the caller, row-major, with
 *    leading dimension `ld` (elements).  For a batched handle the instances are
 *    stored back to back with a batch stride of `ld * rows` elements.  The
 *    library never frees caller memory.
 *  - The handle owns every buffer it allocates (1D tables, eigenvector
 *    matrices, workspaces) and frees them in mofem_destroy.
 *  - Calls are stream-ordered on `stream`.  Argument errors are returned
 *    synchronously.  mofem_pcg_solve and mofem_imex_step synchronise `stream`
 *    before they return (their outer refinement loop reads a status word).
 *  - No exception crosses the ABI; a handle must not be used from two host
 *    threads at once.
 */
#ifndef MOFEM_H
#define MOFEM_H

#include <stddef.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MOFEM_OK = 0,
    MOFEM_ERR_INVALID_ARG = 1,   /* bad size, degree, profile (h <= 0), singular Neumann with gamma = 0 */
    MOFEM_ERR_CUDA = 2,          /* a CUDA runtime / library call failed */
    MOFEM_ERR_EIG = 3,           /* the generalized eigensolver reported failure */
    MOFEM_ERR_NONFINITE = 4,     /* NaN or Inf in an input or a recurrence scalar */
    MOFEM_ERR_BREAKDOWN = 5,     /* <Q, L(Q)> <= 0 in PCG */
    MOFEM_ERR_NOT_CONVERGED = 6, /* max_iter reached; the iterate is kept */
    MOFEM_ERR_TIMEOUT = 7,       /* a bounded device-side wait gave up */
    MOFEM_ERR_OOM = 8,           /* device allocation failed */
    MOFEM_ERR_UNSUPPORTED = 9    /* valid request the library does not implement */
} mofem_status;

typedef enum { MOFEM_BC_DIRICHLET = 0, MOFEM_BC_NEUMANN = 1 } mofem_bc;

/* Arithmetic of the iteration.  FP64: every step in double (preconditioner
 * GEMMs through cuBLAS DGEMM).  MIXED_*: operator apply and vectors in FP32,
 * preconditioner GEMMs on tcgen05 tensor cores with FP32 accumulation and
 * operands in TF32, BF16 or FP16 (FP16: the residual operand is scaled per
 * instance to unit RMS and the scale undone on output), CG scalars and
 * cross-thread dot-product sums in FP64, and FP64 true-residual iterative
 * refinement around the inner FP32 solve. */
typedef enum { MOFEM_FP64 = 0, MOFEM_MIXED_TF32 = 1, MOFEM_MIXED_BF16 = 2, MOFEM_MIXED_FP16 = 3 } mofem_precision;

/* Preconditioner of MO-PCG.  AVERAGED / DOMINANT: the two-term Sylvester
 * preconditioner E1 Z F1^T + E2 Z F2^T = R (E1 = K_s[h] + gamma M_s[h], F1 = M_t,
 * F2 = K_t, E2 = M_s[e2] with e2 the t-average of H^_tt or its t-free part).
 * The others are the paper's single-term preconditioners P(Z) = E Z F^T, applied by
 * the same reduced approach with standard eigenpairs of E and F and the divisor
 * lambda_a mu_b:
 *  PRODUCT   (Sec. 5, Eq. vector_preconditioner): E = K_s[h], F = K_t + K_t[t^2]
 *            (B1 U (A + B2) in the paper's orientation); Dirichlet only.
 *  PARABOLIC (Sec. 6, Eqs. semilinear_heat_equation_fully_discrete_P and its lumped
 *            form _P_lumped, k = 0): the IMEX-step preconditioner
 *            (M3 + d_u tau B1)^-1 U (M + d_u tau (A + B2))^-1, i.e. for a handle set up
 *            with gamma = 1/(d_u tau) (the step scaled by 1/(d_u tau)):
 *            E = K_s[h] + gamma M_s[h], F = M_t + (K_t + K_t[t^2]) / gamma.  Needs
 *            gamma > 0, the same in every instance (F and Q2 are shared); both BCs.
 *  AUA       (Sec. 5.1, Eq. precSquare): E = K_s[h], F = K_t, which on the unit
 *            square is A U A with A the 1D stiffness matrix; Dirichlet only. */
typedef enum {
    MOFEM_PENCIL_AVERAGED = 0,
    MOFEM_PENCIL_DOMINANT = 1,
    MOFEM_PENCIL_PRODUCT = 2,
    MOFEM_PENCIL_PARABOLIC = 3,
    MOFEM_PENCIL_AUA = 4
} mofem_pencil;

/* Domain profile y = g(x) on [0, 1]: host callbacks for g and g', called during
 * setup only (at the quadrature points). */
typedef struct {
    double (*g)(double x, void* ctx);
    double (*dg)(double x, void* ctx);
    void* ctx;
} mofem_profile;

typedef struct {
    int quad_points;       /* Gauss-Legendre points per element for P_k; 0 -> k + 3 */
    mofem_pencil pencil;   /* default MOFEM_PENCIL_AVERAGED */
    int max_outer;         /* refinement steps of the mixed form; 0 -> 20 */
    double inner_rtol;     /* reduction asked of the first inner FP32 solve; later ones aim at
                              rtol, no deeper than inner_rtol / 10.  0 -> 1e-5 */
    int flags;             /* MOFEM_FLAG_* */
} mofem_opts;

#define MOFEM_FLAG_HOST_LOOP 1   /* drive the inner iteration from the host (one graph launch
                                    per iteration) instead of a device-side conditional loop */
#define MOFEM_FLAG_FIXED_ITERS 2 /* run exactly max_iter inner iterations (timing runs) */
#define MOFEM_FLAG_TRUE_RESIDUAL 4 /* mixed forms: recompute B - L(U) in FP64 after every refinement
                                      step (default: update R -= L(d) in double-float arithmetic) */

typedef struct {
    int status;            /* mofem_status of the whole (batched) solve */
    int iterations;        /* total inner PCG iterations (max over instances) */
    int outer_steps;       /* FP64 refinement steps (mixed form); 1 for FP64 */
    int batch;
    double rel_residual;   /* max over instances of ||B - L(U)||_F / ||B||_F (IMEX rule: / ||R_0||_F) of
                              the returned U: the FP64 form's recomputed residual; the mixed forms'
                              residual carried by the double-float updates (exact up to their
                              evaluation error, ~2^-48 q of ||B||), or recomputed in FP64 where
                              mofem_pcg_solve says so */
    double ms_total;       /* device time of the solve (CUDA events) */
    long long kernel_launches; /* libmofem kernels launched by the solve (graph nodes included) */
} mofem_solve_info;

typedef struct mofem_ctx* mofem_handle;

/* Setup (Sec. 3, Sec. 4; paper Eqs. newmatrix_1..7, kronecker_mass_distorted,
 * diagonalisation_1).  Builds the banded 1D factors of the operator, the RHS
 * mass factors, and the generalized eigendecompositions (FP64, on the GPU)
 *   E1 Q1 = E2 Q1 diag(lambda),  Q1^T E2 Q1 = I,
 *   F2 Q2 = F1 Q2 diag(mu),      Q2^T F1 Q2 = I,
 * of the preconditioner pencils E1 = K_s[h] + gamma M_s[h], F1 = M_t,
 * E2 = M_s[e2], F2 = K_t (e2 per mofem_opts.pencil).
 * k: 1..4 (P_k) or 0 (lumped P1).  n_nodes: nodes per direction, (n-1) % max(k,1) == 0.
 * Returns MOFEM_ERR_INVALID_ARG if h = g2 - g1 <= 0 at a quadrature point, if
 * k or n is invalid, or for Neumann with gamma <= 0 (singular, Sec. 4).
 * opts may be NULL (defaults).  *out receives the handle. */
mofem_status mofem_setup(const mofem_profile* g1, const mofem_profile* g2, int k, int n_nodes,
                         double gamma, mofem_bc bc, const mofem_opts* opts,
                         cudaStream_t stream, mofem_handle* out);

/* Batched setup: `batch` independent instances sharing k, n_nodes and bc, each
 * with its own profiles g1[i], g2[i] and gamma[i].  The t-direction factors and
 * Q2 are shared; Q1, lambda and the s-direction factors are per instance. */
mofem_status mofem_setup_batched(int batch, const mofem_profile* g1, const mofem_profile* g2,
                                 int k, int n_nodes, const double* gamma, mofem_bc bc,
                                 const mofem_opts* opts, cudaStream_t stream, mofem_handle* out);

/* Dimensions of a handle (any pointer may be NULL). */
mofem_status mofem_get_dims(mofem_handle h, int* batch, int* n_nodes, int* q, int* n_terms);

/* Operator apply Y = L(X) = sum_i S_i X T_i^T for every instance (Sec. 5,
 * operator L~; Eq. laplace_cap-shaped-domain_sylvester).  X, Y: q x q per
 * instance, leading dimension ld >= q, batch stride ld*q.  FP64 -> double
 * arrays; MIXED_* -> float arrays (FP32 arithmetic).  X and Y must not overlap. */
mofem_status mofem_apply(mofem_handle h, const void* X, void* Y, int ld, mofem_precision prec,
                         cudaStream_t stream);

/* Right-hand side B = M_s[h]_(int,all) F M_t_(int,all)^T (Sec. 5, operator R~):
 * the mass matrix applied to the nodal values F (n x n per instance, ld = n,
 * boundary nodes included).  B: q x q, ld_b >= q.  FP64. */
mofem_status mofem_rhs(mofem_handle h, const double* F, double* B, int ld_b, cudaStream_t stream);

/* Preconditioner Z = P^{-1}(R): the solution of E1 Z F1^T + E2 Z F2^T = R by the
 * reduced approach (Sec. 4, Eq. reduced_formula_for_u):
 *   Z = Q1 ((Q1^T R Q2) ./ (lambda_a + mu_b)) Q2^T.
 * FP64 -> double arrays, four DGEMMs.  MIXED_TF32 / MIXED_BF16 / MIXED_FP16 ->
 * float arrays, four tcgen05 GEMMs with operands rounded to TF32 / BF16 / FP16
 * and FP32 accumulation. */
mofem_status mofem_precond(mofem_handle h, const void* R, void* Z, int ld, mofem_precision prec,
                           cudaStream_t stream);

/* One search-direction step of MO-PCG (Sec. 5, the PCG iteration of Eq.
 * laplace_xnormal_pcg_iteration), by the fused kernel the solver launches every
 * iteration: for each instance i
 *   Q = Z + beta[i] Q_prev,  LQ = L(Q),  alpha[i] = rz[i] / <Q, L(Q)>_F.
 * Z, Q_prev, Q, LQ: device arrays of q x q per instance, leading dimension ld,
 * batch stride ld*q; FP64 -> double arrays, MIXED_* -> float arrays (FP32
 * arithmetic, the inner-solve operator).  Base pointers 16-byte aligned and
 * ld*element size a multiple of 16 bytes; columns q..ld-1 of Q and LQ receive
 * zeros.  Q must not overlap Z or Q_prev.  beta, rz, alpha: host arrays of
 * `batch` doubles.  Synchronises `stream` (alpha is copied back).  Returns
 * MOFEM_ERR_BREAKDOWN (alpha[i] = 0) if <Q, L(Q)> <= 0 for some instance. */
mofem_status mofem_pcg_direction(mofem_handle h, const void* Z, const void* Q_prev, const double* beta,
                                 const double* rz, void* Q, void* LQ, int ld, double* alpha,
                                 mofem_precision prec, cudaStream_t stream);

/* Solve L(U) = B with B = mofem_rhs(F) for every instance by MO-PCG (Sec. 5,
 * Eqs. laplace_xnormal_pcg, laplace_xnormal_pcg_iteration with the standard PCG
 * recurrences) until ||B - L(U)||_F <= rtol ||B||_F, checked on the FP64 true
 * residual.  F: n x n per instance (ld n), FP64.  U: q x q per instance (ld q),
 * FP64, in: initial guess, out: solution.  MIXED_*: flexible PCG in FP32 inside
 * FP64 iterative refinement; after each step the residual is updated (R -= L(d -
 * err), double-float arithmetic, err the exact rounding of the FP64 iterate's
 * update) rather than recomputed, when rtol ||ref|| lies above max(1e-11, 2 u q^2 /
 * pi^2) ||B|| (u = 2^-53; twice the evaluation noise of an FP64 residual of this
 * operator).  The step from a zero guess, of the size of U, takes the difference
 * form with exact row sums and input differences (P1 and P2, or an FP64
 * recomputation for the other degrees); MOFEM_FLAG_TRUE_RESIDUAL recomputes the
 * residual in FP64 after every step.  max_iter bounds the inner iterations of each
 * refinement step (FP64: of the whole solve).  Synchronises `stream`.
 * info may be NULL. */
mofem_status mofem_pcg_solve(mofem_handle h, const double* F, double* U, double rtol, int max_iter,
                             mofem_precision prec, mofem_solve_info* info, cudaStream_t stream);

/* One IMEX Euler step of u_t - d_u Lap u = f (Sec. 6, Eqs.
 * semilinear_heat_equation_fully_discrete_sylvester_pk and _R_pk): solves
 * (M~ + d_u tau A~) U_np1 = M~ (U_n + tau F_n).  The handle must have been set up
 * with gamma = 1 / (d_u tau) (the step is the elliptic solve scaled by d_u tau).
 * U_n, U_np1: q x q (ld q) per instance, FP64; F_n: n x n nodal f(U_n) (ld n),
 * FP64 (boundary entries of U_n are zero under Dirichlet).  Initial guess U_n;
 * stops when ||R_s||_F <= tau ||R_0||_F (Sec. 6 stopping rule).  Synchronises. */
mofem_status mofem_imex_step(mofem_handle h, double d_u, double tau, const double* U_n,
                             const double* F_n, double* U_np1, mofem_precision prec,
                             mofem_solve_info* info, cudaStream_t stream);

/* mofem_imex_step with an explicit stopping rule: rtol > 0 stops at
 * ||B - (M~ + d_u tau A~) U_np1||_F <= rtol ||B||_F on the FP64 true residual
 * (B = M~ (U_n + tau F_n)), as the elliptic solve does; rtol = 0 is the paper's
 * rule of mofem_imex_step.  Tight tolerances make the step a smooth function of
 * its inputs (finite-difference and adjoint checks of a time integration). */
mofem_status mofem_imex_step_tol(mofem_handle h, double d_u, double tau, const double* U_n,
                                 const double* F_n, double* U_np1, double rtol, mofem_precision prec,
                                 mofem_solve_info* info, cudaStream_t stream);

/* One backward step of the discrete adjoint of IMEX Euler with f = 0 (no
 * counterpart in the paper, which does not differentiate; derived from Sec. 6's
 * step S U_np1 = M~ U_n with S = M~ + d_u tau A~ symmetric):
 *   Y = S^{-1} Lam_np1   (the same MO-PCG solve, ||Lam_np1 - S Y|| <= rtol ||Lam_np1||),
 *   Lam_n = M~ Y,
 *   dd_u[i] = -tau <Y, A~ U_np1>_F   (this step's contribution to dJ/dd_u).
 * For a loss J(U_N) start from Lam_N = dJ/dU_N and go n = N-1 .. 0 with U_np1 the
 * forward state after step n; Lam_0 = dJ/dU_0.  Lam_np1, U_np1, Lam_n: q x q per
 * instance (ld q), FP64, device; Lam_n must not alias Lam_np1.  Y: q x q per
 * instance (ld q), FP64, device, in: initial guess of the solve, out: S^{-1} Lam_np1;
 * NULL starts from zero in a library buffer.  Passing the previous step's Y warm-
 * starts the solve (successive adjoint solutions differ by O(d_u tau)).  dd_u: host
 * array of `batch` doubles.  The handle must have gamma = 1/(d_u tau).  Synchronises. */
mofem_status mofem_imex_adjoint_step(mofem_handle h, double d_u, double tau, const double* Lam_np1,
                                     const double* U_np1, double* Lam_n, double* Y, double* dd_u, double rtol,
                                     mofem_precision prec, mofem_solve_info* info, cudaStream_t stream);

/* One IMEX Euler step of u_t - d_u Lap u = f - r u with a nodal source f and a linear
 * reaction -r u, both explicit as Sec. 6 treats the reaction term (Eqs.
 * semilinear_heat_equation_fully_discrete_sylvester_pk and _R_pk with f(u) = f - r u):
 *   (M~ + d_u tau A~) U_np1 = (1 - tau r) M~ U_n + tau M~_all F,
 * M~_all F = M_s[h]_(int,all) F M_t_(int,all)^T.  F: n x n nodal per instance (ld n),
 * FP64 device, constant in time; r: host scalar (r = 0: mofem_imex_step_tol).  The handle
 * must have gamma = 1/(d_u tau).  Layouts and the stopping rule as mofem_imex_step_tol. */
mofem_status mofem_imex_step_src(mofem_handle h, double d_u, double tau, double r, const double* U_n,
                                 const double* F, double* U_np1, double rtol, mofem_precision prec,
                                 mofem_solve_info* info, cudaStream_t stream);

/* One backward step of the discrete adjoint of mofem_imex_step_src (no counterpart in
 * the paper, which does not differentiate; derived from the step above by
 * differentiating it in U_n, F, r and d_u):
 *   Y = S^{-1} Lam_np1   (S = M~ + d_u tau A~ symmetric; the same MO-PCG solve),
 *   Lam_n = (1 - tau r) M~ Y,
 *   dF += tau M~_all^T Y = tau M_s[h] pad(Y) M_t^T   (n x n nodal, accumulated; pad puts
 *                                                    zeros on Dirichlet boundary nodes),
 *   dr[i] = -tau <Y, M~ U_n>_F,   dd_u[i] = -tau <Y, A~ U_np1>_F.
 * Summed over the steps n = N-1 .. 0 these give dJ/dF, dJ/dr and dJ/dd_u of a loss
 * J(U_N), and Lam_0 = dJ/dU_0.  U_n, U_np1: the forward states before and after step n.
 * dF (device, may be NULL), dr and dd_u (host arrays of `batch` doubles; dr may be
 * NULL, then U_n may be NULL).  Y as in mofem_imex_adjoint_step.  Synchronises. */
mofem_status mofem_imex_adjoint_step_src(mofem_handle h, double d_u, double tau, double r, const double* Lam_np1,
                                         const double* U_n, const double* U_np1, double* Lam_n, double* Y,
                                         double* dF, double* dd_u, double* dr, double rtol, mofem_precision prec,
                                         mofem_solve_info* info, cudaStream_t stream);

/* One IMEX Euler step of a batch of reaction-diffusion species (Sec. 6 applied
 * to each species of a system such as Sec. 7's): instance i solves
 *   (M~ + d_i tau A~) U_np1 = M~ (U_n + tau F_n),  d_i = 1/(gamma_i tau),
 * with gamma_i the handle's value for that instance (so species with different
 * diffusion coefficients share one batched solve).  Layouts and stopping rule as
 * mofem_imex_step_tol (rtol = 0: the paper's ||R_s|| <= tau ||R_0||). */
mofem_status mofem_rds_step(mofem_handle h, double tau, const double* U_n, const double* F_n, double* U_np1,
                            double rtol, mofem_precision prec, mofem_solve_info* info, cudaStream_t stream);

/* Parameters of the DIB kinetics (Sec. 7, Eqs. dib_kinetics_f, dib_kinetics_g;
 * Eq. dib_parameters_mixed and the per-domain A2, B, C of Sec. 7.1-7.2). */
typedef struct {
    double alpha, gamma, A1, A2, B, C, D, k2, k3, d_theta;
} mofem_dib_params;

/* f = rho f(eta, theta), g = rho g(eta, theta) elementwise over `count` FP64
 * device values (Sec. 7, Eqs. dib_kinetics_f, dib_kinetics_g). */
mofem_status mofem_dib_kinetics(const mofem_dib_params* p, double rho, const double* eta, const double* theta,
                                double* f, double* g, long long count, cudaStream_t stream);

/* Homogeneous equilibrium of the DIB kinetics, f(eta, theta) = g(eta, theta) = 0,
 * by Newton's method from (0, 1/2) on the host.  The paper states (0, 0.5) as the
 * equilibrium for its printed parameters, which holds only for C = 4; for other C
 * this returns the actual zero (e.g. (-0.2852, 0.4670) for the cap parameters).
 * Returns MOFEM_ERR_NONFINITE if Newton breaks down. */
mofem_status mofem_dib_equilibrium(const mofem_dib_params* p, double* eta, double* theta);

/* n_steps of IMEX Euler for the DIB model (Sec. 7, Eq. dib_model) with zero
 * Neumann data: reaction explicit (mofem_dib_kinetics), diffusion implicit, both
 * species in one batched MO-PCG solve per step.  The handle must be a Neumann
 * handle with batch 2 and gamma = {1/tau, 1/(d_theta tau)} (eta, theta).
 * U: [eta; theta], q x q each (ld q), FP64 device, in: initial data, out: state
 * after n_steps.  rtol as mofem_rds_step.  incr: host array of n_steps doubles
 * receiving ||eta_{k+1} - eta_k||_F (the paper's increment plot), or NULL.
 * info accumulates iterations over the run.  Synchronises `stream`. */
mofem_status mofem_dib_run(mofem_handle h, const mofem_dib_params* p, double rho, double tau, int n_steps,
                           double* U, double rtol, mofem_precision prec, double* incr, mofem_solve_info* info,
                           cudaStream_t stream);

/* ---- heterogeneous batches ------------------------------------------------
 * Many independent elliptic problems of different (k, n, bc, profiles, gamma)
 * solved together: problems of equal (k, n, bc) form one batched handle (as
 * mofem_setup_batched).  Two ways to run the groups:
 *  - lockstep (the default for the mixed forms): every group's inner MO-PCG runs in
 *    one CUDA graph whose conditional loop body holds, per iteration, each group's
 *    operator apply and update (side by side, one graph branch per group) and ONE
 *    persistent tensor-core launch with the preconditioner GEMMs of all groups (any
 *    q); the refinement steps are taken together;
 *  - apart: each group one batched solve on its own stream from a host thread, a
 *    chosen number of groups in flight (the FP64 form always runs this way).
 * No counterpart in the paper (it solves one problem at a time); the arithmetic per
 * problem is that of mofem_pcg_solve, and both ways give the same bits. */
typedef struct {
    mofem_profile g1, g2;   /* host callbacks, used during setup only */
    int k, n_nodes;
    double gamma;
    mofem_bc bc;
} mofem_problem;

typedef struct mofem_group_ctx* mofem_group;

/* Grouping of `count` problems without touching the GPU: *n_groups receives the
 * number of (k, n, bc) groups, group_of[i] (may be NULL) the group of problem i;
 * groups are ordered by decreasing work (n^3 times size). */
mofem_status mofem_group_layout(int count, const mofem_problem* problems, int* n_groups, int* group_of);

/* Set up every group (validation and errors as mofem_setup_batched). */
mofem_status mofem_group_setup(int count, const mofem_problem* problems, const mofem_opts* opts,
                               mofem_group* out);

/* Solve all problems: F[i] nodal n_i x n_i, U[i] q_i x q_i (in: initial guess,
 * out: solution), FP64 device pointers, as mofem_pcg_solve.  infos (may be NULL):
 * `count` records, each the info of the problem's group.  Work starts after prior
 * work on `stream`; returns when all groups are done.  Returns the first error
 * other than MOFEM_ERR_NOT_CONVERGED, else that, else MOFEM_OK. */
mofem_status mofem_group_solve(mofem_group g, const double* const* F, double* const* U, double rtol,
                               int max_iter, mofem_precision prec, mofem_solve_info* infos, cudaStream_t stream);

/* Run-time tuning of how the groups run: one warm-up solve of each way, then one
 * timed solve per candidate (lockstep for the mixed forms, with the operator-apply
 * tiles one wave of CTAs high or half of that; apart with 1, 2, 4, 8, 16 or all
 * groups in flight), each from the caller's initial guesses; the fastest is kept for
 * later solves and written to *chosen (may be NULL): -1 lockstep, else the number of
 * groups in flight (mofem_group_get_tuning also reports the tile height).  U holds
 * the caller's initial guesses again on return. */
mofem_status mofem_group_autotune(mofem_group g, const double* const* F, double* const* U, double rtol,
                                  int max_iter, mofem_precision prec, int* chosen);

/* Choose how later solves run: -1 lockstep (the default), 0 apart with all groups in
 * flight, m > 0 apart with m groups in flight. */
mofem_status mofem_group_set_mode(mofem_group g, int mode);

/* The way later solves run (as mofem_group_set_mode) and the operator-apply tile height
 * the autotuner chose: rows per CTA of one wave of resident CTAs divided by
 * *apply_tile_div (1 or 2).  Either pointer may be NULL. */
mofem_status mofem_group_get_tuning(mofem_group g, int* mode, int* apply_tile_div);

mofem_status mofem_group_destroy(mofem_group g);

/* Benchmark hook (no counterpart in the paper): launch one hot kernel `reps`
 * times on the handle's internal buffers, asynchronously on `stream`, so that
 * a caller can time it with events on that stream.  kernel:
 *   0 = FP32 operator apply with the fused search-direction update (PCG form),
 *   1..4 = preconditioner GEMM G1..G4 (prec MIXED_TF32, MIXED_BF16 or MIXED_FP16),
 *   5 = FP32 PCG update of an even iteration (R, FP16 copy of R, partial sums;
 *       the correction term alpha Q is deferred),
 *   6 = FP64 operator apply (true residual form),
 *   7 = FP32 PCG update of an odd iteration (R, FP16 copy, and the correction
 *       U += alpha_prev Q_prev + alpha Q in double-float),
 *   8 = double-float residual update R64 -= L(d) of a refinement step
 *       (MOFEM_ERR_UNSUPPORTED for forms it does not serve),
 *   9 = the preconditioner's four GEMMs as the solver runs them, one chained
 *       launch (prec MIXED_TF32, MIXED_BF16 or MIXED_FP16),
 *  10 = the residual update of 8 in difference form (the step from zero;
 *       MOFEM_ERR_UNSUPPORTED for forms it does not serve),
 *  11 = the FP64 form's preconditioner (four cuBLAS DGEMMs per instance and the
 *       Hadamard division; prec ignored).
 * The buffers' contents are whatever the last solve left (timing only). */
mofem_status mofem_bench_kernel(mofem_handle h, int kernel, mofem_precision prec, int reps,
                                cudaStream_t stream);

/* Preconditioner without device allocation.  No counterpart in the paper: an
 * interface for callers that cannot allocate device memory where they apply
 * the preconditioner (code that must not trigger the implicit device
 * synchronisation of cudaMalloc/cudaFree in a latency-critical loop, or that
 * runs under a memory budget enforced by its own allocator).
 * Computes the same Z = P^{-1}(R) as mofem_precond(MOFEM_MIXED_BF16): float R
 * and Z, q x q per instance, leading dimension ld >= q, batch stride ld*q.
 * All temporaries (BF16 copies of Q1, Q1^T, Q2, Q2^T and R, and the three GEMM
 * intermediates) live in one static device array of 8 x 2^18 BF16 elements
 * (4 MiB), held by every GPU that loads the library until the process exits.
 * Limit: batch * q * round_up(q, 64) <= 262144 (e.g. one instance with
 * q <= 512); larger handles get MOFEM_ERR_INVALID_ARG (see mofem_last_error).
 * The first call on a device looks up the array's device address; with lazy
 * module loading (the CUDA default) that first call may also load this part of
 * the library, which allocates the 4 MiB array and may synchronise the device.
 * Make one warm-up call on each device before the latency-critical loop and
 * before any stream capture; later calls allocate nothing.  All calls share the
 * array and it keeps the last call's contents: calls that overlap on the GPU race
 * and must be serialised by the caller. */
mofem_status mofem_precond_noalloc(mofem_handle h, const float* R, float* Z, int ld, cudaStream_t stream);

/* Copy of the preconditioner's eigen data computed at setup (Sec. 4, Eq.
 * diagonalisation_1; the pencils of mofem_setup, or the single-term factors of
 * mofem_pencil): Q1 [batch][q][q] (row-major, column i = eigenvector i of instance
 * b's s-pencil), Q2 [q][q] (shared t-pencil), lambda [batch][q] and mu [q], all FP64
 * DEVICE arrays owned by the caller with leading dimension q; any pointer may be
 * NULL.  The preconditioner is Z = Q1 ((Q1^T R Q2) ./ D) Q2^T with D_ab = lambda_a +
 * mu_b, or lambda_a mu_b for the single-term pencils (*divisor_product = 1; may be
 * NULL).  Stream-ordered on `stream`; no synchronisation. */
mofem_status mofem_get_eigen(mofem_handle h, double* Q1, double* Q2, double* lambda, double* mu,
                             int* divisor_product, cudaStream_t stream);

/* Release every buffer the handle owns. */
mofem_status mofem_destroy(mofem_handle h);

/* Human-readable name of a status code (static storage). */
const char* mofem_status_string(mofem_status s);

/* Text of the last error recorded on this host thread (static storage, "" if none). */
const char* mofem_last_error(void);

/* Host-only copy of the setup tables of one instance, computed exactly as
 * mofem_setup computes them but without touching the GPU (for checking the
 * assembly on machines without one).  Banded tables are diagonal-major:
 * tab[term][j][r] = M_term[r][r + off + j - K], K = max(k,1), j = 0..2K,
 * rows r = 0..q-1 of the trimmed matrix.
 *   S, T: [n_terms][2K+1][q] (n_terms <= 8; 5 when g1' = 0 at every quadrature
 *         point, else 8, in the order of the eight-term expansion: mass/stiffness,
 *         M[(1+g1'^2)/h] (x) K_t, [M[2g1'h'/h] (x) K_t[t]], M[h'^2/h] (x) K_t[t^2],
 *         [-G[g1'] (x) C_t^T, -G[g1']^T (x) C_t], -G[h'] (x) C_t[t]^T, -G[h']^T (x) C_t[t]);
 *   Srh, Trh: [2K+1][q], the RHS mass factors (rows trimmed, columns = all n nodes).
 * Any output pointer may be NULL. */
mofem_status mofem_host_tables(const mofem_profile* g1, const mofem_profile* g2, int k, int n_nodes,
                               double gamma, mofem_bc bc, const mofem_opts* opts, int* n_terms, int* q,
                               double* S, double* T, double* Srh, double* Trh);

/* Host-only view of the double-float difference-form tables that the residual update
 * of a refinement step from zero reads (no device work; no counterpart in the paper:
 * the operator of Sec. 5 written in difference form for double-float evaluation).
 * S, T: FP32, a hi plane then a lo plane, each [n_terms][2K+1][q] as in
 * mofem_host_tables (caller-allocated, 2 x n_terms x (2K+1) x q floats; either may be
 * NULL).  Off the diagonal slot K: the FP64 coefficient c as (hi, lo) = (fl32(c),
 * fl32(c - hi)).  On slot K: the row sum of the FP64 coefficients, exact before one
 * rounding to (hi, lo), in every T table and in the S tables of the terms whose s-pass
 * runs in difference form (terms 0, 3, 4 of five; 0, 4..7 of eight), the plain
 * diagonal coefficient in the others.  T table 0 (the mass M_t of term 0) holds
 * N = D^-1 (M_t - D) off the diagonal and D = rowsum M_t on it. */
mofem_status mofem_host_dd_tables(const mofem_profile* g1, const mofem_profile* g2, int k, int n_nodes,
                                  double gamma, mofem_bc bc, const mofem_opts* opts, float* S, float* T);

#ifdef __cplusplus
}
#endif
#endif /* MOFEM_H */
