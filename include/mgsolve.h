/*
 * mgsolve.h - C ABI of the GB300 tensor-product multigrid solver for the LFRic
 * semi-implicit linear system.
 *
 * Method: Maynard, Melvin & Mueller, "Multigrid preconditioners for the mixed finite
 * element dynamical core of the LFRic atmospheric model" (arXiv 2002.00756):
 *   - outer Krylov solve of the mixed (velocity, pressure) system, Sec. 3.3 and Sec. 4.1
 *     (Eq. solver_notation), with GCR as in Sec. 5.1;
 *   - approximate Schur-complement preconditioner, Sec. 3.4 (Steps 1-3);
 *   - Helmholtz (pressure) operator H, Eq. helmholtz_operator and Sec. 3.5;
 *   - one tensor-product multigrid V-cycle for H, Sec. 3.6 and Algorithm 1: horizontal-
 *     only coarsening, block-Jacobi line smoother with an exact tridiagonal solve per
 *     vertical column (Eq. jacobi), injection prolongation (Eq. prolongation) and its
 *     dual as restriction, rediscretised coarse operators, n_coarse smoother sweeps on
 *     the coarsest level.
 *
 * Problem definition used by every entry point (lowest-order, strong volume-normalised
 * form, shallow atmosphere of radius R):
 *   (H x)_i = x_i + sum_{faces f of cell i} a_{i,f} (x_i - x_j(f)),
 *   a_{i,f} = (c_s dt)^2 g_f mu_f A_f / (V_i d_f),   g_f = (g_i + g_j) / 2,
 * A_f face area, V_i cell volume, d_f centre distance (great-circle arc horizontally,
 * centre-to-centre height vertically), mu_f = 1 / (lumped velocity mass of face f) for
 * the mixed system (1 for the pressure-only system).
 * No flux crosses the surface or the lid.
 *
 * Mesh convention (shared by all vectors): equiangular gnomonic cubed sphere C_n.
 * Panel p maps (xi, eta) in [-pi/4, pi/4]^2 to the unit sphere through the cube point
 * (a = tan xi, b = tan eta):
 *   p0 (1, a, b)   p1 (-a, 1, b)   p2 (-1, -a, b)   p3 (a, -1, b)   p4 (-b, a, 1)   p5 (b, a, -1)
 * Cell (p, j, i) spans xi in [-pi/4 + i d, -pi/4 + (i+1) d] (eta likewise with j),
 * d = pi / (2n); its column index is col = p n^2 + j n + i and its centre is the image
 * of the centre angles.  Cell fields are level-major: f[k * ncol + col], k = 0 at the
 * surface, ncol = 6 n^2, N = nlev * ncol.
 * Velocity vectors of the mixed system are [u_h, u_v]: u_h[k * 2ncol + f] over the
 * horizontal faces f of one level, listed once each under the lower-numbered of their
 * two columns, ordered by (that column, side E(+i), W(-i), N(+j), S(-j)); the face
 * normal points from that column to the other one.  u_v[kf * ncol + col], kf = 0..nlev,
 * face kf lying below cell k = kf (kf = 0 surface, kf = nlev lid; both carry no flux).
 *
 * Conventions for all calls:
 *   - vector arguments are DEVICE pointers to FP64 arrays owned by the caller; the
 *     handle owns the hierarchy, coefficients and workspace; solve calls allocate
 *     nothing;
 *   - calls are ordered on the given CUDA stream (0 = legacy default stream); solves
 *     synchronise that stream once per Krylov iteration to test convergence;
 *   - a handle is used by one stream at a time (calls on one handle must not overlap);
 *   - errors are returned as status codes, never as exceptions or process exits.
 */
#ifndef MGSOLVE_H
#define MGSOLVE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MG_OK = 0,
    MG_ERR_ARG = -1,            /* invalid argument (null pointer, size, mesh not divisible) */
    MG_ERR_CUDA = -2,           /* a CUDA runtime call failed */
    MG_ERR_NOMEM = -3,          /* device or host allocation failed in mg_setup */
    MG_ERR_NOT_CONVERGED = -4,  /* max_iter reached; info and the best iterate are filled */
    MG_ERR_BREAKDOWN = -5,      /* Krylov breakdown: <w, w> = 0 or a non-finite scalar */
    MG_ERR_TIMEOUT = -6,        /* reserved for bounded device-side waits */
    MG_ERR_UNSUPPORTED = -7     /* request outside what the handle was set up for */
} mg_status;

/* precision of the V-cycle (the outer Krylov solve is always FP64) */
enum {
    MG_FP64 = 0,            /* FP64 vectors and coefficients (the plain method) */
    MG_FP32 = 1,            /* FP32 vectors, coefficients and accumulation */
    MG_FP32_BF16COEF = 2,   /* FP32 vectors and accumulation, BF16 stored coefficients */
    MG_FP32_P64 = 3         /* MG_FP32, but the finest level's column elimination (Thomas pivots,
                               eliminated right-hand side, multipliers) runs in FP64 on the FP32
                               data; the stash and back substitution stay FP32.  Not with
                               mg_setup_9pt (MG_ERR_UNSUPPORTED) */
};

typedef struct {
    int32_t n;                   /* cubed sphere C_n (n divisible by 2^(levels-1)) */
    int32_t nlev;                /* vertical levels, 1..MG_MAX_NLEV */
    double radius;               /* planet radius R [m] */
    double cs_dt;                /* c_s * dt [m] */
    const double* z_interfaces;  /* HOST, nlev+1 increasing heights [m], z[0] = surface */
} mg_mesh;

typedef struct {
    int32_t levels;              /* multigrid levels L >= 1 (Sec. 3.6; L = 1: smoother only) */
    double omega;                /* over-relaxation of the block-Jacobi sweep (Eq. jacobi) */
    int32_t n_pre, n_post;       /* smoothing sweeps before / after the coarse correction */
    int32_t n_coarse;            /* sweeps from zero on the coarsest level */
    int32_t vcycle_precision;    /* MG_FP64 | MG_FP32 | MG_FP32_BF16COEF | MG_FP32_P64 */
    int32_t gcr_restart;         /* GCR directions kept before a restart, 1..MG_MAX_RESTART */
    int32_t max_iter;            /* Krylov iteration limit */
} mg_params;

/* mixed-system data (Sec. 3.3-3.4): velocity mass M-bar = M2 + tau_u dt M_C + eps B_w.
 *   B_w couples interior vertical face kf to kf+1 with weight beta_up[kf*ncol+col] and to
 *       kf-1 with beta_dn[kf*ncol+col] (only between interior faces; the folded buoyancy
 *       term of Step 1a);
 *   M2  is the identity (lumped mass) with consistent = 0; with consistent = 1 the
 *       consistent lowest-order Raviart-Thomas mass on the reference cell: per cell, with
 *       each face's basis function along the cell's own axis (xi for E/W, eta for N/S, up
 *       for bottom/top), 1/3 with itself and 1/6 with the opposite face of the cell; the
 *       global basis is that times the sign of the face normal along the axis;
 *   M_C is the implicit Coriolis term of Eq. M2muCdef in the traditional approximation:
 *       per cell F_c = coriolis_f0 * sin(latitude of the centre, axis z) times -1/4
 *       between each xi-face (row) and eta-face (column) of the cell and +1/4 between each
 *       eta-face and xi-face; coriolis_f0 = tau_u dt 2 Omega (0: no rotation).
 * The Schur-complement preconditioner lumps M-bar to the row sums taken in each cell's
 * own axes (the literal row sums inside every panel) and scales the Helmholtz coefficient
 * of every face by 1 / that lumped mass; a coarse horizontal face takes the edge-length-
 * weighted mean of its two fine faces' factors, a coarse vertical face the area-weighted
 * mean of its four children's. */
typedef struct {
    const double* beta_up;       /* HOST, (nlev+1) * ncol */
    const double* beta_dn;       /* HOST, (nlev+1) * ncol */
    double eps;
    int32_t consistent;          /* 0 lumped (identity) velocity mass, 1 consistent RT0 mass */
    double coriolis_f0;          /* tau_u dt 2 Omega, dimensionless, |f0| < 1/2 (lumped mass >= 1/2) */
} mg_mixed;

typedef struct {
    int32_t iters;               /* Krylov iterations done */
    double rel_res;              /* final ||b - A x||_2 / ||b||_2 (recursive residual) */
    double ms;                   /* wall time of the call on its stream [ms] */
} mg_solve_info;

#define MG_MAX_NLEV 128
#define MG_MAX_LEVELS 8
#define MG_MAX_RESTART 16

typedef struct mg_handle mg_handle;

/* Build the multigrid hierarchy (Sec. 3.6; coarse meshes C_{n/2}, ..., coarse operators
 * rediscretised from volume-weighted means of the background factors, Sec. 3.6 last
 * paragraph before Algorithm 1 and Sec. 5.1 set-up costs) on the current CUDA device.
 *   g      HOST, N background-state factors (cell field layout), g > 0
 *   mixed  NULL for the Helmholtz system alone; otherwise the mixed-system data, which
 *          also scales the Helmholtz coefficients by 1 / lumped mass of their faces
 * Meshes with 2 * (nlev + 1) * 6 n^2 >= 2^32 (more than about 2^31 horizontal-face values
 * on the finest level, e.g. n > 2240 at nlev = 70) are rejected with MG_ERR_UNSUPPORTED:
 * the column kernels address a level with 32-bit offsets.
 * On success *out holds a handle to release with mg_destroy.  Synchronous. */
mg_status mg_setup(const mg_mesh* mesh, const mg_params* params, const double* g,
                   const mg_mixed* mixed, mg_handle** out);

/* mg_setup for a finest-level operator given by its stencil coefficients (the operator /
 * preconditioner split of Sec. 4.1: the caller supplies the operator A_H, the library builds
 * the preconditioner P_H around it).
 *   coeffs        HOST, 6 N doubles a[s * N + k * ncol + c]: the couplings a_{i,f} of
 *                 Eq. helmholtz_operator in the strong form above for the sides s = E, W, N, S,
 *                 up, down of every finest-level cell (the layout helmholtz_coefficient_gradient
 *                 returns).  The outer Krylov solves, helmholtz_apply and the V-cycle's finest
 *                 level use exactly this operator.
 *   cell_factors  HOST, N background factors g > 0: the coarse operators are rediscretised
 *                 from their volume-weighted means as in mg_setup (Sec. 3.6, last paragraph
 *                 before Algorithm 1), so they approximate the caller's operator only as well
 *                 as g describes it (that affects the convergence rate, not the solution).
 * The operator must be flux-symmetric, V_i a_{i,f} = V_j a_{j,f} for the two cells of every
 * face (to 1e-10 relative; V the cell volumes of the mesh convention above): the V-cycle keeps
 * one value per face, and the adjoint solves rely on V H being symmetric.  Every coupling must
 * be finite and >= 0, and the up coupling of the top cell and the down coupling of the bottom
 * cell must be 0 (no flux through the lid or the surface).  Otherwise MG_ERR_ARG.  The
 * pressure system only (no mixed data).  Synchronous. */
mg_status mg_setup_coeffs(const mg_mesh* mesh, const mg_params* params, const double* coeffs,
                          const double* cell_factors, mg_handle** out);

/* mg_setup for the 9-cell stencil of Sec. 3.5 (Fig. 2): besides the 7-cell stencil above, every
 * cell couples to the cells two levels above and below through the flux
 *   (H x)_i += b_up,i (x_i - x_(k+2)) + b_dn,i (x_i - x_(k-2)),
 *   b_up(k) = T2_k / dz_k, b_dn(k + 2) = T2_k / dz_(k+2),
 *   T2_k = gamma2 (c_s dt)^2 (g_k + g_(k+2)) / 2 / (z_c(k+2) - z_c(k)),
 * on every multigrid level (rediscretised like the rest of H), so V H stays symmetric.  The
 * block-Jacobi smoother solves with the tridiagonal H_z-hat that drops these fluxes (Sec. 3.6):
 * the residual b - H x keeps them, the column solve does not.  A pressure-system handle (no
 * mixed data, no caller coefficients); precisions MG_FP64 and MG_FP32 (MG_ERR_UNSUPPORTED for
 * BF16 coefficients).  Every pressure-system call accepts it except helmholtz_coefficient_gradient,
 * mg_set_coefficients, mg_autotune and mg_smooth_noalloc (MG_ERR_UNSUPPORTED).  Its kernels are
 * plain one-thread-per-cell (per-column for the Thomas solve) versions of the 7-cell ones.
 * gamma2 > 0 and finite, else MG_ERR_ARG.  Synchronous. */
mg_status mg_setup_9pt(const mg_mesh* mesh, const mg_params* params, const double* g, double gamma2,
                       mg_handle** out);

/* Replace the finest-level operator of a pressure handle by new couplings (DEVICE, 6 N doubles,
 * same layout and conditions as mg_setup_coeffs); the coarse operators stay as set up.  This is
 * the forward step of a solve differentiated with respect to its stencil coefficients.  The
 * couplings are checked first; on MG_ERR_ARG the handle's operator is unchanged.
 * MG_ERR_UNSUPPORTED for a handle with mixed data.  Synchronous (ordered on `stream`). */
mg_status mg_set_coefficients(mg_handle* h, const double* coeffs, void* stream);

void mg_destroy(mg_handle* h);

const char* mg_status_string(mg_status s);

/* Name of the CUDA runtime error behind the last MG_ERR_CUDA returned on the calling thread
 * (e.g. "cudaErrorMemoryAllocation"), or "no CUDA error".  A non-sticky error is cleared when it
 * is reported, so it does not surface again in a later call. */
const char* mg_last_cuda_error(void);

/* Test hooks for the error paths (failure detection by host-side injection; no GPU fault).
 * mg_inject_alloc_failure(n), n > 0: the n-th device or pinned-host allocation the library
 * attempts after this call fails as if memory were exhausted, and the call making it returns
 * MG_ERR_NOMEM after releasing everything it had allocated; n <= 0 turns injection off.
 * Returns the number of allocations attempted since the previous call (so a set-up run between
 * two calls counts its allocations).  Process-wide; not for concurrent set-ups.
 * mg_live_allocations: the library's live device and pinned-host allocations over all handles
 * and ensembles (a leak check: it returns to its earlier value once they are destroyed). */
int64_t mg_inject_alloc_failure(int64_t nth);
int64_t mg_live_allocations(void);

/* Sizes of the handle's problem: ncol and N of the finest level, velocity unknowns
 * (0 without mixed data).  Any pointer may be NULL. */
mg_status mg_sizes(const mg_handle* h, int64_t* ncol, int64_t* ncell, int64_t* nu);

/* y = H x on the finest level in FP64 (Eq. helmholtz_operator; Sec. 3.5 stencil).
 * x, y: DEVICE, N doubles, must not overlap. */
mg_status helmholtz_apply(mg_handle* h, const double* x, double* y, void* stream);

/* x = V b: one V-cycle of Algorithm 1 from a zero initial guess (the preconditioner
 * P_H^(MG)(L, omega, n_pre, n_post) of Sec. 4.1), in the handle's V-cycle precision.
 * b, x: DEVICE, N doubles, must not overlap; the FP32 variants convert b on entry and x
 * on exit inside their first and last sweep kernels. */
mg_status vcycle(mg_handle* h, const double* b, double* x, void* stream);

/* Solve H x = b by GCR(gcr_restart) right-preconditioned with one V-cycle per iteration
 * (K_H(A_H, P_H^(MG), tol) of Eq. solver_notation), x0 = 0, stopping when
 * ||b - H x||_2 <= tol ||b||_2 (FP64 vectors, residuals and inner products).
 * b, x: DEVICE, N doubles.  info may be NULL.  Returns MG_ERR_NOT_CONVERGED after
 * max_iter iterations (x then holds the last iterate), MG_ERR_BREAKDOWN on a zero or
 * non-finite <w, w> or residual. */
mg_status pressure_solve(mg_handle* h, const double* b, double* x, double tol,
                         mg_solve_info* info, void* stream);

/* Solve the mixed system A [u; p] = [rhs_u; rhs_p] (Eq. linear_matrix, reduced (u, p)
 * form) by GCR(gcr_restart) right-preconditioned with the approximate Schur complement
 * (Sec. 3.4 Steps 1-3, one V-cycle for Step 2), x0 = 0, stopping on the Euclidean norm of
 * the concatenated residual.  Needs a handle set up with mixed data.
 * rhs_u, u: DEVICE, nu doubles; rhs_p, p: DEVICE, N doubles. */
mg_status mixed_solve(mg_handle* h, const double* rhs_u, const double* rhs_p, double* u,
                      double* p, double tol, mg_solve_info* info, void* stream);

/* ---- single steps of the method, FP64, for checking each kernel on its own ---- */

/* y = H^(level) x on multigrid level `level` (0 = finest); DEVICE arrays of that level's
 * N_l = nlev * 6 (n / 2^level)^2 doubles. */
mg_status mg_level_apply(mg_handle* h, int32_t level, const double* x, double* y, void* stream);

/* x_out = BlockJacobi(H^(level), b, x_in, omega, sweeps) (Eq. jacobi), x_in == NULL meaning
 * a zero initial guess.  x_in and x_out may be the same array; b must not overlap x_out. */
mg_status mg_smooth(mg_handle* h, int32_t level, const double* b, const double* x_in,
                    double* x_out, int32_t sweeps, void* stream);

/* bc = Restrict(b - H^(level) x) onto level+1 (Algorithm 1, residual and restriction). */
mg_status mg_residual_restrict(mg_handle* h, int32_t level, const double* b, const double* x,
                               double* bc, void* stream);

/* x += Prolongate(xc) from level+1 onto level (Eq. prolongation, natural injection). */
mg_status mg_prolong_add(mg_handle* h, int32_t level, const double* xc, double* x, void* stream);

/* Adjoint of pressure_solve: lambda = H^-T g, the gradient dL/db of a loss L(x) of the solution
 * x = H^-1 b given g = dL/dx (the differentiable solve of the batched-ensemble and data
 * assimilation uses).  The strong-form H of this library has V H symmetric (V the cell
 * volumes, Sec. 3.5: the flux through a face is the same seen from both cells), so
 * H^T = V H V^-1 and lambda = V H^-1 (V^-1 g): the same GCR and V-cycle as pressure_solve on
 * the right-hand side V^-1 g, then a multiplication by V.  tol applies to that solve.
 *   g, lambda  DEVICE, N doubles each, g != lambda.  Synchronous. */
mg_status pressure_solve_adjoint(mg_handle* h, const double* g, double* lambda, double tol,
                                 mg_solve_info* info, void* stream);

/* Gradient of a loss L(x), x = H^-1 b, with respect to the six couplings a_{i,f} of every
 * finest-level cell (the strong-form coefficients of Eq. helmholtz_operator): from
 * H x = b, dL = -<lambda, dH x> with lambda = H^-T dL/dx (pressure_solve_adjoint), so
 *     grad[s * N + i] = dL/da_{i,s} = -lambda_i (x_i - x_{j(i,s)}),
 * s = 0..5 for the E, W, N, S, upper and lower neighbour (0 where there is none: top and
 * bottom of a column).  lambda, x: DEVICE, N doubles; grad: DEVICE, 6 N doubles. */
mg_status helmholtz_coefficient_gradient(mg_handle* h, const double* lambda, const double* x, double* grad,
                                         void* stream);

/* Ensemble of independent pressure solves (the batched-ensemble use of Sec. 4.1's solver:
 * many members, each its own mesh, levels and precision): handles[i] solves
 * H_i x[i] = b[i] exactly as pressure_solve does (same kernels in the same order, so the
 * same x bit for bit), and the members' iterations are interleaved: each round launches one
 * GCR iteration of every unfinished member on that member's own stream, so small members run
 * side by side on the GPU, then the host reads their residual norms.
 *   handles   count distinct handles of one device
 *   b, x      count DEVICE pointers each, N_i doubles (x[i] != b[i])
 *   infos     NULL or count entries: iterations, final relative residual, and the member's
 *             time from its first launch to its last on the GPU [ms]
 *   statuses  NULL or count entries: each member's status (as pressure_solve returns it)
 *   stream    the members start after the work queued on this stream so far
 * Synchronous: returns when every member is done.  Returns MG_OK if every member converged,
 * else the first member's non-OK status; MG_ERR_ARG for a NULL or repeated handle, handles
 * on different devices, or x[i] == b[i]. */
mg_status ensemble_pressure_solve(mg_handle* const* handles, int32_t count, const double* const* b,
                                  double* const* x, double tol, mg_solve_info* infos, int32_t* statuses,
                                  void* stream);

/* ---- an ensemble of pressure solves as ONE graph launch ----
 * mg_ensemble_create records, once, the whole of every member's pressure_solve into one CUDA
 * graph: per member the start (r = b, x = 0, <b, b>), then a conditional WHILE node whose body
 * holds one conditional IF node per GCR restart slot j (the V-cycle, the fused apply and the
 * orthogonalisation of slot j, then a single-thread kernel that takes the convergence,
 * iteration-limit and breakdown decisions the host takes in pressure_solve) and one IF node for
 * the solution update that closes a restart cycle.  The members are independent branches of the
 * graph, so members of different meshes, level counts and precisions run side by side, and
 * every decision stays on the device: mg_ensemble_solve is one cudaGraphLaunch followed by one
 * stream synchronisation.  Each member gets exactly what pressure_solve gives it alone (the same
 * kernels in the same order, the same FP64 decisions): the same x bit for bit, the same
 * iteration count and status.  No device-side wait is involved (the conditions are set by a
 * kernel that precedes the nodes reading them).
 *   handles   count distinct pressure handles (no mixed data, not profiling) of one device
 *   b, x      count DEVICE pointers, N_i doubles each (x[i] != b[i]); recorded into the graph, so
 *             every solve reads b[i] and writes x[i] at these addresses (refill b between solves)
 *   tol       relative residual of every member
 * The handles must outlive the ensemble and must not be used by other calls while
 * mg_ensemble_solve runs; launch shapes chosen by a later mg_autotune are not picked up
 * (create the ensemble after tuning).  Synchronous.  MG_ERR_UNSUPPORTED for a mixed or
 * profiling handle. */
typedef struct mg_ensemble mg_ensemble;
mg_status mg_ensemble_create(mg_handle* const* handles, int32_t count, const double* const* b, double* const* x,
                             double tol, mg_ensemble** out);

/* Run every member once (one graph launch, then one synchronisation of `stream`).  infos (may be
 * NULL, count entries): iterations, final relative residual and the member's completion time
 * from the launch [ms]; statuses (may be NULL): each member's status as pressure_solve returns
 * it.  Returns MG_OK if every member converged, else the first member's non-OK status. */
mg_status mg_ensemble_solve(mg_ensemble* e, mg_solve_info* infos, int32_t* statuses, void* stream);

void mg_ensemble_destroy(mg_ensemble* e);

/* [yu; yp] = A [u; p], the mixed operator (needs mixed data). */
mg_status mixed_apply(mg_handle* h, const double* u, const double* p, double* yu, double* yp,
                      void* stream);

/* [yu; yp] = A^T [u; p], the transposed mixed operator, evaluated as S J A-hat J S^-1 (see
 * mixed_solve_adjoint).  Uses the handle's mixed workspace: not concurrent with a mixed
 * solve on the same handle.  u, yu: DEVICE, nu doubles; p, yp: DEVICE, N doubles. */
mg_status mixed_apply_transpose(mg_handle* h, const double* u, const double* p, double* yu, double* yp,
                                void* stream);

/* Adjoint of the mixed solve (the backward step of a differentiable mixed_solve): with
 * g = [g_u; g_p] = dL/d[u; p] for a loss L of the solution of A [u; p] = rhs, computes
 * lambda = A^-T g = dL/drhs.  The discrete integration by parts of the gradient and
 * divergence of Sec. 3.3 (W G = -D^T V with face weights W_f = A_f d_f / g_f, A_f the face
 * area, d_f the centre distance, and V the cell volumes) gives A^T = S J A-hat J S^-1 with
 * S = diag(W, V), J = diag(I, -I) and A-hat the mixed operator whose velocity mass is
 * W^-1 M-bar^T W.  So lambda = S J y with A-hat y = J S^-1 g, solved by GCR(gcr_restart) with
 * the same Schur-complement preconditioner as mixed_solve (its transpose is S J P J S^-1 by
 * the same identity and the V-symmetry of the V-cycle).  tol applies to the relative
 * residual of the A-hat system (W and V are of the same size, so it is close to that of
 * A^T lambda = g); info as for mixed_solve.
 * g_u, lam_u: DEVICE, nu doubles; g_p, lam_p: DEVICE, N doubles; g and lambda must not
 * overlap the handle's buffers (any caller-owned arrays qualify). */
mg_status mixed_solve_adjoint(mg_handle* h, const double* g_u, const double* g_p, double* lam_u, double* lam_p,
                              double tol, mg_solve_info* info, void* stream);

/* Gradient of a loss L of the mixed solution [u; p] = A^-1 rhs with respect to the set-up
 * inputs of the mixed operator, given lam = [lam_u; lam_p] = A^-T dL/d[u; p] (from
 * mixed_solve_adjoint): dL/dtheta = -<lam, (dA/dtheta) [u; p]>.  The background factors g
 * enter A only through the gradient weights kappa_f / d_f = c_s dt (g_i + g_j) / (2 d_f), so
 *   grad_g[k][c]     = -sum over the six faces f of cell (k, c) of lam_f (p_R(f) - p_L(f)) c_s dt / (2 d_f);
 * the couplings of B_w enter as eps beta, so
 *   grad_beta_up[kf][c] = -eps lam_kf u_kf+1,  grad_beta_dn[kf][c] = -eps lam_kf u_kf-1
 * on the vertical faces whose coupling exists (0 elsewhere).  lam_p is not needed (the
 * pressure rows hold no set-up input).  Not through the preconditioner: the solution does
 * not depend on it.
 * lam_u, u: DEVICE, nu doubles; p, grad_g: DEVICE, N doubles; grad_beta_up, grad_beta_dn:
 * DEVICE, (nlev+1) * ncol doubles. */
mg_status mixed_coefficient_gradient(mg_handle* h, const double* lam_u, const double* u, const double* p,
                                     double* grad_g, double* grad_beta_up, double* grad_beta_dn, void* stream);

/* Autotuner of the column tiles: for every multigrid level, times the candidate launch
 * shapes of the block-Jacobi sweep (64 or 128 threads per block: 32 or 64 columns) and of
 * the residual + restriction (4, 8, 16, 24, 35 or 70 levels per thread; on FP32 levels whose
 * n is a multiple of 16 also the copy-ring or register-ring kernel) with CUDA events around
 * every launch of full V-cycles on the handle's own buffers, and keeps the fastest shape per
 * level for every later call.  Every shape gives the same result bit for bit (each output
 * element is computed by one thread from the same inputs in the same order), so tuning
 * changes times only.  Synchronous; a few dozen V-cycles; drops the handle's cached GCR
 * graphs (they are captured again by the next solve).  MG_ERR_UNSUPPORTED while per-launch
 * profiling (mg_profile_start) is on.
 * choices: NULL or 3 * levels int32 written per level: sweep threads per block, restriction
 * levels per thread, 1 copy ring / 0 register ring (0 and -1 on the coarsest level, which has
 * no restriction). */
mg_status mg_autotune(mg_handle* h, int32_t* choices, void* stream);

/* [u; p] = P_mixed [ru; rp], the Schur-complement preconditioner with one V-cycle. */
mg_status schur_precond(mg_handle* h, const double* ru, const double* rp, double* u, double* p,
                        void* stream);

/* ---- the pressure solver of the Schur-complement step (Sec. 4.1, Eq. solver_notation
 * K_mixed(A_mixed, P_mixed(K_H(A_H, P_H, eps_H)), eps); the configurations of Table 1) ---- */
enum {
    MG_PS_MG = 0,               /* MG(L): PreOnly, one V-cycle P_H^(MG)(L, omega, n_pre, n_post) (default) */
    MG_PS_JACOBI = 1,           /* line relaxation: PreOnly, P_H^(Jac)(omega, sweeps) */
    MG_PS_BICGSTAB_JACOBI = 2,  /* Krylov(eps_H): BiCGStab(A_H, P_H^(Jac)(omega, sweeps), eps_H) */
    MG_PS_BICGSTAB_MG = 3       /* Krylov-MG(eps_H, L): BiCGStab(A_H, P_H^(MG)(L, ...), eps_H) */
};

typedef struct {
    int32_t kind;       /* MG_PS_* */
    double eps;         /* eps_H, relative residual of the BiCGStab kinds (Table 1: 1e-2, 1e-3, 1e-6) */
    double omega;       /* over-relaxation of the block-Jacobi kinds (Table 1: 0.8 and 1.0) */
    int32_t sweeps;     /* n_Jac, block-Jacobi sweeps from zero (Table 1: 10 and 1) */
    int32_t max_iter;   /* BiCGStab iteration limit */
} mg_pressure_solver;

/* Select the pressure solver that Step 2 of the Schur-complement preconditioner (schur_precond,
 * mixed_solve, mixed_solve_adjoint) and helmholtz_solve use.  P_H^(Jac)(omega, n) is n
 * block-Jacobi sweeps (Eq. jacobi) from zero on the finest level; BiCGStab is van der Vorst's
 * method with the preconditioner on the right, x0 = 0, shadow residual b, stopping when the
 * recursively updated residual of either half step is below eps ||b||.  BiCGStab synchronises
 * with the host once per iteration, so mixed solves that use it launch their iterations
 * directly (no graphs); an inner solve that reaches max_iter still serves as the
 * preconditioner.  The first selection of a BiCGStab kind allocates its 8 vectors of N doubles.
 * Synchronous.  MG_ERR_ARG for an unknown kind or invalid parameters. */
mg_status mg_set_pressure_solver(mg_handle* h, const mg_pressure_solver* ps);

/* x = K_H(A_H, P_H, eps_H) b, the handle's pressure solver on its own (the "pressure solve" of
 * Table 2), from x = 0.  b, x: DEVICE, N doubles.  *iterations (may be NULL): BiCGStab
 * iterations, a half step counting 0.5 (0 for the PreOnly kinds).  MG_ERR_NOT_CONVERGED when
 * BiCGStab reaches max_iter (x holds its last iterate), MG_ERR_BREAKDOWN on a zero or
 * non-finite scalar.  The BiCGStab kinds are synchronous. */
mg_status helmholtz_solve(mg_handle* h, const double* b, double* x, double* iterations, void* stream);

/* BiCGStab pressure solves run since the last call (inside mixed solves or helmholtz_solve),
 * and their iterations (half steps counting 0.5); resets both.  Either pointer may be NULL. */
mg_status mg_inner_stats(mg_handle* h, int64_t* solves, double* iterations);

/* ---- block-Jacobi smoothing that allocates nothing ----
 * The paper has no counterpart to this call: it is a service for callers that cannot
 * allocate device memory at the point where they smooth, for instance a real-time loop
 * that must not enter the allocator (its latency is unbounded), a host framework whose
 * memory pool owns all device memory after start-up, or a process that runs under a
 * fixed device-memory budget it must not exceed.
 *
 * It computes exactly what mg_smooth computes (same kernels, same order), but it neither
 * allocates nor touches the handle's workspace: intermediate iterates are kept in one
 * fixed device array inside the library of MG_NOALLOC_MAX_CELLS doubles (16 MiB), which
 * every GPU that loads the library holds until the process exits.  Levels with more than
 * MG_NOALLOC_MAX_CELLS cells (nlev * 6 (n / 2^level)^2) are rejected with MG_ERR_ARG.
 * The handle itself still comes from mg_setup.
 *   - The first call on a device looks up the array's device address (with that device
 *     current), so make that first call before any stream capture begins.
 *   - All calls share the one array: calls that overlap on the GPU (on different streams,
 *     or from different threads without ordering) race with each other and must be
 *     serialised by the caller.  The array keeps the last call's contents; nothing in it
 *     needs to start at zero, because every sweep writes all its cells before any is read.
 * Arguments as for mg_smooth (x_in == NULL: zero initial guess; x_in may equal x_out). */
#define MG_NOALLOC_MAX_CELLS (1 << 21)
mg_status mg_smooth_noalloc(mg_handle* h, int32_t level, const double* b, const double* x_in,
                            double* x_out, int32_t sweeps, void* stream);

/* ---- per-launch profiling ----
 * While profiling is on, every kernel launch made by the calls above is bracketed by two
 * CUDA events on its stream, and its kind, multigrid level and algorithmic traffic (every
 * array element the kernel must read or write, counted once) are recorded. */
enum {
    MG_K_SWEEP = 0,       /* block-Jacobi sweep (residual + Thomas + update) */
    MG_K_RESTRICT = 1,    /* residual + restriction */
    MG_K_PROLONG = 2,     /* prolongation (when not fused into a sweep) */
    MG_K_APPLY = 3,       /* Helmholtz apply */
    MG_K_CONVERT = 4,     /* precision conversion */
    MG_K_DOT = 5,         /* inner product */
    MG_K_GCR_DOTS = 6,    /* GCR orthogonalisation inner products */
    MG_K_GCR_ORTH = 7,    /* GCR orthogonalisation update + <w,w>, <r,w> */
    MG_K_GCR_UPDATE = 8,  /* GCR x, r update + <r,r> */
    MG_K_MIXED = 9        /* mixed operator / Schur steps */
};

typedef struct {
    int32_t kind;      /* MG_K_* */
    int32_t level;     /* multigrid level (0 = finest) */
    int32_t variant;   /* sweeps: iterate source, 0 plain, 1 zero, 2 prolongated, 3 prolongation only;
                          fused GCR apply: number of stored directions J; otherwise 0 */
    double bytes;      /* algorithmic bytes of the launch */
    double ms;         /* event-timed duration */
} mg_kernel_record;

/* Start recording up to `capacity` launches (creates the events; not a solve call).  Only
 * launches of the given kind (MG_K_*) and multigrid level are recorded; -1 for either
 * records all kinds or all levels.  Every recorded launch adds two event records to its
 * stream, so a narrow selection keeps the recording cheap inside a timed region. */
mg_status mg_profile_start(mg_handle* h, int32_t capacity, int32_t kind, int32_t level);

/* Stop recording, synchronise the device and copy up to `cap` records to `out` (HOST);
 * *count receives the number recorded (launches beyond the capacity are not timed). */
mg_status mg_profile_stop(mg_handle* h, mg_kernel_record* out, int32_t cap, int32_t* count);

#ifdef __cplusplus
}
#endif
#endif
