/*
 * lt.h -- C ABI of the Laplace-transform / flexible shifted-Krylov engine
 * for parabolic problems  S_s dphi/dt - div(kappa grad phi) = q(t) delta(x - x_s)
 * (Bakhos, Saibaba & Kitanidis, "A fast algorithm for parabolic PDE-based
 * inverse problems based on Laplace transforms and flexible Krylov
 * solvers", Sec. 2-3 and Sec. 5.2).
 *
 * One context drives one GPU.  Every entry point returns an int status:
 * LT_OK (0) or a negative LT_ERR_* code; nothing aborts the process.  On an
 * error, lt_last_error(ctx) returns a message naming the offending argument.
 *
 * Ownership: the caller owns every buffer it passes.  Inputs are copied
 * before the call returns.  Outputs are written into caller buffers.  The
 * context owns its own device workspace (released by lt_destroy).
 *
 * Grid layout: cell (i, j, k), 0 <= i < nx, 0 <= j < ny, 0 <= k < nz, has
 * the linear index c = (k * ny + j) * nx + i (x fastest).  A 2D aquifer is
 * nz = 1 with dz = the aquifer thickness (1 for transmissivity/storativity
 * units, Sec. 2.1), and Neumann faces on z.
 */
#ifndef LT_H
#define LT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define LT_OK                 0
#define LT_ERR_INVALID_ARG   -1   /* bad size, non-positive coefficient, index out of range, t <= 0 */
#define LT_ERR_OOM           -2   /* device allocation failed */
#define LT_ERR_CUDA          -3   /* any other CUDA runtime error */
#define LT_ERR_NOT_CONVERGED -4   /* results written; some shifts above tol (see lt_stats) */
#define LT_ERR_TIMEOUT       -5   /* a bounded device wait expired */
#define LT_ERR_STATE         -6   /* call order violated (e.g. forward before setup_grid) */

/* boundary condition codes, one per face: x-, x+, y-, y+, z-, z+ (Sec. 2.1, Eq. timedomain) */
#define LT_BC_DIRICHLET 0         /* phi = 0 (ghost half a cell outside the face) */
#define LT_BC_NEUMANN   1         /* grad phi . n = 0 */
#define LT_BC_WATERTABLE 2        /* linearised water table: no flux, storage S_y x face area (Sec. 2.1) */

/* preconditioner-shift policies (Sec. 3, last paragraph; Sec. 4.1) */
#define LT_TAU_SINGLE   0         /* one shift: the node with the smallest real part */
#define LT_TAU_FLEXIBLE 1         /* tau_bar1 (smallest Re) x3, tau_bar2 (largest Re) x2, repeated */

typedef struct lt_ctx lt_ctx;

typedef struct {
  int    Nz;            /* contour nodes per time, even, 4..128; Nz/2 shifted systems per time (Eq. half) */
  double tol;           /* relative residual ||b - (K + z M) x|| / ||b|| per shift (default 1e-8) */
  int    maxit;         /* outer flexible-Krylov iterations per basis (default 160) */
  int    tau_policy;    /* LT_TAU_SINGLE or LT_TAU_FLEXIBLE */
  int    tau_project;   /* 1: replace Re(tau) by max(Re(tau), 0) so multigrid stays convergent (default 1) */
  int    groups;        /* number of contiguous time windows, one Krylov basis per (source, window) */
  int    mg_pre;        /* red-black Gauss-Seidel sweeps before the coarse correction (default 2) */
  int    mg_post;       /* ... and after (default 2) */
  int    inner_cycles;  /* V-cycles per refinement round of a preconditioner solve (default 6) */
  int    inner_rounds;  /* refinement rounds per preconditioner solve (default 6; finished solves skip the rest) */
  double inner_tol;     /* relative residual of each preconditioner solve (default 0.01 * tol) */
  int    true_residual; /* 1: compute the true residual of every shift after the solve (default 1) */
  int    check_every;   /* outer iterations between host convergence polls (default 4) */
  int    timing_class;  /* -1: off; else time every launch of this kernel class with CUDA events (LT_KC_*) */
  double inner_relax;   /* 0: fixed inner_tol; > 0: inner tolerance relaxed as inner_tol / (largest unconverged
                           projected residual of the basis), capped at inner_relax (inexact-Krylov relaxation) */
  int    graphs;        /* 1: replay one captured CUDA graph per outer iteration (default); 0: direct launches */
  int    mg_tile;       /* fused 2D smoother tile: 0 = 64x32, 1 = 32x32, 2 = 32x16 cells (default 2) */
  int    precond;       /* 0: multigrid (default); 1: learned initial guess + multigrid (see lt_set_learned_preconditioner) */
  int    mg_tma;        /* 1: stage the fused 2D tiles with TMA bulk tensor copies when alignment allows (default) */
  int    mg_cluster;    /* 1: run each preconditioner solve (all rounds and V-cycles) inside one 8-CTA thread-block
                           cluster with the multigrid levels in distributed shared memory, on grids that allow it
                           (2D, rows divisible into 8 strips per level, levels fit in shared memory; default);
                           2: the same in 16-CTA clusters (non-portable size) of 256 threads with half-height
                           strips, so that two CTAs of different bases share an SM (rows divisible into 16
                           strips per level); 3: 8-CTA clusters of 256 threads with the finest level's iterate
                           in global memory (L2) instead of shared memory, so that two CTAs of different bases
                           share an SM; 4: 4-CTA clusters of 512 threads, finest-level iterate in global
                           memory (half the SMs per basis); 0: batched multigrid launches.  A grid the chosen
                           form does not fit runs the batched launches */
  int    precision;     /* LT_PREC_FP64 (default) or LT_PREC_FP32 (reduced precision, tolerances down to 2e-6) */
  int    krylov;        /* LT_KRYLOV_GMRES (default): minimal-residual coefficients per shift (FGMRES-Sh);
                           LT_KRYLOV_FOM: Petrov-Galerkin coefficients H_j(z_k; T_j) y = beta e_1 (FFOM-Sh),
                           both from Algorithm 1 of Sec. 3 */
  int    stop_rule;     /* LT_STOP_SHIFT (default): each shift stops on its own relative residual <= tol;
                           LT_STOP_QUADRATURE: all shifts of an output time stop together once the
                           quadrature-weighted residual sum_k |w_k qhat(z_k)| rho_k <= tol sum_k |w_k qhat(z_k)|
                           (the a-posteriori bound of Sec. 3.1, Proposition 1; rho_k = |eta_k| for FOM) */
  int    tma_wait_polls;/* polls of the mbarrier before a TMA tile load counts as timed out (default 1 << 26);
                           0 makes every TMA tile load time out at once, which exercises the
                           LT_ERR_TIMEOUT path without a fault */
  int    gram_schmidt;  /* orthogonalisation of s_j = M u_j against V_j (Algorithm 1's inner loop):
                           2 = classical Gram-Schmidt twice, coefficients from float32 dots (default);
                           1 = one classical pass whose coefficients come from df32 dots (V read twice
                           instead of four times per column) */
  int    block;         /* 0: one Krylov basis per (source, window) (default);
                           1: block flexible GMRES-Sh: the sources of a window share one block Krylov space
                           (the block variant of Algorithm 1 that Sec. 6 names as future work).  Each
                           source still gets its own preconditioner solve per iteration; the Arnoldi process
                           and each shift's least squares treat the p sources as p right-hand sides, and each
                           (shift, source) stops on its own residual.  lt_forward and lt_forward_fields only,
                           with 1 <= p <= 16 sources in distinct cells, LT_KRYLOV_GMRES, LT_STOP_SHIFT,
                           LT_PREC_FP64 and no initial state; other entry points return LT_ERR_INVALID_ARG */
} lt_opts;

/* arithmetic of the outer Krylov method (lt_opts.precision) */
#define LT_PREC_FP64    0         /* basis, solutions and residuals carried in double-float32 pairs (about
                                     48 significant bits; every relation checked to ~1e-13): results within
                                     1e-8 of an FP64 solve */
#define LT_PREC_FP32    1         /* single float32 planes for the basis, the preconditioner solutions and x_k
                                     (half the Krylov memory and traffic); tol >= 2e-6, for results within
                                     1e-5 of an FP64 solve.  Rounding a solution to float32 alone leaves a true
                                     residual of about cond(K + z M) * 6e-8 (near 2e-7 for point sources, far
                                     more for smooth right-hand sides such as M phi_0), so in this mode set
                                     true_residual = 0 and decide convergence by the projected residual */
/* coefficient rule of Algorithm 1 (lt_opts.krylov) */
#define LT_KRYLOV_GMRES 0
#define LT_KRYLOV_FOM   1
/* stopping rule (lt_opts.stop_rule) */
#define LT_STOP_SHIFT      0
#define LT_STOP_QUADRATURE 1

/* kernel classes reported in lt_stats.work[] and selectable by lt_opts.timing_class */
#define LT_KC_RBGS       0   /* red-black Gauss-Seidel half-sweep on a fine multigrid level */
#define LT_KC_RESTRICT   1
#define LT_KC_PROLONG    2
#define LT_KC_COARSE     3   /* single-CTA coarse-level V-cycle */
#define LT_KC_EXACT_RES  4   /* df32 residual of a preconditioner solve */
#define LT_KC_UPDATE_U   5
#define LT_KC_DOTS       6   /* Gram-Schmidt coefficients (float32 dots) */
#define LT_KC_ORTHO      7   /* Gram-Schmidt df32 vector updates */
#define LT_KC_NORMALIZE  8
#define LT_KC_SHIFT_LS   9
#define LT_KC_XK        10   /* x_k = U y_k for the true residual */
#define LT_KC_TRUE_RES  11
#define LT_KC_FUSED_DOWN 12  /* fused 2D tile: pre-smoothing + residual + restriction (cells counted once) */
#define LT_KC_FUSED_UP   13  /* fused 2D tile: prolongation + correction + post-smoothing */
#define LT_KC_INNER      15  /* cluster-resident preconditioner solve (fine-level cells x V-cycles) */
#define LT_KC_COUNT     16

typedef struct {
  int    n_bases;             /* Krylov bases built (sources x groups, or receivers x groups) */
  int    n_shift_solves;      /* shifted systems solved = sum over bases of shifts per basis */
  int    n_converged;         /* shifts whose true relative residual is <= tol (or projected, if true_residual = 0) */
  int    outer_iters_max;     /* largest outer iteration count over bases */
  int    outer_iters_sum;     /* sum over bases */
  int    inner_cycles_total;  /* V-cycles issued (per basis, summed) */
  double max_true_residual;   /* max over shifts of the true relative residual (-1 if not computed) */
  double max_proj_residual;   /* max over shifts of the projected (least-squares) residual */
  double max_inner_residual;  /* max relative residual of a preconditioner solve */
  float  ms_total;            /* device time of the call (CUDA events on the context stream) */
  int    kernel_launches;     /* kernels launched by the call */
  float  timed_ms;            /* summed CUDA-event time of the launches of opts.timing_class */
  int    timed_launches;      /* number of those launches */
  unsigned long long work[16];/* cells processed per kernel class (x basis vectors for LT_KC_DOTS/ORTHO) */
} lt_stats;

/* Fill *opts with the defaults listed above.  Returns LT_OK. */
int lt_default_options(lt_opts* opts);

/* Create a context on CUDA device `device`.  *out receives the handle. */
int lt_create(lt_ctx** out, int device);

/* Run all later work on `stream` (a cudaStream_t; NULL = the legacy default stream). */
int lt_set_stream(lt_ctx* ctx, void* stream);

/*
 * Set the grid and coefficients (Sec. 2.1, the semi-discrete system
 * M phi' + K phi = q(t) b restated on a cell-centred finite-volume grid):
 *   kappa, Ss : [nz][ny][nx] float64, every entry > 0 and finite, HOST pointers
 *   dx, dy, dz: cell sizes > 0
 *   bc        : 6 face codes (x-, x+, y-, y+, z-, z+), LT_BC_*; at least one Dirichlet face
 *   Sy        : specific yield [ncell] float64 HOST, finite and >= 0, read for the cells on
 *               water-table faces (required when a face is LT_BC_WATERTABLE, else may be NULL)
 * Face transmissibility between cells a, b: (area/dist) * 2 kappa_a kappa_b / (kappa_a + kappa_b);
 * a Dirichlet face adds 2 kappa_c area / dist to the diagonal; a water-table face carries no flux
 * and adds Sy_c * (face area) to the cell's storage (the boundary term (S_y d phi/dt, psi) of the
 * weak form of Sec. 2.1); M = diag(Ss_c * dx dy dz + water-table storage).  The adjoint's
 * d/d log Ss_c differentiates the Ss_c * dx dy dz part only.
 * Builds the multigrid hierarchy.  Each dimension must be 1 or >= 2, and repeated halving of the
 * even dimensions must reach at most 1024 cells.
 */
int lt_setup_grid(lt_ctx* ctx, int nx, int ny, int nz, double dx, double dy, double dz,
                  const double* kappa, const double* Ss, const int* bc, const double* Sy);

/* Point sources b_s = Q_s e_{cell_s}, constant rate Q_s switched on at t = 0 (Sec. 2.1).
 * cells: HOST int64 [ns], each in [0, ncell); Q: HOST float64 [ns].  Clears any rates set by
 * lt_set_source_rates. */
int lt_set_sources(lt_ctx* ctx, int ns, const int64_t* cells, const double* Q);

/*
 * Time-varying pumping rates (Sec. 2.1-2.2: sources separable in space and time, q(t) with a
 * known Laplace transform; Sec. 2.2 names exponential sums, fitted by Prony's method, for a
 * general q): source s pumps
 *     q_s(t) = sum_{j < nterm[s]} a_j exp(-lambda_j t),   qhat_s(z) = sum_j a_j / (z + lambda_j),
 * which replaces Q_s / z in every quadrature weight (forward and adjoint).
 *   ns     : must equal the number of sources set by lt_set_sources
 *   nterm  : HOST int [ns], each in [1, 64]; NULL restores the constant rates Q_s
 *   a      : HOST float64 [sum nterm], amplitudes (m^3/s), source by source
 *   lambda : HOST float64 [sum nterm], decay rates (1/s), each finite and >= 0 (0 = a constant term)
 * Copied at the call.  LT_ERR_INVALID_ARG on a count mismatch or a bad value.
 */
int lt_set_source_rates(lt_ctx* ctx, int ns, const int* nterm, const double* a, const double* lambda);

/*
 * Initial head phi(0) = phi_0 (Sec. 2.2, F(z) = (K + z M)^{-1} (M phi_0 + qhat(z) b); Sec. 3, the
 * two right-hand sides [b, M phi_0]).  The forward calls then add, for every source, the
 * response to phi_0, solved as one more Krylov basis per time group with the right-hand side
 * M phi_0.  phi0: HOST float64 [ncell], finite; NULL (or all zeros) restores phi_0 = 0.
 * lt_setup_grid clears it.  The adjoint entry points need phi_0 = 0 (LT_ERR_STATE otherwise).
 */
int lt_set_initial_state(lt_ctx* ctx, const double* phi0);

/* Point receivers (measurement cells, Sec. 5.2 functional I(t)).  cells: HOST int64 [nr]. */
int lt_set_receivers(lt_ctx* ctx, int nr, const int64_t* cells);

/* Replace the solver options (copied).  Invalid values give LT_ERR_INVALID_ARG. */
int lt_set_options(lt_ctx* ctx, const lt_opts* opts);

/*
 * Forward problem (Sec. 2.2 Eq. half and Sec. 3 Algorithm 1): for every
 * source s, receiver r and time t,
 *   h[s][r][t] = 2 Re sum_k w_k(t) (qhat_s(z_k) x_{s,k}[cell_r] + beta0 x_{0,k}[cell_r]),
 *   (K + z_k M) x_{s,k} = e_{cell_s},  (K + z_k M) x_{0,k} = M phi_0 / beta0,  beta0 = ||M phi_0||
 * over the N_z/2 upper-half Talbot nodes of each time (qhat_s = Q_s / z without lt_set_source_rates;
 * the x_0 term only with an initial state).
 *   times : HOST float64 [nt], each > 0
 *   h     : float64 [ns][nr][nt], HOST pointer if h_on_device == 0, else a DEVICE pointer
 *   stats : optional (may be NULL)
 * Returns LT_ERR_NOT_CONVERGED (with h written) if any shift misses tol.
 */
int lt_forward(lt_ctx* ctx, int nt, const double* times, double* h, int h_on_device, lt_stats* stats);

/*
 * Forward problems of n independent contexts (aquifers) solved together:
 * h[i] receives context i's float64 [ns_i][nr_i][nt[i]] measurements (all HOST
 * pointers if h_on_device == 0, else all DEVICE pointers); stats: NULL or an
 * array of n.  Each context keeps its own grid, wells and options; the
 * contexts' outer iterations are interleaved on their own streams so that the
 * GPU runs the aquifers concurrently (the batching layer of the engine).
 * Returns LT_ERR_NOT_CONVERGED if any context did not converge (all results
 * written), another error code on the first failing context.
 */
int lt_forward_batch(int n, lt_ctx* const* ctxs, const int* nt, const double* const* times, double* const* h,
                     int h_on_device, lt_stats* stats);

/*
 * Fields phi_s(t) on every cell (Eq. half), float64 [ns][nt][ncell], HOST or DEVICE as flagged.
 * Same solves as lt_forward.
 */
int lt_forward_fields(lt_ctx* ctx, int nt, const double* times, double* phi, int phi_on_device,
                      lt_stats* stats);

/*
 * Laplace-domain adjoint Jacobian (Sec. 5.2): for every (s, r, t)
 *   J[s][r][t][0][c] = d h[s][r][t] / d log kappa_c,   J[s][r][t][1][c] = d h[s][r][t] / d log Ss_c
 *   = -2 Re sum_k w_k (Q_s / z_k) psi_{r,k}^T (dK/dp + z_k dM/dp) x_{s,k},
 * psi_{r,k} = (K + z_k M)^{-1} e_{cell_r} (complex symmetric: transpose, not conjugate).
 *   J : float64 [ns][nr][nt][2][ncell], DEVICE pointer (the caller allocates it)
 */
int lt_adjoint_jacobian(lt_ctx* ctx, int nt, const double* times, double* J, lt_stats* stats);

/*
 * Vector-Jacobian product without materialising J:
 *   grad[p][c] = sum_{s,r,t} g[s][r][t] J[s][r][t][p][c]
 *   g    : float64 [ns][nr][nt], HOST pointer if on_device == 0 else DEVICE
 *   grad : float64 [2][ncell], same memory space as g
 * Also writes h (float64 [ns][nr][nt], same space) when h != NULL.
 */
int lt_adjoint_vjp(lt_ctx* ctx, int nt, const double* times, const double* g, double* grad,
                   double* h, int on_device, lt_stats* stats);

/*
 * Adjoint Jacobians (or vector-Jacobian products) of n independent contexts solved together, the
 * adjoint counterpart of lt_forward_batch: every context's source and receiver bases are built
 * with their outer iterations interleaved on the contexts' own streams, then each context's
 * sensitivities are assembled (Sec. 5.2, the formula of lt_adjoint_jacobian).  All pointers are
 * DEVICE pointers.  For context i:
 *   J[i] non-NULL (J itself non-NULL): the Jacobian float64 [ns][nr][nt][2][ncell] is written;
 *   otherwise the VJP: g[i] float64 [ns][nr][nt] in, grad[i] float64 [2][ncell] out.
 *   h: NULL or an array of n (entries may be NULL): the measurements float64 [ns][nr][nt].
 *   stats: NULL or an array of n.
 * Returns LT_ERR_NOT_CONVERGED if any context did not converge (all results written), another
 * error code on the first failing context.
 */
int lt_adjoint_batch(int n, lt_ctx* const* ctxs, const int* nt, const double* const* times, double* const* J,
                     const double* const* g, double* const* grad, double* const* h, lt_stats* stats);

/*
 * Crank-Nicolson time stepping of the same semi-discrete problem (the time-stepping method the
 * paper compares the Laplace-transform approach against, Sec. 1 and Sec. 5.3), from phi_0 (as set
 * by lt_set_initial_state, else 0) with the sources' rates (lt_set_sources / lt_set_source_rates):
 *   (M + dt/2 K) phi^{n+1} = (M - dt/2 K) phi^n + dt/2 (q(t_n) + q(t_{n+1})) e_s,
 * `steps` uniform steps between consecutive output times (and from 0 to the first), the first
 * step replaced by four backward-Euler quarter steps (Rannacher start, which damps the stiff
 * modes the step source excites).  Each step solves (K + (2/dt) M) phi^{n+1} = ... for all sources
 * together by FP64-residual iterative refinement around the float32 multigrid V-cycles
 * (inner_rounds rounds of inner_cycles V-cycles) to the relative residual opts.tol.
 *   times : HOST float64 [nt], strictly increasing, > 0;  steps in [2, 1e6]
 *   h     : float64 [ns][nr][nt], HOST pointer if h_on_device == 0, else DEVICE
 *   stats : n_shift_solves = steps x sources, max_true_residual = the largest step residual
 * Returns LT_ERR_NOT_CONVERGED (h written) if some step's solve stopped above tol.  The time
 * discretisation error is O(dt^2): two calls with steps and 2 steps allow Richardson extrapolation.
 */
int lt_crank_nicolson(lt_ctx* ctx, int nt, const double* times, int steps, double* h, int h_on_device,
                      lt_stats* stats);

/*
 * One iteration of the quasi-linear geostatistical inversion (Sec. 5.1, Algorithm 2) for
 * s = log kappa on the context's 2D grid, at the current coefficients s_k = log kappa (set by
 * lt_setup_grid), with the prior s ~ N(X beta, Q): X = the column of ones (one drift coefficient),
 * Q_ij = sigma2 exp(-|x_i - x_j| / ell) between cell centres (metres), and data y = h(s) + eps,
 * eps ~ N(0, diag(R)):
 *   J = d h / d s at s_k (the adjoint Jacobian, Sec. 5.2),
 *   [J Q J^T + R, J X; (J X)^T, 0] [xi; beta] = [y - h(s_k) + J s_k; 0],
 *   s_{k+1} = X beta + Q J^T xi,
 * with Q J^T formed by FFT on the circulant embedding of the covariance (exact, no truncation),
 * J Q J^T by an FP64 GEMM and the system through a Cholesky factorisation of J Q J^T + R.
 *   y, R   : HOST float64 [ns][nr][nt] (measurements, noise variances > 0)
 *   s_next : HOST float64 [ncell];  beta : HOST float64 [1]
 *   xi, h  : HOST float64 [ns][nr][nt] or NULL (the multipliers; h(s_k))
 * The caller iterates (lt_setup_grid with kappa = exp(s_next), then this call again).
 * Needs nz = 1 and nx, ny <= 1024.  Returns LT_ERR_NOT_CONVERGED (results written) if a shifted
 * solve of the Jacobian missed tol, LT_ERR_INVALID_ARG if J Q J^T + R is not positive definite.
 */
int lt_geostat_step(lt_ctx* ctx, int nt, const double* times, const double* y, const double* R, double sigma2,
                    double ell, double* s_next, double* beta, double* xi, double* h, lt_stats* stats);

/*
 * lt_forward without device allocation.  The paper has no counterpart: this
 * entry point exists for callers that cannot let a library call cudaMalloc or
 * cudaFree -- services that hand all device memory to their own pool allocator
 * up front (a library allocation would fail or fragment that pool), and
 * pipelines that keep other streams busy, where cudaMalloc/cudaFree may
 * synchronise the device and stall them.
 *
 * Same computation and result as lt_forward, but every device buffer the call
 * needs is taken from one fixed static region of LT_NOALLOC_SCRATCH_MAX bytes
 * inside the library, which each GPU that loads the library holds until the
 * process exits.  The grid, wells and options still come from lt_setup_grid,
 * lt_set_sources/receivers and lt_set_options (those calls do allocate).
 *   h     : float64 [ns][nr][nt], DEVICE pointer
 *   stats : optional; timing_class is ignored (no per-launch events)
 * Returns LT_ERR_INVALID_ARG, before launching anything, when the problem's
 * buffers exceed the static region (the message gives the bytes needed).
 * The first call on a device looks up the region's device address; make that
 * call before any stream capture.  All calls share the region and it keeps the
 * last call's contents (every buffer is re-initialised by the call that uses
 * it), so calls that overlap on the GPU -- from two threads, two contexts or
 * two streams -- race and must be serialised by the caller.
 */
#define LT_NOALLOC_SCRATCH_MAX (32u << 20)
int lt_forward_noalloc(lt_ctx* ctx, int nt, const double* times, double* h, lt_stats* stats);

/* ------------------------------------------------------------------------
 * Learned preconditioner (spec extension; no counterpart in the paper):
 * a small 2D U-Net (bf16 activations, tensor-core 3x3 convolutions, FP32
 * accumulation) that maps a residual of (K + tau M) u = r to an initial guess
 * for the multigrid iteration of the preconditioner solve.
 * Inputs of the network, float32 [nimg][H][W][5] DEVICE: Re r / s, Im r / s,
 * normalised log kappa, Re(tau) m / D, Im(tau) m / D (s = RMS of r, D = the
 * operator's diagonal); output float32 [nimg][H][W][2] DEVICE: the direction of
 * D u (unit RMS); the solver rescales it by the minimal-residual coefficient.
 * H and W must be multiples of 8.  Status: 0 or a negative LT_ERR_* code.
 * ------------------------------------------------------------------------ */
typedef struct lt_unet lt_unet;
int lt_unet_create(lt_unet** out, int device, unsigned long long seed);   /* He-initialised parameters */
int lt_unet_num_params(lt_unet* net);
int lt_unet_get_params(lt_unet* net, float* host, int n);    /* flat FP32: per layer W[9][cout][cin], b[cout] */
int lt_unet_set_params(lt_unet* net, const float* host, int n);
int lt_unet_forward(lt_unet* net, int nimg, int H, int W, const float* in, float* out);
/* loss = mean (out - target)^2 over pixels and the 2 channels; grad_host (HOST, may be NULL) receives d loss / d params */
int lt_unet_grad(lt_unet* net, int nimg, int H, int W, const float* in, const float* target, float* grad_host,
                 double* loss);
/* one Adam step (beta 0.9 / 0.999) on the batch */
int lt_unet_train_step(lt_unet* net, int nimg, int H, int W, const float* in, const float* target, float lr,
                       double* loss);
/* Poll limit of the bounded waits in the tensor-core convolutions (default 4,194,304 polls of the
 * mbarrier that the MMAs complete on).  A wait that reaches the limit raises an error flag, keeps
 * waiting (at most 16,777,216 more polls) until the MMAs in flight have finished, frees the block's
 * tensor memory and returns; the call then returns -5 (LT_ERR_TIMEOUT) and its outputs are not valid.
 * 0 makes every wait run out at once without any fault, which tests use to exercise that path.
 * The limit also applies while the solver runs the network (lt_set_learned_preconditioner), where a
 * timeout is reported as the solve's LT_ERR_TIMEOUT.  Returns 0, or -1 for a null network. */
int lt_unet_set_wait_polls(lt_unet* net, unsigned polls);
const char* lt_unet_last_error(lt_unet* net);
void lt_unet_destroy(lt_unet* net);

/*
 * Multigrid solves of (K + tau_i M) e_i = r_i on the context's grid: `cycles`
 * V-cycles from e = 0 (the preconditioner of Sec. 3's Algorithm 1 applied on
 * its own; used to generate training pairs).  tau: HOST float64 [nimg][2];
 * r, e: DEVICE complex float32 [nimg][ncell][2].
 */
int lt_precond_apply(lt_ctx* ctx, int nimg, const double* tau, const float* r, float* e, int cycles);

/*
 * Talbot nodes and weights of one output time (Sec. 2.2, Eq. half): the N_z/2 upper-half nodes
 * z_k and weights w_k, phi(t) = 2 Re sum_k w_k F(z_k).  project = 1 replaces Re z_k by
 * max(Re z_k, 0) (the rule lt_opts.tau_project applies to preconditioner shifts).
 *   z, w : HOST float64 [Nz/2][2] (re, im); w may be NULL.  No context, no device work.
 * LT_ERR_INVALID_ARG if t <= 0 or Nz is not even in [4, 128].
 */
int lt_contour_nodes(double t, int Nz, int project, double* z, double* w);

/*
 * Training pairs of the learned preconditioner on the context's grid: for residuals r_i and
 * shifts tau_i, the multigrid solution e_i of (K + tau_i M) e_i = r_i (`cycles` V-cycles, as
 * lt_precond_apply), then the network input x_i (the five channels listed above, the residual at
 * unit RMS) and the target y_i = D e_i at unit RMS, all computed on the device.
 *   tau : HOST float64 [nimg][2];  r : DEVICE complex float32 [nimg][ncell][2]
 *   x   : DEVICE float32 [nimg][ncell][5];  y : DEVICE float32 [nimg][ncell][2]
 */
int lt_learned_pairs(lt_ctx* ctx, int nimg, const double* tau, const float* r, int cycles, float* x, float* y);

/*
 * The Krylov vectors v_j of the context's last forward or adjoint solve, with the preconditioner
 * shift tau_j each was solved with (Algorithm 1: (K + tau_j M) u_j = v_j): these are the
 * residuals the preconditioner sees, used as training inputs.  Bases in order, j = 0 .. (outer
 * iterations of the basis) - 1, at most max_n vectors (the float32 hi plane of each).
 *   r   : DEVICE complex float32 [max_n][ncell][2];  tau : HOST float64 [max_n][2]
 *   n_out : number written.  LT_ERR_STATE if the context has not solved yet.
 */
int lt_krylov_vectors(lt_ctx* ctx, int max_n, float* r, double* tau, int* n_out);

/*
 * Attach a trained network (NULL detaches).  With lt_opts.precond = 1 the
 * first refinement round of every preconditioner solve (residual = the Krylov
 * vector v_j) starts its V-cycles from the network's guess (its direction scaled by the minimal-residual coefficient)
 * instead of zero; a guess that removes less than 5% of the residual norm is
 * dropped (multigrid fallback).  2D grids with nx, ny
 * multiples of 8 only.  The network must stay alive while attached.
 */
int lt_set_learned_preconditioner(lt_ctx* ctx, lt_unet* net);

/* Static description of a status code. */
const char* lt_strerror(int status);

/* Message of the last failing call on ctx ("" if none). */
const char* lt_last_error(lt_ctx* ctx);

/* Release the context and its device memory.  NULL is ignored. */
void lt_destroy(lt_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* LT_H */
