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
#define LT_BC_WATERTABLE 2        /* linearised water table; not supported in this version (INVALID_ARG) */

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
                           0: batched multigrid launches */
} lt_opts;

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
 *   bc        : 6 face codes (x-, x+, y-, y+, z-, z+), LT_BC_*
 *   Sy        : specific yield per top-face cell for water-table faces; must be NULL here
 * Face transmissibility between cells a, b: (area/dist) * 2 kappa_a kappa_b / (kappa_a + kappa_b);
 * a Dirichlet face adds 2 kappa_c area / dist to the diagonal; M = diag(Ss_c * dx dy dz).
 * Builds the multigrid hierarchy.  Each dimension must be 1 or >= 2, and repeated halving of the
 * even dimensions must reach at most 1024 cells.
 */
int lt_setup_grid(lt_ctx* ctx, int nx, int ny, int nz, double dx, double dy, double dz,
                  const double* kappa, const double* Ss, const int* bc, const double* Sy);

/* Point sources b_s = Q_s e_{cell_s}, constant rate switched on at t = 0, phi_0 = 0 (Sec. 2.1).
 * cells: HOST int64 [ns], each in [0, ncell); Q: HOST float64 [ns]. */
int lt_set_sources(lt_ctx* ctx, int ns, const int64_t* cells, const double* Q);

/* Point receivers (measurement cells, Sec. 5.2 functional I(t)).  cells: HOST int64 [nr]. */
int lt_set_receivers(lt_ctx* ctx, int nr, const int64_t* cells);

/* Replace the solver options (copied).  Invalid values give LT_ERR_INVALID_ARG. */
int lt_set_options(lt_ctx* ctx, const lt_opts* opts);

/*
 * Forward problem (Sec. 2.2 Eq. half and Sec. 3 Algorithm 1): for every
 * source s, receiver r and time t,
 *   h[s][r][t] = 2 Re sum_k w_k(t) (Q_s / z_k) x_{s,k}[cell_r],   (K + z_k M) x_{s,k} = e_{cell_s}
 * over the N_z/2 upper-half Talbot nodes of each time.
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
