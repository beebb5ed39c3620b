// lt_kernels.h -- host-side launchers of the engine's kernels.
#pragma once
#include <cuda_runtime.h>
#include "lt_internal.h"

namespace lt {

struct MGHost {
  int nlev;                    // levels
  int lc;                      // first level handled by the single-CTA coarse kernel
  int npre, npost;             // smoothing sweeps
  int dmask;                   // Dirichlet faces bitmask (bit 2d: lower face of axis d, 2d+1: upper)
  int coarse_direct;           // 1 if the coarsest level has a dense inverse
  int tile;                    // fused 2D tile shape: 0 = 64x32, 1 = 32x32, 2 = 32x16
  int tma;                     // 1: stage fused tiles with TMA bulk tensor copies where alignment allows
  void* tma_cache;             // host-side cache of tensor maps (owned by mg.cu)
  Level h_levels[kMaxLevels];  // host copy of the level descriptors
  Level* d_levels;             // device copy
};

// -------- inner.cu: the whole preconditioner solve of a basis in one thread-block cluster
struct InnerPlan {
  int ok = 0;                      // 1 if the grid and the device allow the cluster-resident solve
  int cs = 8;                      // CTAs per cluster = row strips per strip level (8, or 16 non-portable)
  int threads = 512;               // threads per CTA
  int u0_global = 0;               // 1: finest-level iterates in a global [nb][N] array, not shared memory
  int ld = 0;                      // levels split into per-CTA row strips: [0, ld); [ld, nlev) in rank 0
  int max_clusters = 0;            // clusters the device can hold at once
  int off_u[kMaxLevels] = {}, off_f[kMaxLevels] = {};               // byte offsets in shared memory
  int off_te[kMaxLevels] = {}, off_tn[kMaxLevels] = {}, off_di[kMaxLevels] = {}, off_rhs = 0;
  size_t smem = 0;                 // dynamic shared memory per CTA
  const float4* p4 = nullptr;      // [N] finest-level faces (Te east, Te west, Tn north, Tn south), set by the host
};
// fills p for clusters of cs CTAs of `threads` threads (p.ok = 0 when the levels do not split into cs
// even row strips, do not fit in shared memory, or the device cannot hold such a cluster); returns p.ok
int inner_cluster_plan(const MGHost& mg, InnerPlan& p, int cs = 8, int threads = 512, int u0_global = 0);
// rounds x cycles V-cycles of every active basis, one cluster per basis (bt.rounds rounds)
// q4: [nb][N] float4 scratch of the finest level (inverse diagonal, right-hand side); u0: [nb][N] float2
// scratch of the finest-level iterates when p.u0_global (else unused)
int launch_inner_cluster(const MGHost& mg, const InnerPlan& p, const Batch& bt, const FineExact& fe, float4* q4,
                         float2* u0, int cycles, cudaStream_t st, Prof* pf);

// one V-cycle on every active basis of the batch whose refinement round `round` is not done
// u0_state: 1 if the finest level's iterate is zero on entry, 0 if it follows a previous cycle's
// post-smoothing (which ends with the red half-sweep), -1 if unknown
int launch_vcycle(const MGHost& mg, const Batch& bt, int round, cudaStream_t st, int* nlaunch, Prof* pf,
                  int u0_state = -1);
void tma_cache_free(MGHost& mg);

// -------- krylov.cu
void launch_prep_iter(const Batch& bt, int j, cudaStream_t st);
void launch_exact_residual(const Batch& bt, const FineExact& fe, const Level& L0, int j, int round, int record_only,
                           cudaStream_t st, Prof* pf);
void launch_update_u(const Batch& bt, const Level& L0, int j, int round, cudaStream_t st);
void launch_inner_record(const Batch& bt, cudaStream_t st);
void launch_arnoldi(const Batch& bt, const FineExact& fe, int j, cudaStream_t st, int* nlaunch, Prof* pf);
void launch_shift_ls(const Batch& bt, int j, cudaStream_t st);   // least squares, then the iteration counter
void launch_shift_ls_only(const Batch& bt, int j, cudaStream_t st);
void launch_next_iter(const Batch& bt, cudaStream_t st);
void launch_init_batch(const Batch& bt, cudaStream_t st);
// y_k for the shifts [s0, s1) (s1 < 0: every shift)
void launch_backsolve_map(const Batch& bt, const int* sh_basis, cudaStream_t st, int s0 = 0, int s1 = -1);

// quadrature-fused measurement: C[q][i] = sum_{k in item q} wq[k] Y[k][i]; h = 2 Re U[rcell] . C
struct QuadItem {            // one (source-or-receiver, time) pair
  int basis;                 // basis that holds the time's shifts
  int sh0, nk;               // global index of its first shift, count
};
void launch_quad_coef(const Batch& bt, const QuadItem* items, int nitems, const double2* wq, double2* C,
                      cudaStream_t st);
// h[s][r][t]: item index q = s*nt + t; dense_q0 >= 0: items dense_q0 + t (the initial-state basis)
// are added to every source's measurements (fields)
void launch_measure(const Batch& bt, const QuadItem* items, const double2* C, int ns, int nr, int nt,
                    const int64_t* rcells, double* h, cudaStream_t st, int dense_q0 = -1);
void launch_fields(const Batch& bt, const QuadItem* items, const double2* C, int nitems, double* phi, cudaStream_t st,
                   int nt = 1, int dense_q0 = -1);

// -------- adjoint.cu
struct SensLaunch {
  int ns, nr, nt, Nk;
  int64_t N;
  int nx, ny, nz;
  const int* sh_src;          // [nt][ns] first shift of (source s, time t)
  const int* sh_rec;          // [nt][nr] first shift of (receiver r, time t)
  const double2* omega;       // [nt][ns][Nk] w_k Q_s / z_k
  const double2* zk;          // [nt][Nk]
  const float2 *X_hi, *X_lo;  // [nsh][N] solutions per shift
  const double *Te, *Tn, *Tu, *kap, *Bd, *m;   // float64 fine-level geometry
  double* J;                  // mode 0: [ns][nr][nt][2][N]
  const double* g;            // mode 1: [ns][nr][nt]
  double* grad;               // mode 1: [2][N] (accumulated)
  int mode;
};
int launch_sens2(const SensLaunch& L, cudaStream_t st);

// -------- cn.cu: Crank-Nicolson time stepping (the paper's comparison method)
struct CnArgs {
  int nb;                                   // sources (one trajectory each)
  int64_t N;
  int nx, ny, nz;
  const double *Te, *Tn, *Tu, *D, *m;       // FP64 fine operator; m includes water-table storage
  double *phi, *x, *f;                      // [nb][N]: state, iterate of the step's solve, right-hand side
  const int64_t* cell;                      // [nb] source cell
  const double* srcw;                       // [steps][nb] source term of each step (q(t) + q(t + dt), or q(t + h))
  double* fnorm2;                           // [nb] ||f||^2 of the current step
  double* maxres2;                          // [1] largest relative residual^2 of any step and source
  int* step;                                // device step counter
  double tau, theta, tol;                   // (K + tau M) x = tau M phi - theta K phi + srcw e_cell
};
int launch_cn_step(const MGHost& mg, const Batch& bt, const CnArgs& a, int cycles, cudaStream_t st, int* nl);
void launch_cn_measure(const CnArgs& a, const int64_t* rcells, int nr, int nt, int t, double* h, cudaStream_t st);

// -------- geostat.cu: one iteration of the quasi-linear geostatistical inversion (Algorithm 2)
int geostat_prepare(int P0, int P1);
int geostat_spectrum(double2* cimg, double2* tmp, int P0, int P1, double* lam, cudaStream_t st);
int geostat_qjt(const double* J, size_t ldj, int row0, int nrows, int nx, int ny, int P0, int P1, const double* lam,
                double2* img, double2* tmp, double* G, cudaStream_t st);
int geostat_solve(const double* J, size_t ldj, const double* G, int ny, int N, const double* R, const double* s,
                  const double* y, const double* h, double* A, double* rhs, double* z, double* beta, double* xi,
                  double* s_next, int* flag, cudaStream_t st);
void launch_xk(const Batch& bt, float2* X_hi, float2* X_lo, cudaStream_t st, Prof* pf);
// squared true residuals of the shifts [s0, s1) into res2 (s1 < 0: every shift)
void launch_true_res(const Batch& bt, const FineExact& fe, const int* sh_basis, const float2* X_hi,
                     const float2* X_lo, double* res2, cudaStream_t st, Prof* pf, int s0 = 0, int s1 = -1);
// block.cu: block flexible GMRES over the sources of each group (Batch::block)
int launch_block_iteration(const Batch& bt, const FineExact& fe, cudaStream_t st, int* nlaunch, Prof* pf);
void launch_block_backsolve(const Batch& bt, const int* sh_basis, cudaStream_t st);
void launch_block_xk(const Batch& bt, float2* X_hi, float2* X_lo, cudaStream_t st, Prof* pf);
void launch_block_quad(const Batch& bt, const QuadItem* items, int nitems, const double2* wq, double2* C,
                       int ns, int nr, int nt, const int64_t* rcells, double* out, int fields, cudaStream_t st);

}  // namespace lt

// -------- unet.cu (learned initial guess of the preconditioner solves)
struct lt_unet;
int learned_prepare(lt_unet* u, int nb, int ny, int nx);
void learned_guess(lt_unet* u, const lt::Batch& bt, const lt::Level& L0, int round, const float* lk, const float* mD,
                   float* xin, float* gnorm2, cudaStream_t q);
void learned_pair_features(int nimg, int N, const float2* r, const float2* e, const double2* tau, const float* lk,
                           const float* mD, const float* D, double* acc, float* x, float* y, cudaStream_t q);

