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
  Level h_levels[kMaxLevels];  // host copy of the level descriptors
  Level* d_levels;             // device copy
};

// one V-cycle on every active basis of the batch whose refinement round `round` is not done
int launch_vcycle(const MGHost& mg, const Batch& bt, int round, cudaStream_t st, int* nlaunch, Prof* pf);

// -------- krylov.cu
void launch_prep_iter(const Batch& bt, int j, cudaStream_t st);
void launch_exact_residual(const Batch& bt, const FineExact& fe, const Level& L0, int j, int round, int record_only,
                           cudaStream_t st, Prof* pf);
void launch_update_u(const Batch& bt, const Level& L0, int j, int round, cudaStream_t st);
void launch_inner_record(const Batch& bt, cudaStream_t st);
void launch_arnoldi(const Batch& bt, const FineExact& fe, int j, cudaStream_t st, int* nlaunch, Prof* pf);
void launch_shift_ls(const Batch& bt, int j, cudaStream_t st);
void launch_init_batch(const Batch& bt, cudaStream_t st);
void launch_backsolve_map(const Batch& bt, const int* sh_basis, cudaStream_t st);

// quadrature-fused measurement: C[q][i] = sum_{k in item q} wq[k] Y[k][i]; h = 2 Re U[rcell] . C
struct QuadItem {            // one (source-or-receiver, time) pair
  int basis;                 // basis that holds the time's shifts
  int sh0, nk;               // global index of its first shift, count
};
void launch_quad_coef(const Batch& bt, const QuadItem* items, int nitems, const double2* wq, double2* C,
                      cudaStream_t st);
// h[s][r][t]: item index q = s*nt + t
void launch_measure(const Batch& bt, const QuadItem* items, const double2* C, int ns, int nr, int nt,
                    const int64_t* rcells, double* h, cudaStream_t st);
void launch_fields(const Batch& bt, const QuadItem* items, const double2* C, int nitems, double* phi, cudaStream_t st);
// true residual of every shift: res2[sh] = ||e_cell - (K + z M) x_sh||^2, x_sh = U y_sh
void launch_true_residual_map(const Batch& bt, const FineExact& fe, const int* sh_basis, float2* X_hi,
                              float2* X_lo, double* res2, cudaStream_t st, int* nlaunch, Prof* pf);

// -------- adjoint.cu
struct SensItem {             // one Jacobian row group (s, r, t)
  int bs, br;                 // forward basis (source) and adjoint basis (receiver)
  int shs, shr;               // first shift of the time in each basis
  int nk;                     // shifts of the time
  int row;                    // output row index ((s*nr + r)*nt + t)
  double Qs;                  // source rate
};
struct SensGeom {             // fine-level derivative weights (double)
  int nx, ny, nz, N;
  const double *Te, *Tn, *Tu, *m;          // face transmissibilities and storage
  const double *kap;                        // kappa per cell
  const double *Bd;                         // Dirichlet boundary transmissibility sum per cell
};
void launch_sens(const Batch& fb, const Batch& rb, const SensGeom& sg, const SensItem* items, int nitems,
                 const double2* wz, const float2* Xs_hi, const float2* Xs_lo, const float2* Xr_hi,
                 const float2* Xr_lo, double* J, const double* g, double* grad, int mode, cudaStream_t st);

}  // namespace lt
