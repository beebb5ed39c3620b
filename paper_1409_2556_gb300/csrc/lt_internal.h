// lt_internal.h -- device data structures shared by the kernels and the
// host driver of the Laplace-transform / flexible shifted-Krylov engine.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace lt {

constexpr int kMaxLevels = 16;

// offset into a df32 lo plane that may be absent (reduced precision: null stays null)
template <class T>
__host__ __device__ __forceinline__ T* lo_at(T* p, size_t off) { return p ? p + off : nullptr; }
constexpr int kCoarseCells = 1024;     // levels at or below this size run in one CTA per basis
constexpr int kDirectCells = 256;      // coarsest level solved by a dense inverse if at most this size
constexpr int kCoarseSweeps = 24;      // RB-GS sweeps at the coarsest level when it is not solved directly

// One multigrid level: fp32 coefficients of K_l and M_l.
struct Level {
  int nx, ny, nz, N;
  int rx, ry, rz;                  // coarsening ratio to the next level (1 or 2 per axis)
  float* Te;                       // face (i,j,k)-(i+1,j,k), 0 on the last column
  float* Tn;                       // face (i,j,k)-(i,j+1,k)
  float* Tu;                       // face (i,j,k)-(i,j,k+1)
  float* D;                        // sum of all face transmissibilities of the cell (incl. Dirichlet)
  float* m;                        // storage S_s * volume
  float2* u;                       // [nb][N] iterate / correction
  float2* f;                       // [nb][N] right-hand side
};

// Fine-level operator in df32 (hi/lo float pairs) for the exact residuals.
struct FineExact {
  int nx, ny, nz, N;
  const float *Te_hi, *Te_lo, *Tn_hi, *Tn_lo, *Tu_hi, *Tu_lo, *D_hi, *D_lo, *m_hi, *m_lo;
};

// Per-basis bookkeeping of a batch of Krylov bases.
struct Batch {
  int nb;                          // bases
  int maxit;                       // columns of U (V has maxit + 1)
  int64_t N;                       // fine cells
  int rounds;                      // refinement rounds per preconditioner solve
  double inner_tol2;               // (inner relative tolerance)^2, before relaxation
  double inner_relax_max;          // > 0: relax the inner tolerance as the outer residual falls, up to this
  double* itol2;                   // [nb] inner tolerance^2 of the current outer iteration
  double* rmax;                    // [nb] largest projected residual over the basis's unconverged shifts
  double tol;                      // outer tolerance (relative)
  float2 *V_hi, *V_lo;             // [nb][maxit+1][N]
  float2 *U_hi, *U_lo;             // [nb][maxit][N]
  float2 *S_hi, *S_lo;             // [nb][N] Arnoldi work vector
  double2* tau_grp;                // [ngroups][2] preconditioner shifts per group
  int* group;                      // [nb]
  int* tau_pattern;                // [5] slot per (j mod 5)
  double2* tau_cur;                // [nb] current preconditioner shift
  int* tau_slot;                   // [nb] current slot (0/1) for the coarse inverse
  double* rnorm2;                  // [nb][rounds+1]
  double2* dot;                    // [nb][2][maxit+1]
  double2* H;                      // [nb][maxit][maxit+1], column j at H + (b*maxit + j)*(maxit+1)
  double* snorm2;                  // [nb]
  int* active;                     // [nb]
  int* nit;                        // [nb] outer iterations done
  double* inner_max;               // [nb]
  int64_t* rhs_cell;               // [nb]
  // shifts: basis b owns shifts [shift_off[b], shift_off[b+1])
  int nsh;
  int* shift_off;                  // [nb+1]
  double2* zsh;                    // [nsh]
  double2* R;                      // [nsh][maxit][maxit]
  double* rc;                      // [nsh][maxit]
  double2* rs;                     // [nsh][maxit]
  double2* g;                      // [nsh][maxit+1]
  int* conv_it;                    // [nsh] iterations at convergence (0 = not yet)
  double* pres;                    // [nsh] projected residual
  double2* Y;                      // [nsh][maxit]
  float2* coarse_inv;              // [ngroups*2][nc*nc] dense inverses of the coarsest operator
  int coarse_direct;               // 1 if coarse_inv is valid
  unsigned long long* work;        // [kWorkSlots] cells processed per kernel class (live roofline), flags
  int* jdev;                       // current outer iteration (shared by all bases of the batch; [8]: one counter
                                   // per part when the parts of the batch run decoupled)
  unsigned tma_polls;              // mbarrier polls of a TMA tile load before it counts as timed out
  int krylov;                      // 0: GMRES-Sh coefficients, 1: FOM-Sh (Algorithm 1)
  int stop_rule;                   // 0: per shift; 1: per output time, quadrature-weighted residual
  int nk;                          // shifts per output time (a basis's shifts are nk per time, contiguous)
  int gs_passes;                   // Gram-Schmidt: 2 = CGS2 with float32 dots, 1 = one pass with df32 dots
  const double* wabs;              // [nsh] |w_k qhat(z_k)| of each shift (quadrature stopping rule)
  // right-hand side of the bases whose rhs_cell is negative: one dense vector of unit 2-norm
  // (M phi_0 / ||M phi_0||), df32 real
  const float* rhs_hi;
  const float* rhs_lo;
  // block flexible GMRES (block = 1): the bases q * ngroups + g, q < bp, of group g form one block
  int block;
  int bp;                          // right-hand sides per block
  int ngroups;                     // groups (blocks)
  int bld;                         // block columns maxit * bp
  int hld;                         // block rows (maxit + 1) * bp
  int nbs;                         // shifts per block, summed over blocks (= the member-0 shifts)
  double2* bdot;                   // [ngroups][2][bld][bp] Gram-Schmidt coefficients of both passes
  double2* bgram;                  // [ngroups][2][bp][bp] Gram matrices of the two CholQR passes
  float2* bw;                      // [ngroups][2][bp][bp] W = R^{-1} of the two passes, as applied
  double2* bH;                     // [ngroups][bld][hld] block Hessenberg, column-major
  double2* bR;                     // [nbs][bld][hld] rotated Hbar(z; T), column-major
  double* brc;                     // [nbs][bld][bp] rotation cosines (p per column)
  double2* brs;                    // [nbs][bld][bp] rotation sines
  double2* bG;                     // [nbs][hld][bp] rotated right-hand sides E_1
  double2* bY;                     // [nsh][bld] coefficients of each (shift, right-hand side)
  int* gany;                       // [ngroups] some (shift, rhs) of the block still open
  unsigned long long* grmax;       // [ngroups] largest open residual (bits of a non-negative double)
};

// kernel classes for the live per-kernel timing and work counters
enum KernelClass {
  KC_RBGS = 0, KC_RESTRICT, KC_PROLONG, KC_COARSE, KC_EXACT_RES, KC_UPDATE_U, KC_DOTS, KC_ORTHO, KC_NORMALIZE,
  KC_SHIFT_LS, KC_XK, KC_TRUE_RES, KC_FUSED_DOWN, KC_FUSED_UP, KC_OTHER, KC_INNER, kNumClasses
};
// Batch::work holds kWorkSlots counters: one per kernel class, then the
// error flag raised by a bounded device wait that expired.
constexpr int kTimeoutSlot = kNumClasses;
constexpr int kWorkSlots = 32;

// CUDA-event timing of the launches of one kernel class (cls < 0: off)
struct Prof {
  int cls = -1;
  int n = 0, cap = 0;
  cudaEvent_t* ev = nullptr;      // 2 * cap events
};
inline void prof_begin(Prof* p, int cls, cudaStream_t st) {
  if (p && p->cls == cls && p->n < p->cap) cudaEventRecord(p->ev[2 * p->n], st);
}
inline void prof_end(Prof* p, int cls, cudaStream_t st) {
  if (p && p->cls == cls && p->n < p->cap) { cudaEventRecord(p->ev[2 * p->n + 1], st); ++p->n; }
}

}  // namespace lt
