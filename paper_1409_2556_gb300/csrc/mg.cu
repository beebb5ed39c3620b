// mg.cu -- geometric multigrid V-cycle for the complex-shifted operator
// K + tau M on the cell-centred finite-volume grid, in float32 complex.
//
// It is the inexact shift-and-invert preconditioner (K + tau_j M)^{-1} of
// the flexible shifted Krylov method (Sec. 3: the paper factorises these
// systems directly; here they are solved iteratively, see krylov.cu for the
// refinement that makes each solve accurate to the outer tolerance).
//
// Components:
//   * red-black Gauss-Seidel smoother (complex diagonal D + tau m);
//   * restriction = sum of the residual over the 2^d children;
//   * prolongation = cell-centred multilinear interpolation (weights 3/4,
//     1/4 per coarsened axis) with odd/even reflection across Dirichlet /
//     Neumann faces;
//   * coarse operators: T_coarse = (1/r) * sum of the fine faces crossing
//     the coarse face (r = ratio along the face normal), m_coarse = sum of
//     the children's m (built on the host);
//   * levels at or below kCoarseCells run inside one CTA per basis
//     (coarse_vcycle), ending in a dense inverse at the coarsest level.
// All kernels are batched over Krylov bases (blockIdx.y = basis) and skip
// bases that are inactive or whose preconditioner solve already converged.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstring>
#include <mutex>
#include <vector>

#include "lt_internal.h"
#include "lt_kernels.h"
#include "mg_dev.cuh"

namespace lt {

__device__ __forceinline__ bool mg_skip(const Batch& bt, int b, int round) {
  if (!bt.active[b]) return true;
  return bt.rnorm2[b * (bt.rounds + 1) + round] <= bt.itol2[b];
}

__device__ __forceinline__ float2 tau32(const Batch& bt, int b) {
  double2 t = bt.tau_cur[b];
  return make_float2((float)t.x, (float)t.y);
}

// ---------------------------------------------------------------- fine-level kernels
__global__ void k_rbgs(Level L, Batch bt, int round, int color) {
  int b = blockIdx.y;
  if (mg_skip(bt, b, round)) return;
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (threadIdx.x == 0) {
    int n = min((int)blockDim.x, L.N - (int)(blockIdx.x * blockDim.x));
    atomicAdd(&bt.work[KC_RBGS], (unsigned long long)n);
  }
  if (c >= L.N) return;
  int i = c % L.nx, j = (c / L.nx) % L.ny, k = c / (L.nx * L.ny);
  if (((i + j + k) & 1) != color) return;
  rbgs_cell(L, L.u + (size_t)b * L.N, L.f + (size_t)b * L.N, c, tau32(bt, b));
}

// Restriction of the residual to coarse cell C, evaluating only the fine cells that can carry one:
// kMgRestrictAll, kMgRestrictBlack (after a sweep ending with the red half-sweep the red cells
// satisfy their equations) or kMgRestrictZeroU (zero iterate: the residual is the right-hand side).
constexpr int kMgRestrictAll = 0, kMgRestrictBlack = 2, kMgRestrictZeroU = 3;
__global__ void k_restrict(Level Lf, Level Lc, Batch bt, int round, int mode) {
  int b = blockIdx.y;
  if (mg_skip(bt, b, round)) return;
  int C = blockIdx.x * blockDim.x + threadIdx.x;
  if (C >= Lc.N) return;
  const float2* uf = Lf.u + (size_t)b * Lf.N;
  const float2* ff = Lf.f + (size_t)b * Lf.N;
  if (mode == kMgRestrictAll) {
    restrict_cell(Lf, Lc, uf, ff, Lc.f + (size_t)b * Lc.N, Lc.u + (size_t)b * Lc.N, C, tau32(bt, b));
    return;
  }
  const float2 tau = tau32(bt, b);
  const int I = C % Lc.nx, J = (C / Lc.nx) % Lc.ny, K = C / (Lc.nx * Lc.ny);
  float2 acc = make_float2(0.f, 0.f);
  for (int dk = 0; dk < Lf.rz; ++dk)
    for (int dj = 0; dj < Lf.ry; ++dj)
      for (int di = 0; di < Lf.rx; ++di) {
        const int i = I * Lf.rx + di, j = J * Lf.ry + dj, k = K * Lf.rz + dk;
        const int c = (k * Lf.ny + j) * Lf.nx + i;
        float2 r;
        if (mode == kMgRestrictZeroU) {
          r = ff[c];
        } else {
          if (((i + j + k) & 1) == 0) continue;   // red: zero residual after the red half-sweep
          r = resid_cell(Lf, uf, ff, c, tau);
        }
        acc.x += r.x; acc.y += r.y;
      }
  Lc.f[(size_t)b * Lc.N + C] = acc;
  Lc.u[(size_t)b * Lc.N + C] = make_float2(0.f, 0.f);
}

__global__ void k_prolong(Level Lf, Level Lc, Batch bt, int round, int dmask) {
  int b = blockIdx.y;
  if (mg_skip(bt, b, round)) return;
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= Lf.N) return;
  prolong_cell(Lf, Lc, Lf.u + (size_t)b * Lf.N, Lc.u + (size_t)b * Lc.N, c, dmask);
}

// ---------------------------------------------------------------- coarse levels in one CTA
// levels[l0 .. nlev-1] are handled here; u at l0 is the current iterate (zero
// when l0 > 0, set by the restriction above), f at l0 the right-hand side.
__global__ void __launch_bounds__(1024) k_coarse_vcycle(const Level* __restrict__ levels, int l0, int nlev, Batch bt,
                                                        int round, int npre, int npost, int dmask, int nc_direct) {
  int b = blockIdx.x;
  if (mg_skip(bt, b, round)) return;
  float2 tau = tau32(bt, b);
  const int tid = threadIdx.x, nth = blockDim.x;
  if (tid == 0) atomicAdd(&bt.work[KC_COARSE], (unsigned long long)levels[l0].N);
  for (int l = l0; l < nlev - 1; ++l) {
    const Level L = levels[l];
    float2* u = L.u + (size_t)b * L.N;
    const float2* f = L.f + (size_t)b * L.N;
    for (int s = 0; s < npre; ++s)
      for (int color = 0; color < 2; ++color) {
        for (int c = tid; c < L.N; c += nth) {
          int i = c % L.nx, j = (c / L.nx) % L.ny, k = c / (L.nx * L.ny);
          if (((i + j + k) & 1) == color) rbgs_cell(L, u, f, c, tau);
        }
        __syncthreads();
      }
    const Level Lc = levels[l + 1];
    for (int C = tid; C < Lc.N; C += nth)
      restrict_cell(L, Lc, u, f, Lc.f + (size_t)b * Lc.N, Lc.u + (size_t)b * Lc.N, C, tau);
    __syncthreads();
  }
  {  // coarsest level
    const Level L = levels[nlev - 1];
    float2* u = L.u + (size_t)b * L.N;
    const float2* f = L.f + (size_t)b * L.N;
    if (nc_direct) {
      const float2* A = bt.coarse_inv + (size_t)bt.tau_slot[b] * L.N * L.N;
      for (int r = tid; r < L.N; r += nth) {
        float2 acc = make_float2(0.f, 0.f);
        const float2* row = A + (size_t)r * L.N;
        for (int c = 0; c < L.N; ++c) {
          float2 a = row[c], x = f[c];
          acc.x += a.x * x.x - a.y * x.y;
          acc.y += a.x * x.y + a.y * x.x;
        }
        u[r] = acc;
      }
      __syncthreads();
    } else {
      for (int s = 0; s < kCoarseSweeps; ++s)
        for (int color = 0; color < 2; ++color) {
          for (int c = tid; c < L.N; c += nth) {
            int i = c % L.nx, j = (c / L.nx) % L.ny, k = c / (L.nx * L.ny);
            if (((i + j + k) & 1) == color) rbgs_cell(L, u, f, c, tau);
          }
          __syncthreads();
        }
    }
  }
  for (int l = nlev - 2; l >= l0; --l) {
    const Level L = levels[l];
    const Level Lc = levels[l + 1];
    float2* u = L.u + (size_t)b * L.N;
    const float2* f = L.f + (size_t)b * L.N;
    for (int c = tid; c < L.N; c += nth) prolong_cell(L, Lc, u, Lc.u + (size_t)b * Lc.N, c, dmask);
    __syncthreads();
    for (int s = 0; s < npost; ++s)
      for (int color = 1; color >= 0; --color) {
        for (int c = tid; c < L.N; c += nth) {
          int i = c % L.nx, j = (c / L.nx) % L.ny, k = c / (L.nx * L.ny);
          if (((i + j + k) & 1) == color) rbgs_cell(L, u, f, c, tau);
        }
        __syncthreads();
      }
  }
}


// ---------------------------------------------------------------- fused 2D tile kernels
// For 2D levels coarsened 2x2, one CTA owns a kTX x kTY tile of fine cells and
// stages the tile plus a halo in shared memory.  A red-black half-sweep only
// reads the other colour, so updating the staged region reproduces the global
// sweep exactly on every cell whose neighbours were valid; each half-sweep
// shrinks the valid region by one ring.
//   down: pre-smoothing (npre sweeps) + residual + restriction (halo 2*npre+1)
//   up:   prolongation + correction + post-smoothing (halo 2*npost)
constexpr int kFusedThreads = 512;


struct Tile2D {
  float2* u;    // [RY][RX]
  float2* f;
  float2* di;   // inverse of the complex diagonal
  float* te;    // east-face transmissibility
  float* tn;    // north-face transmissibility
};

__device__ __forceinline__ void tile_load(const Level& L, const float2* u, const float2* f, float2 tau, Tile2D& T,
                                          int gx0, int gy0, int RX, int RY) {
  for (int idx = threadIdx.x; idx < RX * RY; idx += blockDim.x) {
    int lx = idx % RX, ly = idx / RX;
    int gx = gx0 + lx, gy = gy0 + ly;
    if (gx >= 0 && gx < L.nx && gy >= 0 && gy < L.ny) {
      int c = gy * L.nx + gx;
      T.u[idx] = u[c];
      T.f[idx] = f[c];
      T.te[idx] = L.Te[c];
      T.tn[idx] = L.Tn[c];
      float m = L.m[c];
      T.di[idx] = cinv(make_float2(L.D[c] + tau.x * m, tau.y * m));
    } else {
      T.u[idx] = make_float2(0.f, 0.f);
      T.f[idx] = make_float2(0.f, 0.f);
      T.te[idx] = 0.f;
      T.tn[idx] = 0.f;
      T.di[idx] = make_float2(0.f, 0.f);
    }
  }
}

__device__ __forceinline__ float2 tile_nb(const Tile2D& T, int idx, int RX) {
  float2 s;
  float a = T.te[idx], b = T.te[idx - 1], c = T.tn[idx], d = T.tn[idx - RX];
  float2 ue = T.u[idx + 1], uw = T.u[idx - 1], un = T.u[idx + RX], us = T.u[idx - RX];
  s.x = a * ue.x + b * uw.x + c * un.x + d * us.x;
  s.y = a * ue.y + b * uw.y + c * un.y + d * us.y;
  return s;
}

__device__ __forceinline__ void tile_sweeps(Tile2D& T, const Level& L, int gx0, int gy0, int RX, int RY, int nhalf,
                                            int first_color) {
  for (int h = 0; h < nhalf; ++h) {
    int color = (first_color + h) & 1;
    for (int idx = threadIdx.x; idx < RX * RY; idx += blockDim.x) {
      int lx = idx % RX, ly = idx / RX;
      if (lx < 1 || ly < 1 || lx > RX - 2 || ly > RY - 2) continue;
      int gx = gx0 + lx, gy = gy0 + ly;
      if (((gx + gy) & 1) != color) continue;
      if (gx < 0 || gy < 0 || gx >= L.nx || gy >= L.ny) continue;
      float2 r = tile_nb(T, idx, RX);
      float2 fc = T.f[idx];
      r.x += fc.x; r.y += fc.y;
      T.u[idx] = cmul(r, T.di[idx]);
    }
    __syncthreads();
  }
}

template <int kTX, int kTY>
__global__ void __launch_bounds__(kFusedThreads) k_down2d(Level Lf, Level Lc, Batch bt, int round, int npre) {
  extern __shared__ float4 smem4[];
  int b = blockIdx.y;
  if (mg_skip(bt, b, round)) return;
  const int H = 2 * npre + 1;
  const int RX = kTX + 2 * H, RY = kTY + 2 * H, RN = RX * RY;
  const int ntx = (Lf.nx + kTX - 1) / kTX;
  const int tx0 = (blockIdx.x % ntx) * kTX, ty0 = (blockIdx.x / ntx) * kTY;
  const int gx0 = tx0 - H, gy0 = ty0 - H;
  char* base = (char*)smem4;
  Tile2D T;
  T.u = (float2*)base; T.f = T.u + RN; T.di = T.f + RN;
  T.te = (float*)(T.di + RN); T.tn = T.te + RN;
  float2 tau = tau32(bt, b);
  float2* u = Lf.u + (size_t)b * Lf.N;
  const float2* f = Lf.f + (size_t)b * Lf.N;
  if (threadIdx.x == 0) {
    int n = min(kTX, Lf.nx - tx0) * min(kTY, Lf.ny - ty0);
    atomicAdd(&bt.work[KC_FUSED_DOWN], (unsigned long long)n);
  }
  tile_load(Lf, u, f, tau, T, gx0, gy0, RX, RY);
  __syncthreads();
  tile_sweeps(T, Lf, gx0, gy0, RX, RY, 2 * npre, 0);
  // residual + restriction of the tile's coarse cells; write the smoothed tile
  const int ncx = kTX / 2, ncy = kTY / 2;
  float2* fc = Lc.f + (size_t)b * Lc.N;
  float2* uc = Lc.u + (size_t)b * Lc.N;
  for (int q = threadIdx.x; q < ncx * ncy; q += blockDim.x) {
    int I = tx0 / 2 + q % ncx, J = ty0 / 2 + q / ncx;
    if (I >= Lc.nx || J >= Lc.ny) continue;
    float2 acc = make_float2(0.f, 0.f);
    for (int dj = 0; dj < 2; ++dj)
      for (int di = 0; di < 2; ++di) {
        int lx = H + 2 * (q % ncx) + di, ly = H + 2 * (q / ncx) + dj;
        int idx = ly * RX + lx;
        float2 nbs = tile_nb(T, idx, RX);
        float2 d = cinv(T.di[idx]);
        float2 a = cmul(d, T.u[idx]);
        float2 fv = T.f[idx];
        acc.x += fv.x - a.x + nbs.x;
        acc.y += fv.y - a.y + nbs.y;
      }
    fc[J * Lc.nx + I] = acc;
    uc[J * Lc.nx + I] = make_float2(0.f, 0.f);
  }
  for (int q = threadIdx.x; q < kTX * kTY; q += blockDim.x) {
    int gx = tx0 + q % kTX, gy = ty0 + q / kTX;
    if (gx >= Lf.nx || gy >= Lf.ny) continue;
    u[gy * Lf.nx + gx] = T.u[(H + q / kTX) * RX + H + q % kTX];
  }
}

template <int kTX, int kTY>
__global__ void __launch_bounds__(kFusedThreads) k_up2d(Level Lf, Level Lc, Batch bt, int round, int npost,
                                                       int dmask) {
  extern __shared__ float4 smem4[];
  int b = blockIdx.y;
  if (mg_skip(bt, b, round)) return;
  const int H = 2 * npost;
  const int RX = kTX + 2 * H, RY = kTY + 2 * H, RN = RX * RY;
  const int ntx = (Lf.nx + kTX - 1) / kTX;
  const int tx0 = (blockIdx.x % ntx) * kTX, ty0 = (blockIdx.x / ntx) * kTY;
  const int gx0 = tx0 - H, gy0 = ty0 - H;
  char* base = (char*)smem4;
  Tile2D T;
  T.u = (float2*)base; T.f = T.u + RN; T.di = T.f + RN;
  T.te = (float*)(T.di + RN); T.tn = T.te + RN;
  float2 tau = tau32(bt, b);
  float2* u = Lf.u + (size_t)b * Lf.N;
  const float2* f = Lf.f + (size_t)b * Lf.N;
  const float2* uc = Lc.u + (size_t)b * Lc.N;
  if (threadIdx.x == 0) {
    int n = min(kTX, Lf.nx - tx0) * min(kTY, Lf.ny - ty0);
    atomicAdd(&bt.work[KC_FUSED_UP], (unsigned long long)n);
  }
  tile_load(Lf, u, f, tau, T, gx0, gy0, RX, RY);
  __syncthreads();
  // prolongation + correction on the whole staged region
  for (int idx = threadIdx.x; idx < RN; idx += blockDim.x) {
    int gx = gx0 + idx % RX, gy = gy0 + idx / RX;
    if (gx < 0 || gy < 0 || gx >= Lf.nx || gy >= Lf.ny) continue;
    int I0, I1, J0, J1;
    float wi0, wi1, wj0, wj1, si, sj;
    axis_interp(gx, 2, Lc.nx, dmask & 1, dmask & 2, I0, I1, wi0, wi1, si);
    axis_interp(gy, 2, Lc.ny, dmask & 4, dmask & 8, J0, J1, wj0, wj1, sj);
    wi1 *= si; wj1 *= sj;
    float2 a = uc[J0 * Lc.nx + I0], bq = uc[J0 * Lc.nx + I1], c = uc[J1 * Lc.nx + I0], d = uc[J1 * Lc.nx + I1];
    float w00 = wj0 * wi0, w01 = wj0 * wi1, w10 = wj1 * wi0, w11 = wj1 * wi1;
    float2 v = T.u[idx];
    v.x += w00 * a.x + w01 * bq.x + w10 * c.x + w11 * d.x;
    v.y += w00 * a.y + w01 * bq.y + w10 * c.y + w11 * d.y;
    T.u[idx] = v;
  }
  __syncthreads();
  tile_sweeps(T, Lf, gx0, gy0, RX, RY, 2 * npost, 1);
  for (int q = threadIdx.x; q < kTX * kTY; q += blockDim.x) {
    int gx = tx0 + q % kTX, gy = ty0 + q / kTX;
    if (gx >= Lf.nx || gy >= Lf.ny) continue;
    u[gy * Lf.nx + gx] = T.u[(H + q / kTX) * RX + H + q % kTX];
  }
}

size_t fused_smem(int tx, int ty, int npre_or_post, bool down) {
  int H = down ? 2 * npre_or_post + 1 : 2 * npre_or_post;
  size_t RN = (size_t)(tx + 2 * H) * (ty + 2 * H);
  return RN * (3 * sizeof(float2) + 2 * sizeof(float));
}

// tile shapes selectable by MGHost::tile
static const int kTiles[3][2] = {{64, 32}, {32, 32}, {32, 16}};

template <int TX, int TY>
static void set_attrs() {
  cudaFuncSetAttribute(k_down2d<TX, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fused_smem(TX, TY, 8, true));
  cudaFuncSetAttribute(k_up2d<TX, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fused_smem(TX, TY, 8, false));
}

static void launch_down(int tile, const Level& L, const Level& Lc, const Batch& bt, int round, int npre, cudaStream_t st) {
  const int TX = kTiles[tile][0], TY = kTiles[tile][1];
  dim3 g(((L.nx + TX - 1) / TX) * ((L.ny + TY - 1) / TY), bt.nb);
  size_t sm = fused_smem(TX, TY, npre, true);
  if (tile == 0) k_down2d<64, 32><<<g, kFusedThreads, sm, st>>>(L, Lc, bt, round, npre);
  else if (tile == 1) k_down2d<32, 32><<<g, kFusedThreads, sm, st>>>(L, Lc, bt, round, npre);
  else k_down2d<32, 16><<<g, kFusedThreads, sm, st>>>(L, Lc, bt, round, npre);
}

static void launch_up(int tile, const Level& L, const Level& Lc, const Batch& bt, int round, int npost, int dmask,
                      cudaStream_t st) {
  const int TX = kTiles[tile][0], TY = kTiles[tile][1];
  dim3 g(((L.nx + TX - 1) / TX) * ((L.ny + TY - 1) / TY), bt.nb);
  size_t sm = fused_smem(TX, TY, npost, false);
  if (tile == 0) k_up2d<64, 32><<<g, kFusedThreads, sm, st>>>(L, Lc, bt, round, npost, dmask);
  else if (tile == 1) k_up2d<32, 32><<<g, kFusedThreads, sm, st>>>(L, Lc, bt, round, npost, dmask);
  else k_up2d<32, 16><<<g, kFusedThreads, sm, st>>>(L, Lc, bt, round, npost, dmask);
}

static bool fused_ok(const Level& L) { return L.nz == 1 && L.rx == 2 && L.ry == 2 && L.rz == 1; }


// ---------------------------------------------------------------- TMA-staged fused tiles
// The same fused kernels with the tile + halo brought into shared memory by
// one cp.async.bulk.tensor box per array (out-of-domain cells zero-filled by
// the copy engine), completing on an mbarrier.  The x origin of every box is
// the tile origin minus 8 cells (multiple of 8 elements, so the 16-byte rule
// holds for float and float2 planes); the y halo is what the sweeps need.
constexpr int kTmaHx = 8;
constexpr unsigned kTmaSpin = 1u << 26;   // bounded mbarrier wait (then an error flag is raised)

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void tma_2d(void* dst, const CUtensorMap* tm, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(smem_u32(dst)), "l"((uint64_t)tm), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tma_3d(void* dst, const CUtensorMap* tm, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(smem_u32(dst)), "l"((uint64_t)tm), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

struct TmaMaps { CUtensorMap u, f, te, tn, d, m; };

// stage u, f, Te, Tn, D, m of the region into shared memory and build the inverse diagonal.
// Returns false (and raises bt.work[kTimeoutSlot] as an error flag) if the copy did not complete
// within bt.tma_polls polls of the mbarrier.  Thread 0 alone polls and publishes the outcome in
// shared memory, so every thread of the block takes the same branch.  On a timeout thread 0
// keeps polling for up to kTmaSpin more tries before the block returns, so that copies still in
// flight land in shared memory that the block still owns.
__device__ __forceinline__ bool tile_load_tma(const TmaMaps& M, Tile2D& T, float* Ds, float* ms, uint64_t* bar,
                                              int gx0, int gy0, int b, int RX, int RY, float2 tau, const Batch& bt) {
  __shared__ int s_landed;
  const int RN = RX * RY;
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_expect_tx(bar, (uint32_t)RN * 32u);
    tma_3d(T.u, &M.u, gx0, gy0, b, bar);
    tma_3d(T.f, &M.f, gx0, gy0, b, bar);
    tma_2d(T.te, &M.te, gx0, gy0, bar);
    tma_2d(T.tn, &M.tn, gx0, gy0, bar);
    tma_2d(Ds, &M.d, gx0, gy0, bar);
    tma_2d(ms, &M.m, gx0, gy0, bar);
    int landed = 0;
    for (unsigned it = 0; it < bt.tma_polls; ++it)
      if (mbar_try_wait(bar, 0)) { landed = 1; break; }
    if (!landed) {
      atomicAdd(&bt.work[kTimeoutSlot], 1ull);
      for (unsigned it = 0; it < kTmaSpin; ++it)    // drain: let the copies in flight land
        if (mbar_try_wait(bar, 0)) break;
    }
    s_landed = landed;
  }
  __syncthreads();
  if (!s_landed) return false;
  for (int idx = threadIdx.x; idx < RN; idx += blockDim.x) {
    float dd = Ds[idx], mm = ms[idx];
    float2 dg = make_float2(dd + tau.x * mm, tau.y * mm);
    T.di[idx] = (dd == 0.f && mm == 0.f) ? make_float2(0.f, 0.f) : cinv(dg);
  }
  __syncthreads();
  return true;
}

template <int kTX, int kTY>
__global__ void __launch_bounds__(kFusedThreads) k_down2d_tma(Level Lf, Level Lc, Batch bt, int round, int npre,
                                                             const __grid_constant__ TmaMaps M) {
  extern __shared__ __align__(128) unsigned char smem_t[];
  int b = blockIdx.y;
  if (mg_skip(bt, b, round)) return;
  const int H = 2 * npre + 1;
  const int RX = kTX + 2 * kTmaHx, RY = kTY + 2 * H, RN = RX * RY;
  const int ntx = (Lf.nx + kTX - 1) / kTX;
  const int tx0 = (blockIdx.x % ntx) * kTX, ty0 = (blockIdx.x / ntx) * kTY;
  const int gx0 = tx0 - kTmaHx, gy0 = ty0 - H;
  const size_t A = ((size_t)RN * 8 + 127) & ~(size_t)127, B4 = ((size_t)RN * 4 + 127) & ~(size_t)127;
  Tile2D T;
  T.u = (float2*)smem_t; T.f = (float2*)(smem_t + A); T.di = (float2*)(smem_t + 2 * A);
  T.te = (float*)(smem_t + 3 * A); T.tn = (float*)(smem_t + 3 * A + B4);
  float* Ds = (float*)(smem_t + 3 * A + 2 * B4);
  float* ms = (float*)(smem_t + 3 * A + 3 * B4);
  uint64_t& bar = *(uint64_t*)(smem_t + 3 * A + 4 * B4);
  float2 tau = tau32(bt, b);
  if (threadIdx.x == 0) {
    int n = min(kTX, Lf.nx - tx0) * min(kTY, Lf.ny - ty0);
    atomicAdd(&bt.work[KC_FUSED_DOWN], (unsigned long long)n);
  }
  if (!tile_load_tma(M, T, Ds, ms, &bar, gx0, gy0, b, RX, RY, tau, bt)) return;
  tile_sweeps(T, Lf, gx0, gy0, RX, RY, 2 * npre, 0);
  const int ncx = kTX / 2, ncy = kTY / 2;
  float2* fc = Lc.f + (size_t)b * Lc.N;
  float2* uc = Lc.u + (size_t)b * Lc.N;
  for (int q = threadIdx.x; q < ncx * ncy; q += blockDim.x) {
    int I = tx0 / 2 + q % ncx, J = ty0 / 2 + q / ncx;
    if (I >= Lc.nx || J >= Lc.ny) continue;
    float2 acc = make_float2(0.f, 0.f);
    for (int dj = 0; dj < 2; ++dj)
      for (int di = 0; di < 2; ++di) {
        int lx = kTmaHx + 2 * (q % ncx) + di, ly = H + 2 * (q / ncx) + dj;
        int idx = ly * RX + lx;
        float2 nbs = tile_nb(T, idx, RX);
        float2 d = cinv(T.di[idx]);
        float2 a = cmul(d, T.u[idx]);
        float2 fv = T.f[idx];
        acc.x += fv.x - a.x + nbs.x;
        acc.y += fv.y - a.y + nbs.y;
      }
    fc[J * Lc.nx + I] = acc;
    uc[J * Lc.nx + I] = make_float2(0.f, 0.f);
  }
  float2* u = Lf.u + (size_t)b * Lf.N;
  for (int q = threadIdx.x; q < kTX * kTY; q += blockDim.x) {
    int gx = tx0 + q % kTX, gy = ty0 + q / kTX;
    if (gx >= Lf.nx || gy >= Lf.ny) continue;
    u[gy * Lf.nx + gx] = T.u[(H + q / kTX) * RX + kTmaHx + q % kTX];
  }
}

template <int kTX, int kTY>
__global__ void __launch_bounds__(kFusedThreads) k_up2d_tma(Level Lf, Level Lc, Batch bt, int round, int npost,
                                                           int dmask, const __grid_constant__ TmaMaps M) {
  extern __shared__ __align__(128) unsigned char smem_t[];
  int b = blockIdx.y;
  if (mg_skip(bt, b, round)) return;
  const int H = 2 * npost;
  const int RX = kTX + 2 * kTmaHx, RY = kTY + 2 * H, RN = RX * RY;
  const int ntx = (Lf.nx + kTX - 1) / kTX;
  const int tx0 = (blockIdx.x % ntx) * kTX, ty0 = (blockIdx.x / ntx) * kTY;
  const int gx0 = tx0 - kTmaHx, gy0 = ty0 - H;
  const size_t A = ((size_t)RN * 8 + 127) & ~(size_t)127, B4 = ((size_t)RN * 4 + 127) & ~(size_t)127;
  Tile2D T;
  T.u = (float2*)smem_t; T.f = (float2*)(smem_t + A); T.di = (float2*)(smem_t + 2 * A);
  T.te = (float*)(smem_t + 3 * A); T.tn = (float*)(smem_t + 3 * A + B4);
  float* Ds = (float*)(smem_t + 3 * A + 2 * B4);
  float* ms = (float*)(smem_t + 3 * A + 3 * B4);
  uint64_t& bar = *(uint64_t*)(smem_t + 3 * A + 4 * B4);
  float2 tau = tau32(bt, b);
  const float2* ucb = Lc.u + (size_t)b * Lc.N;
  if (threadIdx.x == 0) {
    int n = min(kTX, Lf.nx - tx0) * min(kTY, Lf.ny - ty0);
    atomicAdd(&bt.work[KC_FUSED_UP], (unsigned long long)n);
  }
  if (!tile_load_tma(M, T, Ds, ms, &bar, gx0, gy0, b, RX, RY, tau, bt)) return;
  for (int idx = threadIdx.x; idx < RN; idx += blockDim.x) {
    int gx = gx0 + idx % RX, gy = gy0 + idx / RX;
    if (gx < 0 || gy < 0 || gx >= Lf.nx || gy >= Lf.ny) continue;
    int I0, I1, J0, J1;
    float wi0, wi1, wj0, wj1, si, sj;
    axis_interp(gx, 2, Lc.nx, dmask & 1, dmask & 2, I0, I1, wi0, wi1, si);
    axis_interp(gy, 2, Lc.ny, dmask & 4, dmask & 8, J0, J1, wj0, wj1, sj);
    wi1 *= si; wj1 *= sj;
    float2 a = ucb[J0 * Lc.nx + I0], bq = ucb[J0 * Lc.nx + I1], c = ucb[J1 * Lc.nx + I0], d = ucb[J1 * Lc.nx + I1];
    float w00 = wj0 * wi0, w01 = wj0 * wi1, w10 = wj1 * wi0, w11 = wj1 * wi1;
    float2 v = T.u[idx];
    v.x += w00 * a.x + w01 * bq.x + w10 * c.x + w11 * d.x;
    v.y += w00 * a.y + w01 * bq.y + w10 * c.y + w11 * d.y;
    T.u[idx] = v;
  }
  __syncthreads();
  tile_sweeps(T, Lf, gx0, gy0, RX, RY, 2 * npost, 1);
  float2* u = Lf.u + (size_t)b * Lf.N;
  for (int q = threadIdx.x; q < kTX * kTY; q += blockDim.x) {
    int gx = tx0 + q % kTX, gy = ty0 + q / kTX;
    if (gx >= Lf.nx || gy >= Lf.ny) continue;
    u[gy * Lf.nx + gx] = T.u[(H + q / kTX) * RX + kTmaHx + q % kTX];
  }
}

static size_t tma_smem(int tx, int ty, int H) {
  size_t RN = (size_t)(tx + 2 * kTmaHx) * (ty + 2 * H);
  size_t A = (RN * 8 + 127) & ~(size_t)127, B4 = (RN * 4 + 127) & ~(size_t)127;
  return 3 * A + 4 * B4 + 16;   // + mbarrier
}

// ---- host: tensor maps (cached per level, tile, halo and workspace)
struct TmaEntry {
  const void *u, *f, *te;
  int nb, lvl, tile, H;
  TmaMaps maps;
};
struct TmaCache { std::vector<TmaEntry> e; };

static PFN_cuTensorMapEncodeTiled_v12000 get_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  });
  return fn;
}

static bool encode(CUtensorMap* tm, const void* base, CUtensorMapDataType dt, int rank, const cuuint64_t* dims,
                   const cuuint64_t* strides, const cuuint32_t* box) {
  auto fn = get_encoder();
  if (!fn) return false;
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = fn(tm, dt, rank, const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// maps for level l with tile shape (tx, ty) and y-halo H, or nullptr if TMA cannot be used
static const TmaMaps* tma_maps(const MGHost& mg, int l, int tile, int tx, int ty, int H, int nb) {
  const Level& L = mg.h_levels[l];
  if (!mg.tma || L.nx % 4 != 0 || H > kTmaHx || ty + 2 * H > 256) return nullptr;
  auto* cache = (TmaCache*)mg.tma_cache;
  if (!cache) return nullptr;
  for (auto& e : cache->e)
    if (e.u == L.u && e.f == L.f && e.te == L.Te && e.nb == nb && e.lvl == l && e.tile == tile && e.H == H)
      return &e.maps;
  TmaEntry e{L.u, L.f, L.Te, nb, l, tile, H, {}};
  const cuuint32_t RX = tx + 2 * kTmaHx, RY = ty + 2 * H;
  cuuint64_t d3[3] = {(cuuint64_t)L.nx, (cuuint64_t)L.ny, (cuuint64_t)nb};
  cuuint64_t s3[2] = {(cuuint64_t)L.nx * 8, (cuuint64_t)L.nx * L.ny * 8};
  cuuint32_t b3[3] = {RX, RY, 1};
  cuuint64_t d2[2] = {(cuuint64_t)L.nx, (cuuint64_t)L.ny};
  cuuint64_t s2[1] = {(cuuint64_t)L.nx * 4};
  cuuint32_t b2[2] = {RX, RY};
  bool ok = encode(&e.maps.u, L.u, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, d3, s3, b3) &&
            encode(&e.maps.f, L.f, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, d3, s3, b3) &&
            encode(&e.maps.te, L.Te, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, d2, s2, b2) &&
            encode(&e.maps.tn, L.Tn, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, d2, s2, b2) &&
            encode(&e.maps.d, L.D, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, d2, s2, b2) &&
            encode(&e.maps.m, L.m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, d2, s2, b2);
  if (!ok) return nullptr;
  cache->e.push_back(e);
  return &cache->e.back().maps;
}

void tma_cache_free(MGHost& mg) {
  delete (TmaCache*)mg.tma_cache;
  mg.tma_cache = nullptr;
}

template <int TX, int TY>
static void set_attrs_tma() {
  cudaFuncSetAttribute(k_down2d_tma<TX, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tma_smem(TX, TY, 7));
  cudaFuncSetAttribute(k_up2d_tma<TX, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tma_smem(TX, TY, 8));
}

static bool launch_down_tma(const MGHost& mg, int l, int tile, const Level& L, const Level& Lc, const Batch& bt,
                            int round, int npre, cudaStream_t st) {
  const int TX = kTiles[tile][0], TY = kTiles[tile][1], H = 2 * npre + 1;
  const TmaMaps* M = tma_maps(mg, l, tile, TX, TY, H, bt.nb);
  if (!M) return false;
  dim3 g(((L.nx + TX - 1) / TX) * ((L.ny + TY - 1) / TY), bt.nb);
  size_t sm = tma_smem(TX, TY, H);
  if (tile == 0) k_down2d_tma<64, 32><<<g, kFusedThreads, sm, st>>>(L, Lc, bt, round, npre, *M);
  else if (tile == 1) k_down2d_tma<32, 32><<<g, kFusedThreads, sm, st>>>(L, Lc, bt, round, npre, *M);
  else k_down2d_tma<32, 16><<<g, kFusedThreads, sm, st>>>(L, Lc, bt, round, npre, *M);
  return true;
}

static bool launch_up_tma(const MGHost& mg, int l, int tile, const Level& L, const Level& Lc, const Batch& bt,
                          int round, int npost, int dmask, cudaStream_t st) {
  const int TX = kTiles[tile][0], TY = kTiles[tile][1], H = 2 * npost;
  const TmaMaps* M = tma_maps(mg, l, tile, TX, TY, H, bt.nb);
  if (!M) return false;
  dim3 g(((L.nx + TX - 1) / TX) * ((L.ny + TY - 1) / TY), bt.nb);
  size_t sm = tma_smem(TX, TY, H);
  if (tile == 0) k_up2d_tma<64, 32><<<g, kFusedThreads, sm, st>>>(L, Lc, bt, round, npost, dmask, *M);
  else if (tile == 1) k_up2d_tma<32, 32><<<g, kFusedThreads, sm, st>>>(L, Lc, bt, round, npost, dmask, *M);
  else k_up2d_tma<32, 16><<<g, kFusedThreads, sm, st>>>(L, Lc, bt, round, npost, dmask, *M);
  return true;
}

// ---------------------------------------------------------------- host launcher
int launch_vcycle(const MGHost& mg, const Batch& bt, int round, cudaStream_t st, int* nlaunch, Prof* pf,
                  int u0_state) {
  const int nb = bt.nb;
  const int T = 256;
  static bool attr_done = false;
  if (!attr_done) {
    set_attrs<64, 32>();
    set_attrs<32, 32>();
    set_attrs<32, 16>();
    set_attrs_tma<64, 32>();
    set_attrs_tma<32, 32>();
    set_attrs_tma<32, 16>();
    attr_done = true;
  }
  if (mg.tma && !mg.tma_cache) const_cast<MGHost&>(mg).tma_cache = new TmaCache();
  const int tile = (mg.tile >= 0 && mg.tile < 3) ? mg.tile : 2;
  for (int l = 0; l < mg.lc; ++l) {
    const Level& L = mg.h_levels[l];
    const Level& Lc = mg.h_levels[l + 1];
    if (fused_ok(L) && mg.npre > 0) {
      prof_begin(pf, KC_FUSED_DOWN, st);
      if (!launch_down_tma(mg, l, tile, L, Lc, bt, round, mg.npre, st)) launch_down(tile, L, Lc, bt, round, mg.npre, st);
      prof_end(pf, KC_FUSED_DOWN, st);
      ++*nlaunch;
      continue;
    }
    dim3 g((L.N + T - 1) / T, nb);
    for (int s = 0; s < mg.npre; ++s)
      for (int color = 0; color < 2; ++color) {
        prof_begin(pf, KC_RBGS, st);
        k_rbgs<<<g, T, 0, st>>>(L, bt, round, color);
        prof_end(pf, KC_RBGS, st);
        ++*nlaunch;
      }
    dim3 gc((Lc.N + T - 1) / T, nb);
    // without pre-smoothing the coarser levels enter with the zero iterate the restriction above
    // left them; the finest level as the caller says (u0_state)
    int mode = kMgRestrictAll;
    if (mg.npre == 0) {
      if (l > 0 || u0_state == 1) mode = kMgRestrictZeroU;
      // (exact only after the plain half-sweeps: the fused tiles' asynchronous halo leaves small red
      // residuals at tile edges)
      else if (u0_state == 0 && mg.npost > 0 && !fused_ok(L)) mode = kMgRestrictBlack;
    }
    prof_begin(pf, KC_RESTRICT, st);
    k_restrict<<<gc, T, 0, st>>>(L, Lc, bt, round, mode); ++*nlaunch;
    prof_end(pf, KC_RESTRICT, st);
  }
  int thr = mg.h_levels[mg.lc].N >= 1024 ? 1024 : ((mg.h_levels[mg.lc].N + 31) / 32) * 32;
  if (thr < 64) thr = 64;
  prof_begin(pf, KC_COARSE, st);
  k_coarse_vcycle<<<nb, thr, 0, st>>>(mg.d_levels, mg.lc, mg.nlev, bt, round, mg.npre, mg.npost, mg.dmask,
                                      mg.coarse_direct);
  prof_end(pf, KC_COARSE, st);
  ++*nlaunch;
  for (int l = mg.lc - 1; l >= 0; --l) {
    const Level& L = mg.h_levels[l];
    const Level& Lc = mg.h_levels[l + 1];
    if (fused_ok(L) && mg.npost > 0) {
      prof_begin(pf, KC_FUSED_UP, st);
      if (!launch_up_tma(mg, l, tile, L, Lc, bt, round, mg.npost, mg.dmask, st))
        launch_up(tile, L, Lc, bt, round, mg.npost, mg.dmask, st);
      prof_end(pf, KC_FUSED_UP, st);
      ++*nlaunch;
      continue;
    }
    dim3 g((L.N + T - 1) / T, nb);
    prof_begin(pf, KC_PROLONG, st);
    k_prolong<<<g, T, 0, st>>>(L, Lc, bt, round, mg.dmask); ++*nlaunch;
    prof_end(pf, KC_PROLONG, st);
    for (int s = 0; s < mg.npost; ++s)
      for (int color = 1; color >= 0; --color) {
        prof_begin(pf, KC_RBGS, st);
        k_rbgs<<<g, T, 0, st>>>(L, bt, round, color);
        prof_end(pf, KC_RBGS, st);
        ++*nlaunch;
      }
  }
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

}  // namespace lt
