// unet.cu -- small 2D U-Net used as a learned initial guess for the
// preconditioner solves (K + tau M) u = r (the multigrid V-cycle stays as the
// convergent iteration and the fallback).
//
// Activations are NHWC bfloat16, convolutions 3x3 (padding 1) run on the
// 5th-generation tensor cores (tcgen05.mma, bf16 operands in shared memory,
// FP32 accumulator in tensor memory) as implicit GEMMs
// (M = 128 pixels, N = output channels, K = 9 taps x input channels); the
// backward-data pass is the same kernel with spatially flipped, transposed
// weights; the weight gradient is an FP32 reduction over pixels.
// Parameters are FP32 masters with Adam; bf16 copies feed the kernels.
//
// Network (base width c = 16, channel counts padded to multiples of 16):
//   enc0: conv(16->c) relu, conv(c->c) relu = s0        (input: 5 channels padded to 16)
//   enc1: pool, conv(c->2c) relu, conv(2c->2c) relu = s1
//   enc2: pool, conv(2c->2c) relu, conv(2c->2c) relu = s2
//   bott: pool, conv(2c->4c) relu, conv(4c->4c) relu = b
//   dec2: up(b) ++ s2 -> conv(6c->2c) relu, conv(2c->2c) relu = d2
//   dec1: up(d2) ++ s1 -> conv(4c->2c) relu, conv(2c->2c) relu = d1
//   dec0: up(d1) ++ s0 -> conv(3c->c) relu, conv(c->c) relu = d0
//   out : conv(c->16) linear (channels 0, 1 used)
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "lt_internal.h"

namespace lt {

using bf16 = __nv_bfloat16;

// ------------------------------------------------------------------ layer table
struct ConvSpec { int cin, cout, relu; };
static const ConvSpec kLayers[15] = {
    {16, 16, 1}, {16, 16, 1},      // enc0
    {16, 32, 1}, {32, 32, 1},      // enc1
    {32, 32, 1}, {32, 32, 1},      // enc2
    {32, 64, 1}, {64, 64, 1},      // bottleneck
    {96, 32, 1}, {32, 32, 1},      // dec2
    {64, 32, 1}, {32, 32, 1},      // dec1
    {48, 16, 1}, {16, 16, 1},      // dec0
    {16, 16, 0}};                  // output (linear)
constexpr int kNumLayers = 15;
constexpr int kInChannels = 5;     // re r, im r, log kappa (normalised), Re(tau) m/D, Im(tau) m/D
constexpr int kOutChannels = 2;

// ------------------------------------------------------------------ tensor-core 3x3 convolution (tcgen05)
// out[img][p][co] = act(bias[co] + sum_{tap,ci} in[img][p + off(tap)][ci] * W[tap][co][ci]) as an
// implicit GEMM on the 5th-generation tensor cores: for each of the 9 taps,
//   D (128 pixels x cout, FP32, tensor memory) += A_tap (128 pixels x cin, bf16) * B_tap^T (cout x cin, bf16)
// with one tcgen05.mma (M = 128, N = cout, K = 16) per 16 input channels, issued by one thread.
// Both operands sit in shared memory in the canonical K-major layout without swizzle: "core
// matrices" of 8 rows x 16 bytes (8 bf16), 128 contiguous bytes each; a matrix descriptor gives
// the byte step between core matrices along K (leading byte offset, LBO) and between groups of 8
// rows (stride byte offset, SBO), so the 8-row groups need not be adjacent.
// Epilogue: warp w reads tensor-memory lanes 32w..32w+31 with tcgen05.ld, adds the bias, applies
// the ReLU and stores bf16 or FP32 rows of 8 channels.
// Every mbarrier wait is bounded: a wait that runs out raises *flag, then waits (again bounded)
// for the MMAs in flight before the block frees its tensor memory and returns.
// in: [nimg][H][W][cin], W: [9][cout][cin]; cin, cout multiples of 16, cin <= 96, cout <= 96.
constexpr int kTcPix = 128;                   // MMA M = tensor-memory lanes = threads per CTA
constexpr unsigned kTcPolls = 1u << 22;       // default mbarrier polls before a wait counts as timed out
constexpr unsigned kTcDrain = 1u << 24;       // further polls for the MMAs in flight after a timeout

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint32_t pack_bf2(float lo, float hi) {
  __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&h);
}

__device__ __forceinline__ bool tc_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
  return ok != 0;
}

// bounded wait for the phase of the given parity; all threads take it, none branches on the outcome
__device__ __forceinline__ void tc_wait(uint32_t bar, uint32_t parity, unsigned polls, unsigned long long* flag) {
  for (unsigned it = 0; it < polls; ++it)
    if (tc_try_wait(bar, parity)) return;
  if (flag) atomicAdd(flag, 1ull);
  for (unsigned it = 0; it < kTcDrain; ++it)
    if (tc_try_wait(bar, parity)) return;
}

// shared-memory matrix descriptor: start address, LBO, SBO (all >> 4), descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t tc_sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
         (1ull << 46);
}

// instruction descriptor of kind::f16: FP32 accumulator, bf16 A and B, both K-major, N x M = n x 128
__device__ __forceinline__ uint32_t tc_idesc(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kTcPix >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
      ::"r"(tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(acc) : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tc_ld8(uint32_t taddr, float* v) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int q = 0; q < 8; ++q) v[q] = __uint_as_float(r[q]);
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// A CTA computes an output tile of 16 image rows x 8 MB columns as MB "M-blocks" of 16 rows x 8
// columns (128 pixels = the MMA's M; a group of 8 rows of the MMA is one image row of the block).
// It stages the tile's halo -- 18 rows x (8 MB + 2) positions, zero outside the image -- once, one
// 16-byte chunk of 8 channels per cp.async, as [cin/8 planes][18][8 MB + 2][8 channels]; the A
// operand of tap (dy, dx) for M-block mb is then the same halo seen through a shifted descriptor:
//   start = plane 0 + ((dy + 1)(8 MB + 2) + 8 mb + dx + 1) x 16 B, SBO = (8 MB + 2) x 16 B (the
//   halo row), LBO = one plane (the next 8 channels)
// so all 9 taps x cin / 16 MMAs of every M-block are issued back to back after one barrier.  The
// weights of all taps are staged in the same way: B per tap [cin/8][cout/8][8][8], LBO = 16 cout,
// SBO = 128.  M-block mb accumulates in tensor-memory columns [mb cout, (mb + 1) cout).
__host__ __device__ constexpr int tc_mb(int cout) { return cout <= 32 ? 4 : cout <= 64 ? 2 : 1; }
__host__ __device__ constexpr int tc_hc(int mb) { return 8 * mb + 2; }                 // halo positions per row
__host__ __device__ constexpr size_t tc_plane(int mb) { return (size_t)18 * tc_hc(mb) * 16; }
// shared memory: [0, 8) mbarrier, [16, 20) tensor-memory address, halo from 128, then B
__host__ __device__ constexpr size_t tc_halo_bytes(int cin, int cout) { return (size_t)(cin / 8) * tc_plane(tc_mb(cout)); }
__host__ __device__ constexpr size_t tc_smem_bytes(int cin, int cout) {
  return 128 + tc_halo_bytes(cin, cout) + (size_t)9 * cout * cin * 2;
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}

__global__ void __launch_bounds__(kTcPix, 1) k_conv3x3_tc(const bf16* __restrict__ in, const bf16* __restrict__ Wt,
                                                          const float* __restrict__ bias, bf16* out_bf, float* out_f,
                                                          int H, int Wd, int cin, int cout, int relu, int tcols,
                                                          const int* img_on, unsigned polls,
                                                          unsigned long long* flag) {
  if (img_on && !img_on[blockIdx.y]) return;   // image not needed (uniform per CTA, before any allocation)
  extern __shared__ __align__(1024) uint8_t tsm[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(tsm);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(tsm + 16);
  const int MB = tc_mb(cout), HC = tc_hc(MB);
  const uint32_t plane = (uint32_t)tc_plane(MB);
  uint8_t* halo = tsm + 128;
  uint8_t* Bs = halo + (size_t)(cin >> 3) * plane;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int img = blockIdx.y;
  const int tiles_x = (Wd + 8 * MB - 1) / (8 * MB);
  const int ty0 = (blockIdx.x / tiles_x) * 16, tx0 = (blockIdx.x % tiles_x) * (8 * MB);
  const int c8n = cin >> 3;
  const bf16* inb = in + (size_t)img * H * Wd * cin;

  if (warp == 0) {   // tensor memory for the FP32 accumulators: tcols >= MB cout columns x 128 lanes
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)), "r"(tcols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // weights: 16-byte chunk q = (tap, co, c8) -> core matrix (c8, co / 8), row co % 8 of the tap's B
  const int nb16 = 9 * cout * c8n;
  for (int q = tid; q < nb16; q += kTcPix) {
    const int c8 = q % c8n, co = (q / c8n) % cout, tap = q / (c8n * cout);
    cp_async16(su32(Bs + (size_t)tap * cout * cin * 2 + ((size_t)c8 * (cout >> 3) + (co >> 3)) * 128 + (co & 7) * 16),
               Wt + ((size_t)tap * cout + co) * cin + c8 * 8, 16u);
  }
  // halo: chunk q = (position, c8), consecutive threads read consecutive 16-byte chunks of a row
  const int nh16 = 18 * HC * c8n;
  for (int q = tid; q < nh16; q += kTcPix) {
    const int c8 = q % c8n, pos = q / c8n;
    const int yy = ty0 - 1 + pos / HC, xx = tx0 - 1 + pos % HC;
    const bool ok = yy >= 0 && yy < H && xx >= 0 && xx < Wd;
    const bf16* src = inb + (ok ? ((size_t)yy * Wd + xx) * cin + c8 * 8 : 0);
    cp_async16(su32(halo + (size_t)c8 * plane + (size_t)pos * 16), src, ok ? 16u : 0u);   // 0 bytes read: zeros
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic-proxy writes -> tensor-core reads
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  if (tid == 0) {
    const uint32_t idesc = tc_idesc(cout);
    const uint32_t h0 = su32(halo), b0 = su32(Bs), b_lbo = (uint32_t)cout * 16, sbo = (uint32_t)HC * 16;
    for (int mb = 0; mb < MB; ++mb)
      for (int tap = 0; tap < 9; ++tap) {
        const uint32_t a_tap = h0 + (uint32_t)(((tap / 3) * HC + 8 * mb + tap % 3) * 16);
        const uint32_t b_tap = b0 + (uint32_t)(tap * cout * cin * 2);
        for (int kk = 0; kk < (cin >> 4); ++kk)
          tc_mma(tmem + (uint32_t)(mb * cout), tc_sdesc(a_tap + kk * 2 * plane, plane, sbo),
                 tc_sdesc(b_tap + kk * 2 * b_lbo, b_lbo, 128), idesc, (tap | kk) ? 1u : 0u);
      }
    tc_commit(su32(bar));
  }
  tc_wait(su32(bar), 0u, polls, flag);
  tc_fence_after();
  // lane 32 warp + l of M-block mb = row g = (32 warp + l) / 8, column j = l % 8 of the block
  const int r = warp * 32 + (tid & 31);
  const int y = ty0 + (r >> 3);
  const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
  for (int mb = 0; mb < MB; ++mb) {
    const int x = tx0 + 8 * mb + (r & 7);
    const bool st = y < H && x < Wd;
    for (int c0 = 0; c0 < cout; c0 += 8) {
      float v[8];
      tc_ld8(trow + (uint32_t)(mb * cout + c0), v);
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        v[q] += bias ? bias[c0 + q] : 0.f;
        if (relu) v[q] = fmaxf(v[q], 0.f);
      }
      if (st) {
        const size_t o = (((size_t)img * H + y) * Wd + x) * cout + c0;
        if (out_bf) {
          uint4 w;
          w.x = pack_bf2(v[0], v[1]); w.y = pack_bf2(v[2], v[3]); w.z = pack_bf2(v[4], v[5]); w.w = pack_bf2(v[6], v[7]);
          *reinterpret_cast<uint4*>(out_bf + o) = w;
        }
        if (out_f) {
          *reinterpret_cast<float4*>(out_f + o) = make_float4(v[0], v[1], v[2], v[3]);
          *reinterpret_cast<float4*>(out_f + o + 4) = make_float4(v[4], v[5], v[6], v[7]);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols) : "memory");
  }
}

// tensor-memory columns of a CTA and the shared memory it requests: every CTA asks for more than
// its share (cols / 512) of an SM's 228 KB, so the CTAs that fit on an SM together -- of this
// launch or of concurrent ones -- never hold more than its 512 columns, and an allocation never waits
static int tc_cols(int cout) {
  const int n = tc_mb(cout) * cout;
  return n <= 32 ? 32 : n <= 64 ? 64 : 128;
}
static size_t tc_launch_smem(int cin, int cout) {
  const size_t need = tc_smem_bytes(cin, cout);
  const size_t floor = (size_t)(228 * 1024) * (size_t)tc_cols(cout) / 512 + 1024;
  return need > floor ? need : floor;
}
constexpr size_t kTcSmemMax = 200 * 1024;   // above every layer's request (largest: 96 -> 32, 173 KB)

static void conv3x3(const bf16* in, const bf16* Wt, const float* bias, bf16* out_bf, float* out_f, int nimg, int H,
                    int Wd, int cin, int cout, int relu, const int* img_on, unsigned polls,
                    unsigned long long* flag, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_conv3x3_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmemMax);
    attr = true;
  }
  const int mb = tc_mb(cout);
  dim3 g((unsigned)(((H + 15) / 16) * ((Wd + 8 * mb - 1) / (8 * mb))), nimg);
  k_conv3x3_tc<<<g, kTcPix, tc_launch_smem(cin, cout), st>>>(in, Wt, bias, out_bf, out_f, H, Wd, cin, cout, relu,
                                                            tc_cols(cout), img_on, polls, flag);
}

// dW[tap][co][ci] += sum_p gout[p][co] * in[p + off(tap)][ci]; db[co] += sum_p gout[p][co]   (FP32)
__global__ void k_conv_wgrad(const bf16* __restrict__ in, const bf16* __restrict__ gout, float* dW, float* db, int H,
                             int Wd, int cin, int cout, int chunk) {
  const int img = blockIdx.z;
  const int HW = H * Wd;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  const int nw = 9 * cout * cin;
  if (idx >= nw + cout) return;
  const int pbeg = blockIdx.y * chunk, pend = min(HW, pbeg + chunk);
  const bf16* inb = in + (size_t)img * HW * cin;
  const bf16* gb = gout + (size_t)img * HW * cout;
  float acc = 0.f;
  if (idx < nw) {
    const int ci = idx % cin, co = (idx / cin) % cout, tap = idx / (cin * cout);
    const int dy = tap / 3 - 1, dx = tap % 3 - 1;
    for (int p = pbeg; p < pend; ++p) {
      int y = p / Wd + dy, x = p % Wd + dx;
      if (y < 0 || y >= H || x < 0 || x >= Wd) continue;
      acc += __bfloat162float(gb[(size_t)p * cout + co]) * __bfloat162float(inb[(size_t)(y * Wd + x) * cin + ci]);
    }
    atomicAdd(&dW[idx], acc);
  } else {
    const int co = idx - nw;
    for (int p = pbeg; p < pend; ++p) acc += __bfloat162float(gb[(size_t)p * cout + co]);
    atomicAdd(&db[co], acc);
  }
}

// Wflip[tap][ci][co] = W[8 - tap][co][ci]   (backward-data weights)
__global__ void k_flip_weights(const bf16* W, bf16* Wf, int cin, int cout) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 9 * cin * cout) return;
  int co = idx % cout, ci = (idx / cout) % cin, tap = idx / (cout * cin);
  Wf[idx] = W[((size_t)(8 - tap) * cout + co) * cin + ci];
}

// ------------------------------------------------------------------ elementwise helpers (NHWC)
// The forward elementwise kernels run on a grid (blocks, nimg) with image blockIdx.y and a
// grid-stride loop over its elements, so an image the solver does not need costs a few CTAs.
// Channels move 8 at a time (16 bytes; every channel count is a multiple of 16).
__global__ void k_pool2(const bf16* in, bf16* out, int H, int Wd, int C, const int* on) {
  const int img = blockIdx.y;
  if (on && !on[img]) return;
  const int h = H / 2, w = Wd / 2, C8 = C / 8;
  const size_t n = (size_t)h * w * C8;
  const uint4* b = reinterpret_cast<const uint4*>(in + (size_t)img * H * Wd * C);
  uint4* o = reinterpret_cast<uint4*>(out + (size_t)img * h * w * C);
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x) {
    const int c8 = idx % C8;
    const size_t pix = idx / C8;
    const int x = pix % w, y = pix / w;
    const size_t r0 = ((size_t)(2 * y) * Wd + 2 * x) * C8 + c8, r1 = r0 + (size_t)Wd * C8;
    const uint4 q[4] = {b[r0], b[r0 + C8], b[r1], b[r1 + C8]};
    uint4 res;
    uint32_t* rw = reinterpret_cast<uint32_t*>(&res);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      float lo = 0.f, hi = 0.f;
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const __nv_bfloat162 v = reinterpret_cast<const __nv_bfloat162*>(&q[t])[k];
        lo += __low2float(v);
        hi += __high2float(v);
      }
      rw[k] = pack_bf2(0.25f * lo, 0.25f * hi);
    }
    o[idx] = res;
  }
}

// gin (fine, FP32 accumulate) += 0.25 * gout (coarse)
__global__ void k_pool2_bwd(const float* gout, float* gin, int H, int Wd, int C, int nimg) {
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t n = (size_t)nimg * H * Wd * C;
  if (idx >= n) return;
  int c = idx % C;
  size_t pix = idx / C;
  int x = pix % Wd, y = (pix / Wd) % H, img = pix / ((size_t)Wd * H);
  gin[idx] += 0.25f * gout[(((size_t)img * (H / 2) + y / 2) * (Wd / 2) + x / 2) * C + c];
}

// out[:, :, :, 0:C1] = up2(a) (coarse a, nearest), out[..., C1:C1+C2] = b
__global__ void k_up_cat(const bf16* a, const bf16* b, bf16* out, int H, int Wd, int C1, int C2, const int* on) {
  const int img = blockIdx.y;
  if (on && !on[img]) return;
  const int A8 = C1 / 8, B8 = C2 / 8, C8 = A8 + B8;
  const size_t n = (size_t)H * Wd * C8;
  const uint4* ai = reinterpret_cast<const uint4*>(a + (size_t)img * (H / 2) * (Wd / 2) * C1);
  const uint4* bi = reinterpret_cast<const uint4*>(b + (size_t)img * H * Wd * C2);
  uint4* o = reinterpret_cast<uint4*>(out + (size_t)img * H * Wd * (C1 + C2));
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x) {
    const int c8 = idx % C8;
    const size_t pix = idx / C8;
    const int x = pix % Wd, y = pix / Wd;
    o[idx] = c8 < A8 ? ai[((size_t)(y / 2) * (Wd / 2) + x / 2) * A8 + c8] : bi[pix * B8 + (c8 - A8)];
  }
}

// split gradient of the concat: ga (coarse, FP32 +=) gets the up-sampled part summed, gb (fine, FP32 +=)
__global__ void k_up_cat_bwd(const float* g, float* ga, float* gb, int H, int Wd, int C1, int C2, int nimg) {
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int C = C1 + C2;
  size_t n = (size_t)nimg * H * Wd * C;
  if (idx >= n) return;
  int c = idx % C;
  size_t pix = idx / C;
  int x = pix % Wd, y = (pix / Wd) % H, img = pix / ((size_t)Wd * H);
  if (c < C1) atomicAdd(&ga[(((size_t)img * (H / 2) + y / 2) * (Wd / 2) + x / 2) * C1 + c], g[idx]);
  else gb[pix * C2 + (c - C1)] += g[idx];
}

// gbf = bf16(g * (y > 0)) for a ReLU output y (or plain conversion when relu == 0)
__global__ void k_relu_mask(const float* g, const bf16* y, bf16* gbf, size_t n, int relu) {
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n) return;
  float v = g[idx];
  if (relu && __bfloat162float(y[idx]) <= 0.f) v = 0.f;
  gbf[idx] = __float2bfloat16(v);
}

__global__ void k_to_f32(const float* in_dummy, const bf16* in, float* out, size_t n) {
  (void)in_dummy;
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < n) out[idx] = __bfloat162float(in[idx]);
}

// FP32 [nimg][HW][5] -> bf16 [nimg][HW][16] (zero padded)
__global__ void k_pack_input(const float* in, bf16* x, size_t hw, const int* on) {
  const int img = blockIdx.y;
  if (on && !on[img]) return;
  const float* ii = in + (size_t)img * hw * kInChannels;
  bf16* o = x + (size_t)img * hw * 16;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < hw * 16; idx += (size_t)gridDim.x * blockDim.x) {
    const int c = idx % 16;
    const size_t p = idx / 16;
    o[idx] = __float2bfloat16(c < kInChannels ? ii[p * kInChannels + c] : 0.f);
  }
}

// loss = mean over pixels and the 2 used channels of (out - target)^2; grad (FP32, [npix][16]) = d loss / d out
__global__ void k_mse(const float* out, const float* target, float* grad, double* loss, size_t npix, float scale) {
  size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  float l = 0.f;
  if (idx < npix * 16) {
    int c = idx % 16;
    size_t p = idx / 16;
    float gval = 0.f;
    if (c < kOutChannels) {
      float d = out[idx] - target[p * kOutChannels + c];
      l = d * d;
      gval = 2.f * d * scale;
    }
    grad[idx] = gval;
  }
  for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
  if ((threadIdx.x & 31) == 0 && l != 0.f) atomicAdd(loss, (double)l);
}

__global__ void k_adam(float* w, const float* g, float* m, float* v, bf16* wb, size_t n, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float gi = g[i];
  float mi = b1 * m[i] + (1.f - b1) * gi;
  float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  w[i] = wi;
  wb[i] = __float2bfloat16(wi);
}

__global__ void k_f32_to_bf16(const float* a, bf16* b, size_t n) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = __float2bfloat16(a[i]);
}

}  // namespace lt

// ==================================================================== host side
using lt::bf16;
using lt::kNumLayers;

struct lt_unet {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  // parameters: per layer W[9][cout][cin] then b[cout], FP32 masters
  std::vector<size_t> woff, boff;
  size_t nparams = 0;
  float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
  bf16 *wb = nullptr, *wflip = nullptr;
  int step = 0;
  // activation workspace
  int cap_img = 0, cap_H = 0, cap_W = 0;
  std::vector<void*> acts;
  bf16* A[32] = {};     // bf16 activations
  float* G[32] = {};    // FP32 gradients
  bf16* gbf = nullptr;  // bf16 masked gradient scratch
  float* outf = nullptr;
  float* gout = nullptr;
  double* dloss = nullptr;
  // error flag of the bounded tensor-core waits: own counter, or the solver's while it runs the network
  unsigned long long* dflag = nullptr;
  unsigned long long* flag = nullptr;
  // images the network runs on (nullptr: all); set by the solver for the bases that still use the guess
  const int* img_on = nullptr;
  unsigned polls = lt::kTcPolls;   // mbarrier polls of the convolutions before a wait counts as timed out
};

static size_t unet_npix(int nimg, int H, int W, int lvl) { return (size_t)nimg * (H >> lvl) * (W >> lvl); }

// activation slots (level, channels)
enum {
  X0 = 0, A1, S0, P0, A3, S1, P1, A5, S2, P2, A7, BB, C2, A9, D2, C1, A11, D1, C0, A13, D0, NSLOT
};
static const int kSlotLvl[NSLOT] = {0, 0, 0, 1, 1, 1, 2, 2, 2, 3, 3, 3, 2, 2, 2, 1, 1, 1, 0, 0, 0};
static const int kSlotC[NSLOT] = {16, 16, 16, 16, 32, 32, 32, 32, 32, 32, 64, 64, 96, 32, 32, 64, 32, 32, 48, 16, 16};

static int unet_fail(lt_unet* u, int code, const char* msg) {
  if (u) u->err = msg;
  return code;
}

// wait for the network's stream; a bounded tensor-core wait that ran out is reported as -5 (timeout)
static int unet_sync(lt_unet* u, const char* what) {
  if (cudaStreamSynchronize(u->stream) != cudaSuccess) return unet_fail(u, -3, what);
  unsigned long long f = 0;
  if (cudaMemcpy(&f, u->dflag, sizeof(f), cudaMemcpyDeviceToHost) != cudaSuccess) return unet_fail(u, -3, what);
  if (f) {
    cudaMemset(u->dflag, 0, sizeof(f));
    return unet_fail(u, -5, "a bounded wait of the tensor-core convolution ran out");
  }
  return 0;
}

static int unet_ensure(lt_unet* u, int nimg, int H, int W) {
  if (nimg <= u->cap_img && H == u->cap_H && W == u->cap_W) return 0;
  for (void* p : u->acts) cudaFree(p);
  u->acts.clear();
  for (int s = 0; s < NSLOT; ++s) {
    size_t n = unet_npix(nimg, H, W, kSlotLvl[s]) * kSlotC[s];
    if (cudaMalloc(&u->A[s], n * sizeof(bf16)) != cudaSuccess) return -2;
    if (cudaMalloc(&u->G[s], n * sizeof(float)) != cudaSuccess) return -2;
    u->acts.push_back(u->A[s]);
    u->acts.push_back(u->G[s]);
  }
  size_t n0 = unet_npix(nimg, H, W, 0) * 96;
  if (cudaMalloc(&u->gbf, n0 * sizeof(bf16)) != cudaSuccess) return -2;
  u->acts.push_back(u->gbf);
  if (cudaMalloc(&u->outf, unet_npix(nimg, H, W, 0) * 16 * sizeof(float)) != cudaSuccess) return -2;
  u->acts.push_back(u->outf);
  if (cudaMalloc(&u->gout, unet_npix(nimg, H, W, 0) * 16 * sizeof(float)) != cudaSuccess) return -2;
  u->acts.push_back(u->gout);
  u->cap_img = nimg;
  u->cap_H = H;
  u->cap_W = W;
  return 0;
}

// layer l: input slot, output slot, level
static const int kLIn[15] = {X0, A1, P0, A3, P1, A5, P2, A7, C2, A9, C1, A11, C0, A13, D0};
static const int kLOut[15] = {A1, S0, A3, S1, A5, S2, A7, BB, A9, D2, A11, D1, A13, D0, -1};
static const int kLLvl[15] = {0, 0, 1, 1, 2, 2, 3, 3, 2, 2, 1, 1, 0, 0, 0};

static inline unsigned nblk(size_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }
// grid of a per-image elementwise kernel: at most 512 grid-stride blocks per image (blockIdx.y = image)
static dim3 per_img(size_t n_per_image, int nimg) {
  const unsigned b = nblk(n_per_image);
  return dim3(b < 512u ? b : 512u, (unsigned)nimg);
}

static void unet_forward_dev(lt_unet* u, int nimg, int H, int W) {
  cudaStream_t st = u->stream;
  auto conv = [&](int l) {
    const lt::ConvSpec& c = lt::kLayers[l];
    int h = H >> kLLvl[l], w = W >> kLLvl[l];
    bf16* out = kLOut[l] >= 0 ? u->A[kLOut[l]] : nullptr;
    float* outf = kLOut[l] >= 0 ? nullptr : u->outf;
    lt::conv3x3(u->A[kLIn[l]], u->wb + u->woff[l], u->w + u->boff[l], out, outf, nimg, h, w, c.cin, c.cout, c.relu,
                u->img_on, u->polls, u->flag, st);
  };
  auto pool = [&](int src, int dst) {
    int lv = kSlotLvl[src];
    size_t n = unet_npix(nimg, H, W, lv + 1) * kSlotC[src];
    lt::k_pool2<<<per_img(n / nimg / 8, nimg), 256, 0, st>>>(u->A[src], u->A[dst], H >> lv, W >> lv, kSlotC[src],
                                                        u->img_on);
  };
  auto upcat = [&](int a, int b, int dst) {
    int lv = kSlotLvl[dst];
    size_t n = unet_npix(nimg, H, W, lv) * kSlotC[dst];
    lt::k_up_cat<<<per_img(n / nimg / 8, nimg), 256, 0, st>>>(u->A[a], u->A[b], u->A[dst], H >> lv, W >> lv, kSlotC[a],
                                                         kSlotC[b], u->img_on);
  };
  conv(0); conv(1); pool(S0, P0);
  conv(2); conv(3); pool(S1, P1);
  conv(4); conv(5); pool(S2, P2);
  conv(6); conv(7);
  upcat(BB, S2, C2); conv(8); conv(9);
  upcat(D2, S1, C1); conv(10); conv(11);
  upcat(D1, S0, C0); conv(12); conv(13);
  conv(14);
}

// gradient of the loss w.r.t. every parameter (u->g), from u->gout (d loss / d output, FP32 [npix][16])
static void unet_backward_dev(lt_unet* u, int nimg, int H, int W) {
  cudaStream_t st = u->stream;
  cudaMemsetAsync(u->g, 0, u->nparams * sizeof(float), st);
  for (int s : {D1, D2, BB, S0, S1, S2})
    cudaMemsetAsync(u->G[s], 0, unet_npix(nimg, H, W, kSlotLvl[s]) * kSlotC[s] * sizeof(float), st);
  auto layer_bwd = [&](int l, const float* gy) {
    const lt::ConvSpec& c = lt::kLayers[l];
    int lv = kLLvl[l], h = H >> lv, w = W >> lv;
    size_t n = unet_npix(nimg, H, W, lv) * c.cout;
    const bf16* y = kLOut[l] >= 0 ? u->A[kLOut[l]] : nullptr;
    lt::k_relu_mask<<<nblk(n), 256, 0, st>>>(gy, y, u->gbf, n, c.relu && y != nullptr);
    const int nw = 9 * c.cout * c.cin;
    const int chunk = 4096;
    dim3 gw(nblk(nw + c.cout), (h * w + chunk - 1) / chunk, nimg);
    lt::k_conv_wgrad<<<gw, 256, 0, st>>>(u->A[kLIn[l]], u->gbf, u->g + u->woff[l], u->g + u->boff[l], h, w, c.cin,
                                        c.cout, chunk);
    if (l > 0)   // backward data: conv with flipped, transposed weights, FP32 output
      lt::conv3x3(u->gbf, u->wflip + u->woff[l], nullptr, nullptr, u->G[kLIn[l]], nimg, h, w, c.cout, c.cin, 0,
                  nullptr, u->polls, u->flag, st);
  };
  auto upcat_bwd = [&](int a, int b, int dst) {
    int lv = kSlotLvl[dst];
    size_t n = unet_npix(nimg, H, W, lv) * kSlotC[dst];
    lt::k_up_cat_bwd<<<nblk(n), 256, 0, st>>>(u->G[dst], u->G[a], u->G[b], H >> lv, W >> lv, kSlotC[a], kSlotC[b],
                                             nimg);
  };
  auto pool_bwd = [&](int src, int dst) {   // src = fine slot, dst = pooled slot
    int lv = kSlotLvl[src];
    size_t n = unet_npix(nimg, H, W, lv) * kSlotC[src];
    lt::k_pool2_bwd<<<nblk(n), 256, 0, st>>>(u->G[dst], u->G[src], H >> lv, W >> lv, kSlotC[src], nimg);
  };
  layer_bwd(14, u->gout);
  layer_bwd(13, u->G[D0]);
  layer_bwd(12, u->G[A13]);
  upcat_bwd(D1, S0, C0);
  layer_bwd(11, u->G[D1]);
  layer_bwd(10, u->G[A11]);
  upcat_bwd(D2, S1, C1);
  layer_bwd(9, u->G[D2]);
  layer_bwd(8, u->G[A9]);
  upcat_bwd(BB, S2, C2);
  layer_bwd(7, u->G[BB]);
  layer_bwd(6, u->G[A7]);
  pool_bwd(S2, P2);
  layer_bwd(5, u->G[S2]);
  layer_bwd(4, u->G[A5]);
  pool_bwd(S1, P1);
  layer_bwd(3, u->G[S1]);
  layer_bwd(2, u->G[A3]);
  pool_bwd(S0, P0);
  layer_bwd(1, u->G[S0]);
  layer_bwd(0, u->G[A1]);
}

static void unet_refresh_bf16(lt_unet* u) {
  lt::k_f32_to_bf16<<<nblk(u->nparams), 256, 0, u->stream>>>(u->w, u->wb, u->nparams);
  for (int l = 0; l < kNumLayers; ++l) {
    const lt::ConvSpec& c = lt::kLayers[l];
    lt::k_flip_weights<<<nblk(9 * c.cin * c.cout), 256, 0, u->stream>>>(u->wb + u->woff[l], u->wflip + u->woff[l],
                                                                       c.cin, c.cout);
  }
}

static int unet_prepare(lt_unet* u, int nimg, int H, int W, const float* in) {
  if (nimg < 1 || H < 8 || W < 8 || (H % 8) || (W % 8)) return unet_fail(u, -1, "images must be at least 8x8 with sides divisible by 8");
  if (!in) return unet_fail(u, -1, "input is null");
  cudaSetDevice(u->device);
  if (unet_ensure(u, nimg, H, W)) return unet_fail(u, -2, "device allocation failed");
  lt::k_pack_input<<<per_img((size_t)H * W * 16, nimg), 256, 0, u->stream>>>(in, u->A[X0], (size_t)H * W, nullptr);
  return 0;
}

static int unet_loss_grad(lt_unet* u, int nimg, int H, int W, const float* in, const float* target, double* loss) {
  int rc = unet_prepare(u, nimg, H, W, in);
  if (rc) return rc;
  if (!target) return unet_fail(u, -1, "target is null");
  size_t npix = unet_npix(nimg, H, W, 0);
  unet_forward_dev(u, nimg, H, W);
  cudaMemsetAsync(u->dloss, 0, sizeof(double), u->stream);
  float scale = 1.f / (float)(npix * lt::kOutChannels);
  lt::k_mse<<<nblk(npix * 16), 256, 0, u->stream>>>(u->outf, target, u->gout, u->dloss, npix, scale);
  unet_backward_dev(u, nimg, H, W);
  double l = 0.0;
  cudaMemcpyAsync(&l, u->dloss, sizeof(double), cudaMemcpyDeviceToHost, u->stream);
  if ((rc = unet_sync(u, "CUDA error in the network step"))) return rc;
  if (loss) *loss = l * scale;
  return 0;
}

__global__ void k_take2(const float* outf, float* out, size_t npix) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < npix * 2) out[i] = outf[(i / 2) * 16 + (i % 2)];
}

extern "C" {

int lt_unet_create(lt_unet** out, int device, unsigned long long seed) {
  if (!out) return -1;
  *out = nullptr;
  if (cudaSetDevice(device) != cudaSuccess) return -3;
  lt_unet* u = new lt_unet();
  u->device = device;
  size_t off = 0;
  for (int l = 0; l < kNumLayers; ++l) {
    const lt::ConvSpec& c = lt::kLayers[l];
    u->woff.push_back(off);
    off += (size_t)9 * c.cin * c.cout;
    u->boff.push_back(off);
    off += c.cout;
  }
  u->nparams = off;
  std::vector<float> w(off, 0.f);
  std::mt19937_64 rng(seed);
  std::normal_distribution<float> nd(0.f, 1.f);
  for (int l = 0; l < kNumLayers; ++l) {
    const lt::ConvSpec& c = lt::kLayers[l];
    int cin_real = l == 0 ? lt::kInChannels : c.cin;
    float sd = std::sqrt(2.f / (9.f * cin_real)) * (l == kNumLayers - 1 ? 0.1f : 1.f);
    for (int tap = 0; tap < 9; ++tap)
      for (int co = 0; co < c.cout; ++co)
        for (int ci = 0; ci < c.cin; ++ci)
          w[u->woff[l] + ((size_t)tap * c.cout + co) * c.cin + ci] = (ci < cin_real) ? sd * nd(rng) : 0.f;
  }
  bool ok = cudaMalloc(&u->w, off * 4) == cudaSuccess && cudaMalloc(&u->g, off * 4) == cudaSuccess &&
            cudaMalloc(&u->m, off * 4) == cudaSuccess && cudaMalloc(&u->v, off * 4) == cudaSuccess &&
            cudaMalloc(&u->wb, off * 2) == cudaSuccess && cudaMalloc(&u->wflip, off * 2) == cudaSuccess &&
            cudaMalloc(&u->dloss, sizeof(double)) == cudaSuccess &&
            cudaMalloc(&u->dflag, sizeof(unsigned long long)) == cudaSuccess;
  if (!ok) { delete u; return -2; }
  cudaMemcpy(u->w, w.data(), off * 4, cudaMemcpyHostToDevice);
  cudaMemset(u->m, 0, off * 4);
  cudaMemset(u->v, 0, off * 4);
  cudaMemset(u->dflag, 0, sizeof(unsigned long long));
  u->flag = u->dflag;
  unet_refresh_bf16(u);
  if (cudaStreamSynchronize(u->stream) != cudaSuccess) { delete u; return -3; }
  *out = u;
  return 0;
}

int lt_unet_num_params(lt_unet* u) { return u ? (int)u->nparams : -1; }

int lt_unet_get_params(lt_unet* u, float* host, int n) {
  if (!u || !host || n != (int)u->nparams) return -1;
  cudaSetDevice(u->device);
  return cudaMemcpy(host, u->w, n * 4, cudaMemcpyDeviceToHost) == cudaSuccess ? 0 : -3;
}

int lt_unet_set_params(lt_unet* u, const float* host, int n) {
  if (!u || !host || n != (int)u->nparams) return -1;
  cudaSetDevice(u->device);
  if (cudaMemcpy(u->w, host, n * 4, cudaMemcpyHostToDevice) != cudaSuccess) return -3;
  unet_refresh_bf16(u);
  return cudaStreamSynchronize(u->stream) == cudaSuccess ? 0 : -3;
}

int lt_unet_forward(lt_unet* u, int nimg, int H, int W, const float* in, float* out) {
  if (!u || !out) return -1;
  int rc = unet_prepare(u, nimg, H, W, in);
  if (rc) return rc;
  unet_forward_dev(u, nimg, H, W);
  size_t npix = unet_npix(nimg, H, W, 0);
  k_take2<<<nblk(npix * 2), 256, 0, u->stream>>>(u->outf, out, npix);
  return unet_sync(u, "CUDA error in forward");
}

int lt_unet_grad(lt_unet* u, int nimg, int H, int W, const float* in, const float* target, float* grad_host,
                 double* loss) {
  if (!u) return -1;
  int rc = unet_loss_grad(u, nimg, H, W, in, target, loss);
  if (rc) return rc;
  if (grad_host) cudaMemcpy(grad_host, u->g, u->nparams * 4, cudaMemcpyDeviceToHost);
  return 0;
}

int lt_unet_train_step(lt_unet* u, int nimg, int H, int W, const float* in, const float* target, float lr,
                       double* loss) {
  if (!u) return -1;
  int rc = unet_loss_grad(u, nimg, H, W, in, target, loss);
  if (rc) return rc;
  ++u->step;
  const float b1 = 0.9f, b2 = 0.999f;
  float c1 = 1.f - std::pow(b1, (float)u->step), c2 = 1.f - std::pow(b2, (float)u->step);
  lt::k_adam<<<nblk(u->nparams), 256, 0, u->stream>>>(u->w, u->g, u->m, u->v, u->wb, u->nparams, lr, b1, b2, 1e-8f,
                                                     c1, c2);
  for (int l = 0; l < kNumLayers; ++l) {
    const lt::ConvSpec& c = lt::kLayers[l];
    lt::k_flip_weights<<<nblk(9 * c.cin * c.cout), 256, 0, u->stream>>>(u->wb + u->woff[l], u->wflip + u->woff[l],
                                                                       c.cin, c.cout);
  }
  return cudaStreamSynchronize(u->stream) == cudaSuccess ? 0 : unet_fail(u, -3, "CUDA error in the Adam step");
}

int lt_unet_set_wait_polls(lt_unet* u, unsigned polls) {
  if (!u) return -1;
  u->polls = polls;
  return 0;
}

const char* lt_unet_last_error(lt_unet* u) { return u ? u->err.c_str() : "null network"; }

void lt_unet_destroy(lt_unet* u) {
  if (!u) return;
  cudaSetDevice(u->device);
  for (void* p : u->acts) cudaFree(p);
  for (void* p : {(void*)u->w, (void*)u->g, (void*)u->m, (void*)u->v, (void*)u->wb, (void*)u->wflip, (void*)u->dloss,
                  (void*)u->dflag})
    if (p) cudaFree(p);
  cudaGetLastError();
  delete u;
}

}  // extern "C"

// ==================================================================== use inside the preconditioner solves
namespace lt {

__device__ __forceinline__ bool lg_skip(const Batch& bt, int b, int round) {
  if (!bt.active[b]) return true;
  return bt.rnorm2[b * (bt.rounds + 1) + round] <= bt.itol2[b];
}

// Gate of the learned guess per basis (int on[nb], int run[nb] after the four accumulators of each
// basis): on[b] starts at 1 for every solve and drops to 0 for good once the basis's guess is
// rejected; the network runs this round on the bases with run[b] = on[b] and an open solve.
__device__ __forceinline__ int* gate_on(float* gn, int nb) { return reinterpret_cast<int*>(gn + 4 * nb); }

// network input from the round's float32 residual f0 = L0.f; run[b] for the network's kernels
__global__ void k_net_pack(Batch bt, Level L0, int round, const float* lk, const float* mD, float* x, float* gn) {
  int b = blockIdx.y;
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  const bool run = gate_on(gn, bt.nb)[b] && !lg_skip(bt, b, round);
  if (c == 0) gate_on(gn, bt.nb)[bt.nb + b] = run ? 1 : 0;
  if (c >= L0.N || !run) return;
  double rn = bt.rnorm2[b * (bt.rounds + 1) + round];
  float s = (float)sqrt(rn / (double)L0.N);
  float inv = s > 0.f ? 1.f / s : 0.f;
  float2 f = L0.f[(size_t)b * L0.N + c];
  double2 t = bt.tau_cur[b];
  float* o = x + ((size_t)b * L0.N + c) * kInChannels;
  o[0] = f.x * inv;
  o[1] = f.y * inv;
  o[2] = lk[c];
  o[3] = (float)t.x * mD[c];
  o[4] = (float)t.y * mD[c];
}

// w = (out0 + i out1) / D  (direction of the guess; scaled below)
__global__ void k_net_unpack(Batch bt, Level L0, int round, const float* outf, float* gn) {
  int b = blockIdx.y;
  if (lg_skip(bt, b, round)) return;
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= L0.N) return;
  if (c < 4) gn[b * 4 + c] = 0.f;
  if (!gate_on(gn, bt.nb)[b]) {   // guess switched off: the V-cycles start from zero
    L0.u[(size_t)b * L0.N + c] = make_float2(0.f, 0.f);
    return;
  }
  const float* o = outf + ((size_t)b * L0.N + c) * 16;
  float Dc = L0.D[c];
  L0.u[(size_t)b * L0.N + c] = make_float2(o[0] / Dc, o[1] / Dc);
}

// per basis: a = sum conj(A w) f (complex), q = sum |A w|^2   (float32 level-0 operator)
__global__ void k_net_dots(Batch bt, Level L0, int round, float* gn) {
  int b = blockIdx.y;
  if (lg_skip(bt, b, round)) return;
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  float ar = 0.f, ai = 0.f, q = 0.f;
  if (c < L0.N) {
    const float2* u = L0.u + (size_t)b * L0.N;
    int i = c % L0.nx, j = c / L0.nx;
    double2 t = bt.tau_cur[b];
    float m = L0.m[c];
    float2 d = make_float2(L0.D[c] + (float)t.x * m, (float)t.y * m);
    float2 uc = u[c];
    float ax = d.x * uc.x - d.y * uc.y, ay = d.x * uc.y + d.y * uc.x;
    if (i + 1 < L0.nx) { ax -= L0.Te[c] * u[c + 1].x; ay -= L0.Te[c] * u[c + 1].y; }
    if (i > 0) { ax -= L0.Te[c - 1] * u[c - 1].x; ay -= L0.Te[c - 1] * u[c - 1].y; }
    if (j + 1 < L0.ny) { ax -= L0.Tn[c] * u[c + L0.nx].x; ay -= L0.Tn[c] * u[c + L0.nx].y; }
    if (j > 0) { ax -= L0.Tn[c - L0.nx] * u[c - L0.nx].x; ay -= L0.Tn[c - L0.nx] * u[c - L0.nx].y; }
    float2 f = L0.f[(size_t)b * L0.N + c];
    ar = ax * f.x + ay * f.y;
    ai = ax * f.y - ay * f.x;
    q = ax * ax + ay * ay;
  }
  for (int o = 16; o > 0; o >>= 1) {
    ar += __shfl_xor_sync(0xffffffffu, ar, o);
    ai += __shfl_xor_sync(0xffffffffu, ai, o);
    q += __shfl_xor_sync(0xffffffffu, q, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&gn[b * 4 + 0], ar);
    atomicAdd(&gn[b * 4 + 1], ai);
    atomicAdd(&gn[b * 4 + 2], q);
  }
}

// u0 = alpha w with the minimal-residual alpha = a / q; the residual is then
// ||f||^2 - |a|^2 / q <= ||f||^2, and a guess that removes less than 5% of the
// residual norm is dropped in favour of the zero guess (multigrid fallback); the
// basis then solves without the network for the rest of the solve
__global__ void k_net_scale(Batch bt, Level L0, int round, float* gn) {
  int b = blockIdx.y;
  if (lg_skip(bt, b, round)) return;
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= L0.N) return;
  float ar = gn[b * 4 + 0], ai = gn[b * 4 + 1], q = gn[b * 4 + 2];
  double f2 = bt.rnorm2[b * (bt.rounds + 1) + round];
  double gain = q > 0.f ? ((double)ar * ar + (double)ai * ai) / q : 0.0;   // ||f||^2 - ||f - alpha A w||^2
  bool keep = q > 0.f && gain >= (1.0 - 0.95 * 0.95) * f2;
  float2 w = L0.u[(size_t)b * L0.N + c];
  float2 a = keep ? make_float2(ar / q, ai / q) : make_float2(0.f, 0.f);
  L0.u[(size_t)b * L0.N + c] = make_float2(a.x * w.x - a.y * w.y, a.x * w.y + a.y * w.x);
  if (c == 0) {   // the only thread of this launch that touches the gate
    int* on = gate_on(gn, bt.nb);
    if (keep && on[b]) atomicAdd(&bt.work[KC_OTHER], 1ull);   // guesses kept (statistics)
    if (!keep) on[b] = 0;
  }
}

// ---- training pairs (residual r, multigrid solution e of (K + tau M) e = r) -> (input, target)
// acc[img] += sum_c |v_c|^2 (scale_c = 1) or |scale_c v_c|^2
__global__ void k_img_norm2(const float2* v, const float* scale, int N, double* acc) {
  const int img = blockIdx.y;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  float q = 0.f;
  if (c < N) {
    float2 a = v[(size_t)img * N + c];
    float f = scale ? scale[c] : 1.f;
    q = f * f * (a.x * a.x + a.y * a.y);
  }
  for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(&acc[img], (double)q);
}

// network input (the same channels as k_net_pack) and target: D e at unit RMS
__global__ void k_pair_pack(const float2* r, const float2* e, const double2* tau, const float* lk, const float* mD,
                            const float* D, const double* rn2, const double* en2, int N, float* x, float* y) {
  const int img = blockIdx.y;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= N) return;
  const size_t i = (size_t)img * N + c;
  const float rs = (float)sqrt(rn2[img] / N), es = (float)sqrt(en2[img] / N);
  const float ir = rs > 0.f ? 1.f / rs : 0.f, ie = es > 0.f ? 1.f / es : 0.f;
  const float2 f = r[i], u = e[i];
  const double2 t = tau[img];
  float* o = x + i * kInChannels;
  o[0] = f.x * ir;
  o[1] = f.y * ir;
  o[2] = lk[c];
  o[3] = (float)t.x * mD[c];
  o[4] = (float)t.y * mD[c];
  y[2 * i] = D[c] * u.x * ie;
  y[2 * i + 1] = D[c] * u.y * ie;
}

}  // namespace lt

// inputs x [nimg][N][5] and targets y [nimg][N][2] of training pairs from residuals r and their
// multigrid solutions e (all DEVICE); tau: DEVICE [nimg]; lk, mD, D: DEVICE [N]; acc: DEVICE [2 nimg]
void learned_pair_features(int nimg, int N, const float2* r, const float2* e, const double2* tau, const float* lk,
                           const float* mD, const float* D, double* acc, float* x, float* y, cudaStream_t q) {
  cudaMemsetAsync(acc, 0, 2 * (size_t)nimg * sizeof(double), q);
  dim3 g((N + 255) / 256, nimg);
  lt::k_img_norm2<<<g, 256, 0, q>>>(r, nullptr, N, acc);
  lt::k_img_norm2<<<g, 256, 0, q>>>(e, D, N, acc + nimg);
  lt::k_pair_pack<<<g, 256, 0, q>>>(r, e, tau, lk, mD, D, acc, acc + nimg, N, x, y);
}

// workspace for nb images of ny x nx (call before graph capture)
int learned_prepare(lt_unet* u, int nb, int ny, int nx) {
  if (!u) return -1;
  if (ny % 8 || nx % 8 || ny < 8 || nx < 8) return -1;
  return unet_ensure(u, nb, ny, nx) ? -2 : 0;
}

// learned initial guess for round `round` of every active basis (kernels only; capturable)
void learned_guess(lt_unet* u, const lt::Batch& bt, const lt::Level& L0, int round, const float* lk, const float* mD,
                   float* xin, float* gnorm2, cudaStream_t q) {
  const int nb = bt.nb;
  dim3 g((L0.N + 255) / 256, nb);
  lt::k_net_pack<<<g, 256, 0, q>>>(bt, L0, round, lk, mD, xin, gnorm2);
  cudaStream_t saved = u->stream;
  unsigned long long* saved_flag = u->flag;
  const int* run = reinterpret_cast<const int*>(gnorm2 + 4 * nb) + nb;
  u->stream = q;
  u->flag = bt.work + lt::kTimeoutSlot;   // a timed-out wait is reported with the solve's status
  u->img_on = run;
  lt::k_pack_input<<<per_img((size_t)L0.N * 16, nb), 256, 0, q>>>(xin, u->A[X0], (size_t)L0.N, run);
  unet_forward_dev(u, nb, L0.ny, L0.nx);
  u->stream = saved;
  u->flag = saved_flag;
  u->img_on = nullptr;
  lt::k_net_unpack<<<g, 256, 0, q>>>(bt, L0, round, u->outf, gnorm2);
  lt::k_net_dots<<<g, 256, 0, q>>>(bt, L0, round, gnorm2);
  lt::k_net_scale<<<g, 256, 0, q>>>(bt, L0, round, gnorm2);
}
