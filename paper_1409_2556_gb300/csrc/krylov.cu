// krylov.cu -- flexible Krylov method for shifted systems (Sec. 3,
// Algorithm 1), batched over bases (one basis per right-hand side and
// preconditioner-shift group), plus the quadrature-fused measurements
// (Eq. half) and the true-residual check.
//
// Per outer iteration j of every active basis:
//   1. preconditioner solve (K + tau_j M) u_j = v_j to a relative residual
//      inner_tol: rounds of  r = v_j - (K + tau_j M) u_j  in df32 (exact),
//      float32 V-cycles on A d = r, u_j += d;
//   2. s_j = M u_j, classical Gram-Schmidt with reorthogonalisation against
//      V_j: coefficient dots in float32 (they only need to be close), the
//      vector updates s -= V c in df32 so that M u_j = V_{j+1} hbar_j holds
//      to ~1e-13 whatever the rounding of c;  h_{j+1,j} = ||s||,
//      v_{j+1} = s / h_{j+1,j};
//   3. for every unconverged shift z_k of the basis: the new column of
//      Hbar(z_k; T_j) = [I; 0] + Hbar_j (z_k I - T_j) is reduced by the
//      shift's stored Givens rotations (GMRES-Sh least squares), giving the
//      residual |g_{j+1}| (relative, b = e_cell has unit norm).
// V and U are kept in df32 (hi, lo float2 planes); the hi plane alone feeds
// the float32 dot products.
#include <cstdio>
#include "df32.cuh"
#include "exact.cuh"
#include "lt_internal.h"
#include "lt_kernels.h"

namespace lt {

template <int NV>
__device__ __forceinline__ void block_reduce_add(float* v, float* smem /* [32*NV] */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < NV; ++q) smem[warp * NV + q] = v[q];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] = lane < nw ? smem[lane * NV + q] : 0.f;
#pragma unroll
    for (int q = 0; q < NV; ++q)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
  }
  __syncthreads();
}

// ------------------------------------------------------------ batch init
__global__ void k_init_vectors(Batch bt) {
  int b = blockIdx.y;
  int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= bt.N) return;
  size_t idx = (size_t)b * (bt.maxit + 1) * bt.N + c;
  const int64_t rc = bt.rhs_cell[b];
  float hi = (c == rc) ? 1.f : 0.f, lo = 0.f;
  if (rc < 0) { hi = bt.rhs_hi[c]; lo = bt.rhs_lo[c]; }    // dense right-hand side (initial state)
  if (bt.V_lo) {
    bt.V_hi[idx] = make_float2(hi, 0.f);
    bt.V_lo[idx] = make_float2(lo, 0.f);
  } else {
    bt.V_hi[idx] = make_float2(hi + lo, 0.f);
  }
}

__global__ void k_init_shifts(Batch bt) {
  int sh = blockIdx.x * blockDim.x + threadIdx.x;
  if (sh < bt.nsh) {
    bt.g[(size_t)sh * (bt.maxit + 1)] = make_double2(1.0, 0.0);
    bt.conv_it[sh] = 0;
    bt.pres[sh] = 1.0;
  }
  if (sh < 8) bt.jdev[sh] = 0;   // (slots 1-7: the counters of the other parts when the bases run decoupled)
  if (sh < bt.nb) {
    bt.active[sh] = 1;
    bt.nit[sh] = 0;
    bt.inner_max[sh] = 0.0;
    bt.rmax[sh] = 1.0;
  }
}

void launch_init_batch(const Batch& bt, cudaStream_t st) {
  dim3 g((unsigned)((bt.N + 255) / 256), bt.nb);
  k_init_vectors<<<g, 256, 0, st>>>(bt);
  int n = bt.nsh > bt.nb ? bt.nsh : bt.nb;
  k_init_shifts<<<(n + 255) / 256, 256, 0, st>>>(bt);
}

// ------------------------------------------------------------ per-iteration prep
__global__ void k_prep_iter(Batch bt, int) {
  const int j = *bt.jdev;   // outer iteration (device counter, so one captured graph serves every j)
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= bt.nb) return;
  if (!bt.active[b]) return;
  int slot = bt.tau_pattern[j % 5];
  int g = bt.group[b];
  bt.tau_cur[b] = bt.tau_grp[2 * g + slot];
  bt.tau_slot[b] = 2 * g + slot;
  // inexact-Krylov relaxation: the preconditioner-solve error e_j enters the
  // true residual as e_j y_j, and |y_j| falls with the outer residual, so the
  // inner tolerance may grow as 1 / (largest unconverged projected residual)
  double it2 = bt.inner_tol2;
  if (bt.inner_relax_max > 0.0 && j > 0) {
    double r = bt.rmax[b] > 0.0 ? bt.rmax[b] : 1.0;
    double f = 1.0 / r;
    double lim = bt.inner_relax_max * bt.inner_relax_max / bt.inner_tol2;
    f = f * f;
    if (f > lim) f = lim;
    if (f < 1.0) f = 1.0;
    it2 *= f;
  }
  bt.itol2[b] = it2;
  for (int r = 0; r <= bt.rounds; ++r) bt.rnorm2[b * (bt.rounds + 1) + r] = 0.0;
  for (int i = 0; i < 2 * (bt.maxit + 1); ++i) bt.dot[(size_t)b * 2 * (bt.maxit + 1) + i] = make_double2(0.0, 0.0);
  bt.snorm2[b] = 0.0;
}

void launch_prep_iter(const Batch& bt, int j, cudaStream_t st) {
  k_prep_iter<<<(bt.nb + 127) / 128, 128, 0, st>>>(bt, j);
}

// ------------------------------------------------------------ preconditioner-solve rounds
__global__ void k_exact_residual(Batch bt, FineExact fe, Level L0, int, int round, int record_only) {
  const int j = *bt.jdev;   // outer iteration (device counter, so one captured graph serves every j)
  __shared__ float red[32];
  int b = blockIdx.y;
  if (!bt.active[b]) return;
  const int R1 = bt.rounds + 1;
  if (!record_only && round > 0 && bt.rnorm2[b * R1 + round - 1] <= bt.itol2[b]) return;
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  float acc[1] = {0.f};
  if (c < fe.N) {
    size_t vi = ((size_t)b * (bt.maxit + 1) + j) * bt.N + c;
    cdf r = load_cdf(bt.V_hi, bt.V_lo, vi);
    if (round > 0) {
      double2 t = bt.tau_cur[b];
      df taur = df_from_double(t.x), taui = df_from_double(t.y);
      size_t ub = ((size_t)b * bt.maxit + j) * bt.N;
      cdf au = apply_exact(fe, bt.U_hi + ub, lo_at(bt.U_lo, ub), c, taur, taui);
      r = cdf_sub(r, au);
    }
    if (!record_only) {
      L0.f[(size_t)b * L0.N + c] = make_float2(r.re.hi, r.im.hi);
      L0.u[(size_t)b * L0.N + c] = make_float2(0.f, 0.f);
    }
    acc[0] = r.re.hi * r.re.hi + r.im.hi * r.im.hi;
  }
  block_reduce_add<1>(acc, red);
  if (threadIdx.x == 0) {
    atomicAdd(&bt.rnorm2[b * R1 + round], (double)acc[0]);
    atomicAdd(&bt.work[KC_EXACT_RES], (unsigned long long)min((int)blockDim.x, fe.N - (int)(blockIdx.x * blockDim.x)));
  }
}

void launch_exact_residual(const Batch& bt, const FineExact& fe, const Level& L0, int j, int round, int record_only,
                           cudaStream_t st, Prof* pf) {
  dim3 g((fe.N + 255) / 256, bt.nb);
  prof_begin(pf, KC_EXACT_RES, st);
  k_exact_residual<<<g, 256, 0, st>>>(bt, fe, L0, j, round, record_only);
  prof_end(pf, KC_EXACT_RES, st);
}

__global__ void k_update_u(Batch bt, Level L0, int, int round) {
  const int j = *bt.jdev;   // outer iteration (device counter, so one captured graph serves every j)
  int b = blockIdx.y;
  if (!bt.active[b]) return;
  if (bt.rnorm2[b * (bt.rounds + 1) + round] <= bt.itol2[b]) return;
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= L0.N) return;
  float2 d = L0.u[(size_t)b * L0.N + c];
  size_t ui = ((size_t)b * bt.maxit + j) * bt.N + c;
  if (round == 0) {
    bt.U_hi[ui] = d;
    if (bt.U_lo) bt.U_lo[ui] = make_float2(0.f, 0.f);
  } else {
    cdf u = load_cdf(bt.U_hi, bt.U_lo, ui);
    u.re = df_add_f(u.re, d.x);
    u.im = df_add_f(u.im, d.y);
    store_cdf(bt.U_hi, bt.U_lo, ui, u);
  }
}

void launch_update_u(const Batch& bt, const Level& L0, int j, int round, cudaStream_t st) {
  dim3 g((L0.N + 255) / 256, bt.nb);
  k_update_u<<<g, 256, 0, st>>>(bt, L0, j, round);
}

__global__ void k_inner_record(Batch bt) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= bt.nb || !bt.active[b]) return;
  double r = sqrt(bt.rnorm2[b * (bt.rounds + 1) + bt.rounds]);
  if (r > bt.inner_max[b]) bt.inner_max[b] = r;
}

void launch_inner_record(const Batch& bt, cudaStream_t st) {
  k_inner_record<<<(bt.nb + 127) / 128, 128, 0, st>>>(bt);
}

// ------------------------------------------------------------ Arnoldi (Algorithm 1, s_j = M u_j and CGS2)
constexpr int kArnT = 256;   // threads per block
constexpr int kCPT = 4;      // cells per thread
constexpr int kIG = 4;       // basis vectors reduced together

constexpr int kWarps = kArnT / 32;
constexpr int kMaxCol = 256;   // columns of V (maxit + 1 <= 251)

// Sum 8 values over the 32 lanes of a warp in 9 shuffles: each step trades half of the lane's
// remaining values with the partner lane (offsets 16, 8, 4), then offsets 2 and 1 finish the sum.
// Afterwards lane 4k (k = 0..7) holds the warp's sum of value k.
template <class T>
__device__ __forceinline__ T warp_sum8(T (&v)[8], int lane) {
  const bool up16 = lane & 16, up8 = lane & 8, up4 = lane & 4;
  T a[4], b2[2], c;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    T send = up16 ? v[k] : v[k + 4];
    T keep = up16 ? v[k + 4] : v[k];
    a[k] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    T send = up8 ? a[k] : a[k + 2];
    T keep = up8 ? a[k + 2] : a[k];
    b2[k] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  {
    T send = up4 ? b2[0] : b2[1];
    T keep = up4 ? b2[1] : b2[0];
    c = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
  c += __shfl_xor_sync(0xffffffffu, c, 2);
  c += __shfl_xor_sync(0xffffffffu, c, 1);
  return c;   // value index: 4 * up16 + 2 * up8 + up4 = lane >> 2
}

// Column dots conj(V_i)^T s (i = 0..j) from the hi plane over the thread's cells: four columns at a
// time, reduced per warp into part[warp][i] without block barriers, then once across the warps
// with one double atomicAdd per column into dst.
__device__ __forceinline__ void column_dots(const float2* V, size_t N, int Nc, int c0, const float2 (&s)[kCPT],
                                            int j, float2 (*part)[kMaxCol], double2* dst) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i0 = 0; i0 <= j; i0 += kIG) {
    float acc[2 * kIG];
#pragma unroll
    for (int q = 0; q < 2 * kIG; ++q) acc[q] = 0.f;
#pragma unroll
    for (int ii = 0; ii < kIG; ++ii) {
      const int i = i0 + ii;
      if (i > j) break;
      const float2* v = V + (size_t)i * N;
#pragma unroll
      for (int q = 0; q < kCPT; ++q) {
        const int c = c0 + q * kArnT;
        if (c < Nc) {
          const float2 a = v[c];
          acc[2 * ii] += a.x * s[q].x + a.y * s[q].y;      // conj(a) * s
          acc[2 * ii + 1] += a.x * s[q].y - a.y * s[q].x;
        }
      }
    }
    const float r = warp_sum8(acc, lane);
    const int k = lane >> 2;
    if ((lane & 3) == 0 && i0 + (k >> 1) <= j) {
      float* slot = reinterpret_cast<float*>(&part[warp][i0 + (k >> 1)]);
      slot[k & 1] = r;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i <= j; i += blockDim.x) {
    float re = 0.f, im = 0.f;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
      re += part[w][i].x;
      im += part[w][i].y;
    }
    atomicAdd(&dst[i].x, (double)re);
    atomicAdd(&dst[i].y, (double)im);
  }
}

// pass 1: dot[0][i] = V_hi[i]^H s_hi, s = M u_j (float32 estimate)
__global__ void __launch_bounds__(kArnT, 6) k_dots1(Batch bt, FineExact fe, int) {
  const int j = *bt.jdev;   // outer iteration (device counter, so one captured graph serves every j)
  __shared__ float2 part[kWarps][kMaxCol];
  int b = blockIdx.y;
  if (!bt.active[b]) return;
  const int N = fe.N;
  int c0 = blockIdx.x * kArnT * kCPT + threadIdx.x;
  float2 s[kCPT];
  size_t ub = ((size_t)b * bt.maxit + j) * bt.N;
#pragma unroll
  for (int q = 0; q < kCPT; ++q) {
    int c = c0 + q * kArnT;
    if (c < N) {
      float2 u = bt.U_hi[ub + c];
      float m = fe.m_hi[c];
      s[q] = make_float2(m * u.x, m * u.y);
    } else {
      s[q] = make_float2(0.f, 0.f);
    }
  }
  column_dots(bt.V_hi + (size_t)b * (bt.maxit + 1) * bt.N, bt.N, N, c0, s, j, part,
              bt.dot + (size_t)b * 2 * (bt.maxit + 1));
  if (threadIdx.x == 0) {
    int n = min(kArnT * kCPT, N - (int)(blockIdx.x * kArnT * kCPT));
    atomicAdd(&bt.work[KC_DOTS], (unsigned long long)n * (unsigned long long)(j + 1));
  }
}

// mode 0 (pass 2): s' = M u_j - V c1 (df32, exact); dot[1][i] = V_hi[i]^H s'_hi; S <- s'
// mode 1 (pass 3): s'' = S - V c2; snorm2 += ||s''||^2; S <- s''.  The second-pass coefficients are
//   of the order of the first pass's float32 dot error (about 2^-24 ||M u_j||), so their products
//   are formed in float32 from the hi plane and folded into the df32 s every 8 columns: the
//   Arnoldi relation keeps an error near 2^-48 * 8 * sqrt(columns / 8) of ||M u_j|| (about 1e-13),
//   and the pass reads only the hi plane of V (k_update_second)
// mode 2 (the one-pass form): s' = M u_j - V c1 with c1 from the df32 dots; snorm2 += ||s'||^2; S <- s'
__global__ void __launch_bounds__(kArnT, 6) k_update(Batch bt, FineExact fe, int, int mode) {
  const bool from_u = mode != 1, do_dots = mode == 0;
  const int second = mode == 1;
  const int j = *bt.jdev;   // outer iteration (device counter, so one captured graph serves every j)
  __shared__ float red[32 * 2 * kIG];
  __shared__ float2 part[kWarps][kMaxCol];
  __shared__ float2 cf[kMaxCol];
  __shared__ float2 cl[kMaxCol];     // mode 2: the low words of the df32-accurate coefficients
  int b = blockIdx.y;
  if (!bt.active[b]) return;
  const int N = fe.N;
  const double2* dsrc = bt.dot + (size_t)b * 2 * (bt.maxit + 1) + (second ? (bt.maxit + 1) : 0);
  for (int i = threadIdx.x; i <= j; i += blockDim.x) {
    const float hx = (float)dsrc[i].x, hy = (float)dsrc[i].y;
    cf[i] = make_float2(hx, hy);
    cl[i] = make_float2((float)(dsrc[i].x - (double)hx), (float)(dsrc[i].y - (double)hy));
  }
  __syncthreads();
  int c0 = blockIdx.x * kArnT * kCPT + threadIdx.x;
  cdf s[kCPT];
  size_t ub = ((size_t)b * bt.maxit + j) * bt.N;
  size_t sb = (size_t)b * bt.N;
#pragma unroll
  for (int q = 0; q < kCPT; ++q) {
    int c = c0 + q * kArnT;
    if (c < N) {
      if (from_u) {
        df m = ldf(fe.m_hi, fe.m_lo, c);
        s[q] = cdf_mul_r(load_cdf(bt.U_hi, bt.U_lo, ub + c), m);
      } else {
        s[q] = load_cdf(bt.S_hi, bt.S_lo, sb + c);
      }
    } else {
      s[q] = {{0.f, 0.f}, {0.f, 0.f}};
    }
  }
  size_t vb = (size_t)b * (bt.maxit + 1) * bt.N;
#pragma unroll 2
  for (int i = 0; i <= j; ++i) {
    float2 ci = cf[i];
    const float2 cli = cl[i];
    const float2* vh = bt.V_hi + vb + (size_t)i * bt.N;
    const float2* vl = lo_at(bt.V_lo, vb + (size_t)i * bt.N);
#pragma unroll
    for (int q = 0; q < kCPT; ++q) {
      int c = c0 + q * kArnT;
      if (c < N) {
        float2 h = vh[c], l = vl ? vl[c] : make_float2(0.f, 0.f);
        cdf v = {{h.x, l.x}, {h.y, l.y}};
        s[q] = cdf_sub_mul_cf(s[q], v, ci.x, ci.y);
        if (mode == 2) {   // - V_hi c_lo: the rest of the coefficient (V_lo c_lo is below 1e-14 |c|)
          s[q].re = df_add_f(s[q].re, -(h.x * cli.x - h.y * cli.y));
          s[q].im = df_add_f(s[q].im, -(h.x * cli.y + h.y * cli.x));
        }
      }
    }
  }
#pragma unroll
  for (int q = 0; q < kCPT; ++q) {
    int c = c0 + q * kArnT;
    if (c < N) store_cdf(bt.S_hi, bt.S_lo, sb + c, s[q]);
  }
  if (do_dots) {
    float2 sh[kCPT];
#pragma unroll
    for (int q = 0; q < kCPT; ++q) sh[q] = make_float2(s[q].re.hi, s[q].im.hi);
    column_dots(bt.V_hi + vb, bt.N, N, c0, sh, j, part, bt.dot + (size_t)b * 2 * (bt.maxit + 1) + (bt.maxit + 1));
  } else {
    float acc[1] = {0.f};
#pragma unroll
    for (int q = 0; q < kCPT; ++q) acc[0] += s[q].re.hi * s[q].re.hi + s[q].im.hi * s[q].im.hi;
    block_reduce_add<1>(acc, red);
    if (threadIdx.x == 0) atomicAdd(&bt.snorm2[b], (double)acc[0]);
  }
  if (threadIdx.x == 0) {
    int n = min(kArnT * kCPT, N - (int)(blockIdx.x * kArnT * kCPT));
    atomicAdd(&bt.work[KC_ORTHO], (unsigned long long)n * (unsigned long long)(j + 1));
  }
}

// pass 3 of CGS2 (mode 1 above): s'' = S - V c2 with float32 products folded every 8 columns
__global__ void __launch_bounds__(kArnT, 6) k_update_second(Batch bt, FineExact fe) {
  const int j = *bt.jdev;
  __shared__ float red[32];
  __shared__ float2 cf[kMaxCol];
  const int b = blockIdx.y;
  if (!bt.active[b]) return;
  const int N = fe.N;
  const double2* dsrc = bt.dot + (size_t)b * 2 * (bt.maxit + 1) + (bt.maxit + 1);
  for (int i = threadIdx.x; i <= j; i += blockDim.x) cf[i] = make_float2((float)dsrc[i].x, (float)dsrc[i].y);
  __syncthreads();
  const int c0 = blockIdx.x * kArnT * kCPT + threadIdx.x;
  const size_t sb = (size_t)b * bt.N, vb = (size_t)b * (bt.maxit + 1) * bt.N;
  cdf s[kCPT];
#pragma unroll
  for (int q = 0; q < kCPT; ++q) {
    const int c = c0 + q * kArnT;
    s[q] = c < N ? load_cdf(bt.S_hi, bt.S_lo, sb + c) : cdf{{0.f, 0.f}, {0.f, 0.f}};
  }
  for (int i0 = 0; i0 <= j; i0 += 8) {
    const int ie = min(i0 + 8, j + 1);
    float2 t[kCPT];
#pragma unroll
    for (int q = 0; q < kCPT; ++q) t[q] = make_float2(0.f, 0.f);
    for (int i = i0; i < ie; ++i) {
      const float2 ci = cf[i];
      const float2* vh = bt.V_hi + vb + (size_t)i * bt.N;
#pragma unroll
      for (int q = 0; q < kCPT; ++q) {
        const int c = c0 + q * kArnT;
        if (c < N) {
          const float2 h = vh[c];
          t[q].x = fmaf(h.x, ci.x, fmaf(-h.y, ci.y, t[q].x));
          t[q].y = fmaf(h.x, ci.y, fmaf(h.y, ci.x, t[q].y));
        }
      }
    }
#pragma unroll
    for (int q = 0; q < kCPT; ++q) {
      s[q].re = df_add_f(s[q].re, -t[q].x);
      s[q].im = df_add_f(s[q].im, -t[q].y);
    }
  }
  float acc[1] = {0.f};
#pragma unroll
  for (int q = 0; q < kCPT; ++q) {
    const int c = c0 + q * kArnT;
    if (c < N) {
      store_cdf(bt.S_hi, bt.S_lo, sb + c, s[q]);
      acc[0] += s[q].re.hi * s[q].re.hi + s[q].im.hi * s[q].im.hi;
    }
  }
  block_reduce_add<1>(acc, red);
  if (threadIdx.x == 0) {
    atomicAdd(&bt.snorm2[b], (double)acc[0]);
    const int n = min(kArnT * kCPT, N - (int)(blockIdx.x * kArnT * kCPT));
    atomicAdd(&bt.work[KC_ORTHO], (unsigned long long)n * (unsigned long long)(j + 1));
  }
}

// v_{j+1} = s'' / h, h = float(||s''||); H column j
__global__ void k_normalize(Batch bt, int) {
  const int j = *bt.jdev;   // outer iteration (device counter, so one captured graph serves every j)
  int b = blockIdx.y;
  if (!bt.active[b]) return;
  float h = (float)sqrt(bt.snorm2[b]);
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < bt.N) {
    size_t si = (size_t)b * bt.N + c;
    cdf s = load_cdf(bt.S_hi, bt.S_lo, si);
    cdf v;
    if (h > 0.f) {
      v.re = df_div_f(s.re, h);
      v.im = df_div_f(s.im, h);
    } else {
      v = {{0.f, 0.f}, {0.f, 0.f}};
    }
    store_cdf(bt.V_hi, bt.V_lo, ((size_t)b * (bt.maxit + 1) + j + 1) * bt.N + c, v);
  }
  if (blockIdx.x == 0) {
    const double2* d = bt.dot + (size_t)b * 2 * (bt.maxit + 1);
    double2* Hc = bt.H + ((size_t)b * bt.maxit + j) * (bt.maxit + 1);
    for (int i = threadIdx.x; i <= j + 1; i += blockDim.x) {
      if (i <= j) {
        // exactly the coefficients the updates subtracted: float c1 + float c2 (two passes), or the
        // hi + lo float pair of the df32-accurate c1 (one pass)
        double2 a = d[i], a2 = d[bt.maxit + 1 + i];
        if (bt.gs_passes == 1) {
          const float hx = (float)a.x, hy = (float)a.y;
          Hc[i] = make_double2((double)hx + (double)(float)(a.x - (double)hx),
                               (double)hy + (double)(float)(a.y - (double)hy));
        } else {
          Hc[i] = make_double2((double)(float)a.x + (double)(float)a2.x, (double)(float)a.y + (double)(float)a2.y);
        }
      } else {
        Hc[i] = make_double2((double)h, 0.0);
      }
    }
  }
}

void launch_dots_df(const Batch& bt, const FineExact& fe, dim3 g, cudaStream_t st);

void launch_arnoldi(const Batch& bt, const FineExact& fe, int j, cudaStream_t st, int* nlaunch, Prof* pf) {
  dim3 g((fe.N + kArnT * kCPT - 1) / (kArnT * kCPT), bt.nb);
  if (bt.gs_passes == 1) {
    // one classical pass whose coefficients come from df32 dots (V read twice per column)
    prof_begin(pf, KC_DOTS, st);
    launch_dots_df(bt, fe, g, st);
    prof_end(pf, KC_DOTS, st);
    prof_begin(pf, KC_ORTHO, st);
    k_update<<<g, kArnT, 0, st>>>(bt, fe, j, 2);
    prof_end(pf, KC_ORTHO, st);
    *nlaunch -= 1;
  } else {
    prof_begin(pf, KC_DOTS, st);
    k_dots1<<<g, kArnT, 0, st>>>(bt, fe, j);
    prof_end(pf, KC_DOTS, st);
    prof_begin(pf, KC_ORTHO, st);
    k_update<<<g, kArnT, 0, st>>>(bt, fe, j, 0);
    prof_end(pf, KC_ORTHO, st);
    prof_begin(pf, KC_ORTHO, st);
    k_update_second<<<g, kArnT, 0, st>>>(bt, fe);
    prof_end(pf, KC_ORTHO, st);
  }
  dim3 gn((fe.N + 255) / 256, bt.nb);
  k_normalize<<<gn, 256, 0, st>>>(bt, j);
  *nlaunch += 4;
}

// ------------------------------------------------------------ all-shift least squares (GMRES-Sh)
__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 zconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double zabs(double2 a) { return hypot(a.x, a.y); }

__global__ void k_shift_ls(Batch bt, int) {
  const int j = *bt.jdev;   // outer iteration (device counter, so one captured graph serves every j)
  __shared__ double2 hcol[1024];
  __shared__ int any;
  __shared__ unsigned long long rmax_bits;
  int b = blockIdx.x;
  if (!bt.active[b]) return;
  if (threadIdx.x == 0) { any = 0; rmax_bits = 0ull; }
  const double2* Hc = bt.H + ((size_t)b * bt.maxit + j) * (bt.maxit + 1);
  for (int i = threadIdx.x; i <= j + 1; i += blockDim.x) hcol[i] = Hc[i];
  __syncthreads();
  double2 tau = bt.tau_cur[b];
  const int M = bt.maxit;
  int mine = 0;
  for (int sh = bt.shift_off[b] + threadIdx.x; sh < bt.shift_off[b + 1]; sh += blockDim.x) {
    if (bt.conv_it[sh] > 0) continue;
    double2 z = bt.zsh[sh];
    double2 dz = make_double2(z.x - tau.x, z.y - tau.y);
    double2* Rc = bt.R + ((size_t)sh * M + j) * M;
    double* rc = bt.rc + (size_t)sh * M;
    double2* rs = bt.rs + (size_t)sh * M;
    double2 carry = zmul(dz, hcol[0]);
    if (j == 0) carry.x += 1.0;
    for (int i = 0; i < j; ++i) {
      double2 nxt = zmul(dz, hcol[i + 1]);
      if (i + 1 == j) nxt.x += 1.0;
      double c = rc[i];
      double2 s = rs[i];
      double2 top = zmul(s, nxt);
      top.x += c * carry.x; top.y += c * carry.y;
      double2 bot = zmul(zconj(s), carry);
      bot.x = c * nxt.x - bot.x; bot.y = c * nxt.y - bot.y;
      Rc[i] = top;
      carry = bot;
    }
    double2 bb = zmul(dz, hcol[j + 1]);
    double na = zabs(carry), nb = zabs(bb);
    double rho = hypot(na, nb);
    double c;
    double2 s;
    double2 rjj;
    if (rho == 0.0) {
      c = 1.0; s = make_double2(0.0, 0.0); rjj = make_double2(0.0, 0.0);
    } else if (na == 0.0) {
      c = 0.0; s = make_double2(bb.x / nb, -bb.y / nb); rjj = make_double2(nb, 0.0);
    } else {
      c = na / rho;
      double2 ph = make_double2(carry.x / na, carry.y / na);
      s = zmul(ph, make_double2(bb.x / rho, -bb.y / rho));
      rjj = make_double2(ph.x * rho, ph.y * rho);
    }
    Rc[j] = rjj;
    rc[j] = c;
    rs[j] = s;
    double2* g = bt.g + (size_t)sh * (M + 1);
    double2 gj = g[j];
    g[j] = make_double2(c * gj.x, c * gj.y);
    double2 gn = zmul(zconj(s), gj);
    g[j + 1] = make_double2(-gn.x, -gn.y);
    // GMRES-Sh: the least-squares residual |g_{j+1}|.  FOM-Sh: the square system H_j(z; T_j) y = e_1
    // is the Givens-reduced one without the last rotation, whose residual is
    // |eta_k| = |h_{j+1,j} (z - tau_j) y_j| = |g_{j+1}| / c_j (Sec. 3.1, Proposition 1); c_j = 0 means
    // H_j(z; T_j) is singular and the FOM coefficients do not exist at this j.
    double res = zabs(g[j + 1]);
    if (bt.krylov == 1) res = c > 0.0 ? res / c : INFINITY;
    bt.pres[sh] = res;
    if (bt.stop_rule == 0) {
      // stop at half the tolerance: the true residual adds the (relaxed) inner-solve
      // error e_j y_j and the float32 loss of orthogonality on top of the projected one
      if (res <= 0.5 * bt.tol || rho == 0.0 || hcol[j + 1].x == 0.0) {
        bt.conv_it[sh] = j + 1;
      } else {
        mine = 1;
        atomicMax(&rmax_bits, (unsigned long long)__double_as_longlong(res));   // res >= 0: bit order = value order
      }
    }
  }
  if (bt.stop_rule == 1) {
    // quadrature-weighted rule: the nk shifts of one output time stop together once
    // sum_k |w_k qhat_k| rho_k <= tol/2 sum_k |w_k qhat_k| (the bound of Proposition 1 on the
    // residual of the quadrature sum, relative to that of its right-hand side)
    __syncthreads();
    const int s0 = bt.shift_off[b], s1 = bt.shift_off[b + 1], nk = bt.nk;
    for (int t0 = s0 + threadIdx.x * nk; t0 < s1; t0 += blockDim.x * nk) {
      if (bt.conv_it[t0] > 0) continue;
      double num = 0.0, den = 0.0, worst = 0.0;
      for (int sh = t0; sh < t0 + nk; ++sh) {
        num += bt.wabs[sh] * bt.pres[sh];
        den += bt.wabs[sh];
        worst = fmax(worst, bt.pres[sh]);
      }
      if (num <= 0.5 * bt.tol * den || hcol[j + 1].x == 0.0) {
        for (int sh = t0; sh < t0 + nk; ++sh) bt.conv_it[sh] = j + 1;
      } else {
        mine = 1;
        atomicMax(&rmax_bits, (unsigned long long)__double_as_longlong(worst));
      }
    }
  }
  if (mine) atomicOr(&any, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    bt.nit[b] = j + 1;
    bt.active[b] = (any && j + 1 < M) ? 1 : 0;
    bt.rmax[b] = __longlong_as_double((long long)rmax_bits);
  }
}

__global__ void k_next_iter(Batch bt) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *bt.jdev += 1;
}

void launch_shift_ls(const Batch& bt, int j, cudaStream_t st) {
  k_shift_ls<<<bt.nb, 256, 0, st>>>(bt, j);
  k_next_iter<<<1, 32, 0, st>>>(bt);
}
void launch_shift_ls_only(const Batch& bt, int j, cudaStream_t st) { k_shift_ls<<<bt.nb, 256, 0, st>>>(bt, j); }
void launch_next_iter(const Batch& bt, cudaStream_t st) { k_next_iter<<<1, 32, 0, st>>>(bt); }

// y_k = R^{-1} g over the shift's converged (or final) column count
__global__ void k_backsolve(Batch bt, const int* sh_basis, int s0, int s1) {
  int sh = s0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (sh >= s1) return;
  const int M = bt.maxit;
  int m = bt.conv_it[sh] > 0 ? bt.conv_it[sh] : bt.nit[sh_basis[sh]];
  const double2* R = bt.R + (size_t)sh * M * M;
  const double2* g = bt.g + (size_t)sh * (M + 1);
  double2* y = bt.Y + (size_t)sh * M;
  for (int i = m; i < M; ++i) y[i] = make_double2(0.0, 0.0);
  // FOM-Sh: the last equation of the square system takes the pre-rotation entries, which
  // amounts to g_{m-1} / c_{m-1}^2 against the rotated R (the other rows are the same)
  const double cl = bt.rc[(size_t)sh * M + (m > 0 ? m - 1 : 0)];
  for (int i = m - 1; i >= 0; --i) {
    double2 acc = g[i];
    if (bt.krylov == 1 && i == m - 1) {
      const double f = cl > 0.0 ? 1.0 / (cl * cl) : 0.0;
      acc.x *= f; acc.y *= f;
    }
    for (int l = i + 1; l < m; ++l) {
      double2 t = zmul(R[(size_t)l * M + i], y[l]);
      acc.x -= t.x; acc.y -= t.y;
    }
    double2 d = R[(size_t)i * M + i];
    double den = d.x * d.x + d.y * d.y;
    y[i] = den > 0 ? make_double2((acc.x * d.x + acc.y * d.y) / den, (acc.y * d.x - acc.x * d.y) / den)
                   : make_double2(0.0, 0.0);
  }
}

void launch_backsolve_map(const Batch& bt, const int* sh_basis, cudaStream_t st, int s0, int s1) {
  if (s1 < 0) s1 = bt.nsh;
  if (s1 <= s0) return;
  k_backsolve<<<(s1 - s0 + 127) / 128, 128, 0, st>>>(bt, sh_basis, s0, s1);
}

// ------------------------------------------------------------ quadrature (Eq. half)
__global__ void k_quad_coef(Batch bt, const QuadItem* items, int nitems, const double2* wq, double2* C) {
  int q = blockIdx.x;
  if (q >= nitems) return;
  QuadItem it = items[q];
  const int M = bt.maxit;
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    double2 acc = make_double2(0.0, 0.0);
    for (int k = 0; k < it.nk; ++k) {
      double2 t = zmul(wq[it.sh0 + k], bt.Y[(size_t)(it.sh0 + k) * M + i]);
      acc.x += t.x; acc.y += t.y;
    }
    C[(size_t)q * M + i] = acc;
  }
}

void launch_quad_coef(const Batch& bt, const QuadItem* items, int nitems, const double2* wq, double2* C,
                      cudaStream_t st) {
  k_quad_coef<<<nitems, 128, 0, st>>>(bt, items, nitems, wq, C);
}

// Re (U_b[cell] . C_q) over the basis's columns, df32 U read as double
__device__ __forceinline__ double quad_dot(const Batch& bt, const QuadItem& it, const double2* C, int q, int64_t cell,
                                           int m) {
  const int M = bt.maxit;
  double acc = 0.0;
  for (int i = 0; i < m; ++i) {
    size_t ui = ((size_t)it.basis * M + i) * bt.N + cell;
    float2 hi = bt.U_hi[ui], lo = bt.U_lo ? bt.U_lo[ui] : make_float2(0.f, 0.f);
    double2 c = C[(size_t)q * M + i];
    acc += ((double)hi.x + (double)lo.x) * c.x - ((double)hi.y + (double)lo.y) * c.y;
  }
  return acc;
}

// h[s][r][t] = 2 Re (U[rcell] . C_{s,t}) (+ the initial-state item dense_q0 + t, the same for every s)
__global__ void k_measure(Batch bt, const QuadItem* items, const double2* C, int ns, int nr, int nt,
                          const int64_t* rcells, double* h, int dense_q0) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= ns * nr * nt) return;
  int t = idx % nt, r = (idx / nt) % nr, s = idx / (nt * nr);
  int q = s * nt + t;
  int64_t cell = rcells[r];
  const QuadItem it = items[q];
  double acc = quad_dot(bt, it, C, q, cell, bt.nit[it.basis]);
  if (dense_q0 >= 0) {
    const QuadItem id = items[dense_q0 + t];
    acc += quad_dot(bt, id, C, dense_q0 + t, cell, bt.nit[id.basis]);
  }
  h[idx] = 2.0 * acc;
}

void launch_measure(const Batch& bt, const QuadItem* items, const double2* C, int ns, int nr, int nt,
                    const int64_t* rcells, double* h, cudaStream_t st, int dense_q0) {
  int n = ns * nr * nt;
  k_measure<<<(n + 127) / 128, 128, 0, st>>>(bt, items, C, ns, nr, nt, rcells, h, dense_q0);
}

// phi[q][c] for the items q = s * nt + t (+ the initial-state item dense_q0 + t)
__global__ void k_fields(Batch bt, const QuadItem* items, const double2* C, double* phi, int nt, int dense_q0) {
  int q = blockIdx.y;
  int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= bt.N) return;
  QuadItem it = items[q];
  double acc = quad_dot(bt, it, C, q, c, bt.nit[it.basis]);
  if (dense_q0 >= 0) {
    const int qd = dense_q0 + q % nt;
    acc += quad_dot(bt, items[qd], C, qd, c, bt.nit[items[qd].basis]);
  }
  phi[(size_t)q * bt.N + c] = 2.0 * acc;
}

void launch_fields(const Batch& bt, const QuadItem* items, const double2* C, int nitems, double* phi,
                   cudaStream_t st, int nt, int dense_q0) {
  dim3 g((unsigned)((bt.N + 255) / 256), nitems);
  k_fields<<<g, 256, 0, st>>>(bt, items, C, phi, nt, dense_q0);
}

// ------------------------------------------------------------ true residual (the convergence check)
constexpr int kXS = 16;   // shifts per pass (U is read once per pass)

// one-pass Gram-Schmidt: dot[0][i] = V_i^H (M u_j) with V and M u_j in df32; each thread sums its
// cells in df32, the block and the grid in double (a few additions per block)
__global__ void __launch_bounds__(kArnT) k_dots_df(Batch bt, FineExact fe) {
  const int j = *bt.jdev;
  __shared__ double2 part[kWarps][kMaxCol];
  const int b = blockIdx.y;
  if (!bt.active[b]) return;
  const int N = fe.N;
  const int c0 = blockIdx.x * kArnT * kCPT + threadIdx.x;
  cdf s[kCPT];
  const size_t ub = ((size_t)b * bt.maxit + j) * bt.N;
#pragma unroll
  for (int q = 0; q < kCPT; ++q) {
    const int c = c0 + q * kArnT;
    s[q] = c < N ? cdf_mul_r(load_cdf(bt.U_hi, bt.U_lo, ub + c), ldf(fe.m_hi, fe.m_lo, c))
                 : cdf{{0.f, 0.f}, {0.f, 0.f}};
  }
  const size_t vb = (size_t)b * (bt.maxit + 1) * bt.N;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i0 = 0; i0 <= j; i0 += kIG) {
    double acc[2 * kIG];
#pragma unroll
    for (int ii = 0; ii < kIG; ++ii) {
      acc[2 * ii] = acc[2 * ii + 1] = 0.0;
      const int i = i0 + ii;
      if (i > j) continue;
      const float2* vh = bt.V_hi + vb + (size_t)i * bt.N;
      const float2* vl = lo_at(bt.V_lo, vb + (size_t)i * bt.N);
      df re = {0.f, 0.f}, im = {0.f, 0.f};
#pragma unroll
      for (int q = 0; q < kCPT; ++q) {
        const int c = c0 + q * kArnT;
        if (c < N) {
          const cdf v = load_cdf(vh, vl, c);
          re = df_fma2(re, v.re, s[q].re, df_neg(v.im), s[q].im);   // + vr sr + vi si
          im = df_fma2(im, v.re, s[q].im, v.im, s[q].re);           // + vr si - vi sr
        }
      }
      acc[2 * ii] = (double)re.hi + (double)re.lo;
      acc[2 * ii + 1] = (double)im.hi + (double)im.lo;
    }
    const double r = warp_sum8(acc, lane);
    const int k = lane >> 2;
    if ((lane & 3) == 0 && i0 + (k >> 1) <= j) {
      double* slot = reinterpret_cast<double*>(&part[warp][i0 + (k >> 1)]);
      slot[k & 1] = r;
    }
  }
  __syncthreads();
  double2* dst = bt.dot + (size_t)b * 2 * (bt.maxit + 1);
  for (int i = threadIdx.x; i <= j; i += blockDim.x) {
    double re = 0.0, im = 0.0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
      re += part[w][i].x;
      im += part[w][i].y;
    }
    atomicAdd(&dst[i].x, re);
    atomicAdd(&dst[i].y, im);
  }
  if (threadIdx.x == 0) {
    const int n = min(kArnT * kCPT, N - (int)(blockIdx.x * kArnT * kCPT));
    atomicAdd(&bt.work[KC_DOTS], (unsigned long long)n * (unsigned long long)(j + 1));
  }
}

void launch_dots_df(const Batch& bt, const FineExact& fe, dim3 g, cudaStream_t st) {
  k_dots_df<<<g, kArnT, 0, st>>>(bt, fe);
}


// X[sh] = U_b y_sh for every shift of basis b (df32 accumulation); ys: [kXS][maxit] in shared memory.
// A chunk of kXS shifts runs over the columns of its latest-converging shift only (the coefficients
// of a shift beyond its own convergence are zero).
__global__ void __launch_bounds__(256) k_xk(Batch bt, float2* X_hi, float2* X_lo) {
  extern __shared__ cdf ys[];
  __shared__ int s_m;
  int b = blockIdx.y;
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int M = bt.maxit;
  int s0 = bt.shift_off[b], s1 = bt.shift_off[b + 1];
  size_t ub = (size_t)b * M * bt.N;
  for (int sa = s0; sa < s1; sa += kXS) {
    __syncthreads();
    if (threadIdx.x == 0) {
      int mm = 0;
      for (int sh = sa; sh < min(sa + kXS, s1); ++sh) mm = max(mm, bt.conv_it[sh] > 0 ? bt.conv_it[sh] : bt.nit[b]);
      s_m = min(mm, bt.nit[b]);
    }
    __syncthreads();
    const int m = s_m;
    for (int idx = threadIdx.x; idx < kXS * m; idx += blockDim.x) {
      int q = idx / m, i = idx % m;
      int sh = sa + q;
      double2 y = sh < s1 ? bt.Y[(size_t)sh * M + i] : make_double2(0.0, 0.0);
      ys[q * m + i] = {df_from_double(y.x), df_from_double(y.y)};
    }
    __syncthreads();
    if (c < bt.N) {
      cdf acc[kXS];
#pragma unroll
      for (int q = 0; q < kXS; ++q) acc[q] = {{0.f, 0.f}, {0.f, 0.f}};
      for (int i = 0; i < m; ++i) {
        cdf u = load_cdf(bt.U_hi, bt.U_lo, ub + (size_t)i * bt.N + c);
#pragma unroll
        for (int q = 0; q < kXS; ++q) acc[q] = cdf_fma(acc[q], u, ys[q * m + i]);
      }
#pragma unroll
      for (int q = 0; q < kXS; ++q)
        if (sa + q < s1) store_cdf(X_hi, X_lo, (size_t)(sa + q) * bt.N + c, acc[q]);
    }
  }
}

void launch_xk(const Batch& bt, float2* X_hi, float2* X_lo, cudaStream_t st, Prof* pf) {
  static bool attr = false;
  const size_t smem_max = (size_t)kXS * 256 * sizeof(cdf);   // maxit <= 250
  if (!attr) {
    cudaFuncSetAttribute(k_xk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max);
    attr = true;
  }
  dim3 g((unsigned)((bt.N + 255) / 256), bt.nb);
  prof_begin(pf, KC_XK, st);
  k_xk<<<g, 256, (size_t)kXS * bt.maxit * sizeof(cdf), st>>>(bt, X_hi, X_lo);
  prof_end(pf, KC_XK, st);
}

__global__ void k_true_res(Batch bt, FineExact fe, const int* sh_basis, const float2* X_hi, const float2* X_lo,
                           double* res2, int s0) {
  __shared__ float red[32];
  int sh = s0 + blockIdx.y;
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  float acc[1] = {0.f};
  if (c < fe.N) {
    double2 z = bt.zsh[sh];
    df zr = df_from_double(z.x), zi = df_from_double(z.y);
    const float2* xh = X_hi + (size_t)sh * bt.N;
    const float2* xl = lo_at(X_lo, (size_t)sh * bt.N);
    cdf ax = apply_exact(fe, xh, xl, c, zr, zi);
    const int64_t rc = bt.rhs_cell[sh_basis[sh]];
    df e = {(c == rc) ? 1.f : 0.f, 0.f};
    if (rc < 0) e = {bt.rhs_hi[c], bt.rhs_lo[c]};
    cdf r = cdf_sub({e, {0.f, 0.f}}, ax);
    acc[0] = r.re.hi * r.re.hi + r.im.hi * r.im.hi;
  }
  block_reduce_add<1>(acc, red);
  if (threadIdx.x == 0) atomicAdd(&res2[sh], (double)acc[0]);
}

void launch_true_res(const Batch& bt, const FineExact& fe, const int* sh_basis, const float2* X_hi,
                     const float2* X_lo, double* res2, cudaStream_t st, Prof* pf, int s0, int s1) {
  if (s1 < 0) s1 = bt.nsh;
  if (s1 <= s0) return;
  dim3 g2((unsigned)((bt.N + 255) / 256), s1 - s0);
  prof_begin(pf, KC_TRUE_RES, st);
  k_true_res<<<g2, 256, 0, st>>>(bt, fe, sh_basis, X_hi, X_lo, res2, s0);
  prof_end(pf, KC_TRUE_RES, st);
}

}  // namespace lt
