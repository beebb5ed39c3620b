// block.cu -- block flexible GMRES for shifted systems: Algorithm 1 (Sec. 3) with the point sources
// of one time group taken as one block of right-hand sides (the block Krylov variant that Sec. 6
// leaves to future work).
//
// The p sources of group g keep their own bases b_q = q * G + g, so their preconditioner solves
// are the ordinary ones; the Arnoldi process and the least squares are shared by the block:
//   s_q = M u_j^{(q)} is orthogonalised against every member's columns v_i^{(q')}, i <= j, by
//   classical Gram-Schmidt twice (float32 dots, df32 updates; V is read once for all p members);
//   the p vectors are orthonormalised together by CholQR2: Gram matrix from the hi planes,
//   Cholesky in double, V <- S W with W = R^{-1} rounded to float32 and applied in df32, twice;
//   the subdiagonal block H_{j+1,j} = (W_1 W_2)^{-1} is exactly the inverse of what was applied,
//   so M U_j = V_{j+1} Hbar_j holds to df32 accuracy whatever the rounding of W;
//   every shift solves min || E_1 - Hbar(z_k; T_j) Y || for its p right-hand sides at once by
//   Givens rotations, p per column (the lower bandwidth of the block Hessenberg matrix is p);
//   right-hand side q of shift k stops when its residual, the norm of rows (j+1)p..(j+2)p-1 of
//   column q of the rotated E_1, falls to tol/2.
// Column c = i * p + q' of the block is column i of member q'.  The point right-hand sides e_cell
// of distinct cells are orthonormal, so V_1 = B and beta = I.
#include <algorithm>
#include <cstdio>
#include "df32.cuh"
#include "exact.cuh"
#include "lt_internal.h"
#include "lt_kernels.h"

namespace lt {

constexpr int kBT = 256;        // threads per CTA of the vector kernels
constexpr int kBAcc = 2048;     // float2 accumulators / coefficients staged in shared memory

__device__ __forceinline__ size_t vcol_off(const Batch& bt, int g, int col) {
  const int p = bt.bp, i = col / p, q = col - i * p;
  return ((size_t)(q * bt.ngroups + g) * (bt.maxit + 1) + i) * bt.N;
}
__device__ __forceinline__ size_t ucol_off(const Batch& bt, int g, int col) {
  const int p = bt.bp, i = col / p, q = col - i * p;
  return ((size_t)(q * bt.ngroups + g) * bt.maxit + i) * bt.N;
}

// Sum of NV = 2^k values over the warp, scattered: on return lane l holds the warp total of value
// index l >> (5 - k) (halving exchanges while the values outnumber the lanes left, then plain
// butterfly steps): NV - 1 shuffles instead of 5 NV.
template <int NV>
__device__ __forceinline__ float warp_reduce_scatter(float (&v)[NV], int lane) {
  int o = 16;
#pragma unroll
  for (int h = NV / 2; h >= 1; h >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < h; ++i) {
      const float send = up ? v[i] : v[i + h];
      const float keep = up ? v[i + h] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
    o >>= 1;
  }
  float r = v[0];
  for (; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
  return r;
}
template <int NV>
struct Log2 { static constexpr int v = 1 + Log2<NV / 2>::v; };
template <>
struct Log2<1> { static constexpr int v = 0; };

// Tiles of kBT * CPT cells; a CTA takes tiles blockIdx.x, blockIdx.x + gridDim.x, ...
template <int CPT>
__device__ __forceinline__ int n_tiles(int N) { return (N + kBT * CPT - 1) / (kBT * CPT); }

// Column dots D[col][q] += x_col^H s_q for col < ncol, q < p, from the hi planes, over the CTA's
// tiles: load(cell0, s) gives the members' values at the thread's CPT cells (cell0 + c * kBT) of a
// tile; xcol(col) points at column col.  Per column each warp reduce-scatters its 2 PMAX partial
// sums and adds them into float shared accumulators; a chunk of columns ends with one double
// atomicAdd per (col, q) and CTA.
template <int PMAX, int CPT, class Load, class XCol>
__device__ void block_dots(Load load, XCol xcol, int ncol, int p, int N, double2* D, float2* acc) {
  constexpr int CH = kBAcc / PMAX;
  constexpr int NV = 2 * PMAX <= 8 ? 8 : 2 * PMAX <= 16 ? 16 : 32;   // values reduced, padded to a power of two
  constexpr int SH = 5 - Log2<NV>::v;
  const int lane = threadIdx.x & 31;
  const int idx = lane >> SH;
  const bool owner = (lane & ((1 << SH) - 1)) == 0 && idx < 2 * PMAX;
  const int q_own = idx < PMAX ? idx : idx - PMAX;
  const int nt = n_tiles<CPT>(N);
  for (int cb = 0; cb < ncol; cb += CH) {
    const int ce = min(cb + CH, ncol);
    for (int i = threadIdx.x; i < (ce - cb) * p; i += blockDim.x) acc[i] = make_float2(0.f, 0.f);
    __syncthreads();
    for (int tile = blockIdx.x; tile < nt; tile += gridDim.x) {
      const int cell0 = tile * kBT * CPT + threadIdx.x;
      float2 s[PMAX][CPT];
      load(cell0, s);
      for (int col = cb; col < ce; ++col) {
        const float2* x = xcol(col);
        float v[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) v[q] = 0.f;
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
          const int cell = cell0 + c * kBT;
          if (cell < N) {
            const float2 a = x[cell];
#pragma unroll
            for (int q = 0; q < PMAX; ++q) {
              v[q] = fmaf(a.x, s[q][c].x, fmaf(a.y, s[q][c].y, v[q]));
              v[PMAX + q] = fmaf(a.x, s[q][c].y, fmaf(-a.y, s[q][c].x, v[PMAX + q]));
            }
          }
        }
        const float r = warp_reduce_scatter<NV>(v, lane);
        if (owner && q_own < p) {
          float* dst = idx < PMAX ? &acc[(col - cb) * p + q_own].x : &acc[(col - cb) * p + q_own].y;
          atomicAdd(dst, r);
        }
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < (ce - cb) * p; i += blockDim.x) {
      atomicAdd(&D[(size_t)cb * p + i].x, (double)acc[i].x);
      atomicAdd(&D[(size_t)cb * p + i].y, (double)acc[i].y);
    }
    __syncthreads();
  }
}

// per-iteration reset of the group's accumulators (before the Gram-Schmidt dots)
__global__ void k_bzero(Batch bt) {
  const int g = blockIdx.x;
  if (!bt.active[g]) return;
  const int j = *bt.jdev, p = bt.bp;
  const size_t n = (size_t)(j + 1) * p * p;
  double2* d = bt.bdot + (size_t)g * 2 * bt.bld * p;
  for (size_t i = threadIdx.x; i < n; i += blockDim.x) {
    d[i] = make_double2(0.0, 0.0);
    d[(size_t)bt.bld * p + i] = make_double2(0.0, 0.0);
  }
  double2* gm = bt.bgram + (size_t)g * 2 * p * p;
  for (int i = threadIdx.x; i < 2 * p * p; i += blockDim.x) gm[i] = make_double2(0.0, 0.0);
  if (threadIdx.x == 0) {
    bt.gany[g] = 0;
    bt.grmax[g] = 0ull;
  }
}

// first Gram-Schmidt pass: bdot[g][0][col][q] = v_col^H (M u_j^{(q)})
template <int PMAX, int CPT>
__global__ void __launch_bounds__(kBT) k_bdots(Batch bt, FineExact fe) {
  __shared__ float2 acc[kBAcc];
  const int g = blockIdx.y;
  if (!bt.active[g]) return;
  const int j = *bt.jdev, p = bt.bp, N = fe.N, G = bt.ngroups;
  auto load = [&](int cell0, float2 (&s)[PMAX][CPT]) {
#pragma unroll
    for (int q = 0; q < PMAX; ++q)
#pragma unroll
      for (int c = 0; c < CPT; ++c) {
        const int cell = cell0 + c * kBT;
        s[q][c] = make_float2(0.f, 0.f);
        if (q < p && cell < N) {
          const float2 u = bt.U_hi[((size_t)(q * G + g) * bt.maxit + j) * bt.N + cell];
          const float m = fe.m_hi[cell];
          s[q][c] = make_float2(m * u.x, m * u.y);
        }
      }
  };
  const float2* V = bt.V_hi;
  auto xcol = [&](int col) { return V + vcol_off(bt, g, col); };
  block_dots<PMAX, CPT>(load, xcol, (j + 1) * p, p, N, bt.bdot + (size_t)g * 2 * bt.bld * p, acc);
}

// Gram-Schmidt updates of the block over the CTA's tiles.
// mode 0: s_q = M u_j^{(q)} - sum_col v_col c1[col][q] in df32 (the first pass cancels most of
//   M u_j, so every product enters exactly), S_q <- s_q, then the second pass's dots
//   bdot[g][1] = V^H S;
// mode 1: S_q <- S_q - sum_col v_col c2[col][q].  The second-pass coefficients are of the order of
//   the first pass's float32 dot error (about 2^-24 ||M u_j||), so their products are formed in
//   float32 from the hi planes and folded into the df32 S every 8 columns: the Arnoldi relation
//   keeps an error near 2^-24 * 2^-24 * 8 * sqrt(columns / 8) of ||M u_j|| (about 1e-13), while
//   the pass costs a seventh of the df32 one.
template <int PMAX, int CPT>
__global__ void __launch_bounds__(kBT) k_bupdate(Batch bt, FineExact fe, int mode) {
  __shared__ float2 cf[kBAcc];
  __shared__ float2 acc[kBAcc];
  constexpr int CH = kBAcc / PMAX;
  const int g = blockIdx.y;
  if (!bt.active[g]) return;
  const int j = *bt.jdev, p = bt.bp, N = fe.N, G = bt.ngroups;
  const int ncol = (j + 1) * p;
  const int nt = n_tiles<CPT>(N);
  const double2* D = bt.bdot + ((size_t)g * 2 + mode) * bt.bld * p;
  unsigned long long cells = 0;
  for (int tile = blockIdx.x; tile < nt; tile += gridDim.x) {
    const int cell0 = tile * kBT * CPT + threadIdx.x;
    cdf s[PMAX][CPT];
#pragma unroll
    for (int q = 0; q < PMAX; ++q)
#pragma unroll
      for (int c = 0; c < CPT; ++c) {
        const int cell = cell0 + c * kBT;
        s[q][c] = {{0.f, 0.f}, {0.f, 0.f}};
        if (q < p && cell < N) {
          const size_t b = (size_t)(q * G + g);
          s[q][c] = mode == 0 ? cdf_mul_r(load_cdf(bt.U_hi, bt.U_lo, (b * bt.maxit + j) * bt.N + cell),
                                          ldf(fe.m_hi, fe.m_lo, cell))
                              : load_cdf(bt.S_hi, bt.S_lo, b * bt.N + cell);
        }
      }
    for (int cb = 0; cb < ncol; cb += CH) {
      const int ce = min(cb + CH, ncol);
      __syncthreads();
      for (int i = threadIdx.x; i < (ce - cb) * p; i += blockDim.x) {
        const double2 d = D[(size_t)cb * p + i];
        cf[i] = make_float2((float)d.x, (float)d.y);
      }
      __syncthreads();
      if (mode == 0) {
        for (int col = cb; col < ce; ++col) {
          const size_t off = vcol_off(bt, g, col);
          const float2* vh = bt.V_hi + off;
          const float2* vl = lo_at(bt.V_lo, off);
#pragma unroll
          for (int c = 0; c < CPT; ++c) {
            const int cell = cell0 + c * kBT;
            if (cell < N) {
              const cdf v = load_cdf(vh, vl, cell);
#pragma unroll
              for (int q = 0; q < PMAX; ++q)
                if (q < p) {
                  const float2 k = cf[(col - cb) * p + q];
                  s[q][c] = cdf_sub_mul_cf(s[q][c], v, k.x, k.y);
                }
            }
          }
        }
      } else {
        for (int c8 = cb; c8 < ce; c8 += 8) {
          const int c8e = min(c8 + 8, ce);
          float2 t[PMAX][CPT];
#pragma unroll
          for (int q = 0; q < PMAX; ++q)
#pragma unroll
            for (int c = 0; c < CPT; ++c) t[q][c] = make_float2(0.f, 0.f);
          for (int col = c8; col < c8e; ++col) {
            const float2* vh = bt.V_hi + vcol_off(bt, g, col);
#pragma unroll
            for (int c = 0; c < CPT; ++c) {
              const int cell = cell0 + c * kBT;
              if (cell < N) {
                const float2 v = vh[cell];
#pragma unroll
                for (int q = 0; q < PMAX; ++q)
                  if (q < p) {
                    const float2 k = cf[(col - cb) * p + q];
                    t[q][c].x = fmaf(v.x, k.x, fmaf(-v.y, k.y, t[q][c].x));
                    t[q][c].y = fmaf(v.x, k.y, fmaf(v.y, k.x, t[q][c].y));
                  }
              }
            }
          }
#pragma unroll
          for (int q = 0; q < PMAX; ++q)
#pragma unroll
            for (int c = 0; c < CPT; ++c) {
              s[q][c].re = df_add_f(s[q][c].re, -t[q][c].x);
              s[q][c].im = df_add_f(s[q][c].im, -t[q][c].y);
            }
        }
      }
    }
#pragma unroll
    for (int q = 0; q < PMAX; ++q)
#pragma unroll
      for (int c = 0; c < CPT; ++c) {
        const int cell = cell0 + c * kBT;
        if (q < p && cell < N) store_cdf(bt.S_hi, bt.S_lo, (size_t)(q * G + g) * bt.N + cell, s[q][c]);
      }
    cells += (unsigned long long)min(kBT * CPT, N - tile * kBT * CPT);
  }
  if (mode == 0) {
    // the thread reads back the S cells it wrote itself
    auto load = [&](int cell0, float2 (&sh)[PMAX][CPT]) {
#pragma unroll
      for (int q = 0; q < PMAX; ++q)
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
          const int cell = cell0 + c * kBT;
          sh[q][c] = (q < p && cell < N) ? bt.S_hi[(size_t)(q * G + g) * bt.N + cell] : make_float2(0.f, 0.f);
        }
    };
    const float2* V = bt.V_hi;
    auto xcol = [&](int col) { return V + vcol_off(bt, g, col); };
    block_dots<PMAX, CPT>(load, xcol, ncol, p, N, bt.bdot + ((size_t)g * 2 + 1) * bt.bld * p, acc);
  }
  if (threadIdx.x == 0) atomicAdd(&bt.work[KC_ORTHO], cells * (unsigned long long)ncol * p);
}

// Gram matrix of the block's new vectors, from the hi planes: pass 0 of S (after Gram-Schmidt),
// pass 1 of V_{j+1} (after the first CholQR step).  bgram[g][pass][a][q] = x_a^H x_q.
template <int PMAX, int CPT>
__global__ void __launch_bounds__(kBT) k_bgram(Batch bt, int pass) {
  __shared__ float2 acc[kBAcc];
  const int g = blockIdx.y;
  if (!bt.active[g]) return;
  const int j = *bt.jdev, p = bt.bp, N = (int)bt.N, G = bt.ngroups;
  auto xcol = [&](int a) {
    const size_t b = (size_t)(a * G + g);
    return pass == 0 ? bt.S_hi + b * bt.N : bt.V_hi + (b * (bt.maxit + 1) + j + 1) * bt.N;
  };
  auto load = [&](int cell0, float2 (&s)[PMAX][CPT]) {
#pragma unroll
    for (int q = 0; q < PMAX; ++q) {
      const float2* x = xcol(q < p ? q : 0);
#pragma unroll
      for (int c = 0; c < CPT; ++c) {
        const int cell = cell0 + c * kBT;
        s[q][c] = (q < p && cell < N) ? x[cell] : make_float2(0.f, 0.f);
      }
    }
  };
  block_dots<PMAX, CPT>(load, xcol, p, p, N, bt.bgram + ((size_t)g * 2 + pass) * p * p, acc);
}


__device__ __forceinline__ double2 bz_mul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 bz_cmul(double2 a, double2 b) {   // conj(a) * b
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ double2 bz_div(double2 a, double2 b) {
  const double d = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

// inverse of an upper-triangular p x p matrix (row-major, complex double): X = A^{-1}, thread q < p
// solving for column q (call from every thread; a barrier follows in the caller)
__device__ void upper_inverse_cols(const double2* A, double2* X, int p) {
  const int q = threadIdx.x;
  if (q >= p) return;
  for (int l = 0; l < p; ++l) X[l * p + q] = make_double2(0.0, 0.0);
  X[q * p + q] = bz_div(make_double2(1.0, 0.0), A[q * p + q]);
  for (int l = q - 1; l >= 0; --l) {
    double2 acc = make_double2(0.0, 0.0);
    for (int k = l + 1; k <= q; ++k) {
      const double2 t = bz_mul(A[l * p + k], X[k * p + q]);
      acc.x += t.x; acc.y += t.y;
    }
    X[l * p + q] = bz_div(make_double2(-acc.x, -acc.y), A[l * p + l]);
  }
}

// CholQR step of pass `pass`: Gram = R^H R (right-looking Cholesky in double, the row and trailing
// updates of each step spread over the CTA), W = R^{-1} rounded to float32 into bw[g][pass].  A
// pivot below 1e-26 of its column's squared norm (numerical rank loss of the block) is raised to
// that floor, so W stays finite; the Arnoldi relation still holds exactly because H takes the
// inverse of the W that was applied.  Pass 1 also writes block column j of H: rows i p + q' (i <= j)
// the Gram-Schmidt coefficients the updates subtracted, rows (j+1)p + l the subdiagonal block
// (W_1 W_2)^{-1}.
__global__ void __launch_bounds__(256) k_bchol(Batch bt, int pass) {
  __shared__ double2 Gm[256], Rm[256], Wd[256], T[256];
  __shared__ double diag0[16];
  const int g = blockIdx.x;
  if (!bt.active[g]) return;
  const int j = *bt.jdev, p = bt.bp, tid = threadIdx.x, nt = blockDim.x;
  const double2* gram = bt.bgram + ((size_t)g * 2 + pass) * p * p;
  float2* W = bt.bw + ((size_t)g * 2 + pass) * p * p;
  for (int i = tid; i < p * p; i += nt) {
    Gm[i] = gram[i];
    Rm[i] = make_double2(0.0, 0.0);
  }
  __syncthreads();
  if (tid < p) diag0[tid] = Gm[tid * p + tid].x;
  __syncthreads();
  for (int q = 0; q < p; ++q) {
    if (tid == 0) {
      double d = Gm[q * p + q].x;
      const double floor_d = fmax(1e-26 * diag0[q], 1e-280);
      if (!(d > floor_d)) d = floor_d;
      Rm[q * p + q] = make_double2(sqrt(d), 0.0);
    }
    __syncthreads();
    const double rq = Rm[q * p + q].x;
    for (int c = q + 1 + tid; c < p; c += nt) {
      const double2 a = Gm[q * p + c];
      Rm[q * p + c] = make_double2(a.x / rq, a.y / rq);
    }
    __syncthreads();
    const int w = p - q - 1;
    for (int idx = tid; idx < w * w; idx += nt) {
      const int a = q + 1 + idx / w, c = q + 1 + idx % w;
      if (a <= c) {
        const double2 t = bz_cmul(Rm[q * p + a], Rm[q * p + c]);
        Gm[a * p + c].x -= t.x;
        Gm[a * p + c].y -= t.y;
      }
    }
    __syncthreads();
  }
  upper_inverse_cols(Rm, Wd, p);
  __syncthreads();
  // W as applied: float32 entries
  for (int i = tid; i < p * p; i += nt) {
    const float2 wf = make_float2((float)Wd[i].x, (float)Wd[i].y);
    W[i] = wf;
    Wd[i] = make_double2((double)wf.x, (double)wf.y);
  }
  if (pass == 0) return;
  __syncthreads();
  // T = W_1 W_2 (both upper triangular, float entries), then Hsub = T^{-1} into Rm
  const float2* W1 = bt.bw + (size_t)g * 2 * p * p;
  for (int idx = tid; idx < p * p; idx += nt) {
    const int l = idx / p, q = idx % p;
    double2 acc = make_double2(0.0, 0.0);
    for (int k = l; k <= q; ++k) {
      const double2 t = bz_mul(make_double2(W1[l * p + k].x, W1[l * p + k].y), Wd[k * p + q]);
      acc.x += t.x; acc.y += t.y;
    }
    T[idx] = acc;
  }
  __syncthreads();
  upper_inverse_cols(T, Rm, p);
  __syncthreads();
  const int rows = (j + 2) * p, nr = (j + 1) * p;
  const double2* D1 = bt.bdot + (size_t)g * 2 * bt.bld * p;
  const double2* D2 = D1 + (size_t)bt.bld * p;
  for (int idx = tid; idx < p * rows; idx += nt) {
    const int q = idx / rows, r = idx - q * rows;
    const int c = j * p + q;
    double2 h;
    if (r < nr) {
      const double2 a = D1[(size_t)r * p + q], b = D2[(size_t)r * p + q];
      h = make_double2((double)(float)a.x + (double)(float)b.x, (double)(float)a.y + (double)(float)b.y);
    } else {
      const int l = r - nr;
      h = l <= q ? Rm[l * p + q] : make_double2(0.0, 0.0);
    }
    bt.bH[((size_t)g * bt.bld + c) * bt.hld + r] = h;
  }
}

// V_{j+1}^{(q)} = sum_{l <= q} x_l W[l][q] in df32 (float32 coefficients): pass 0 reads x = S,
// pass 1 reads x = V_{j+1} (in place)
template <int PMAX, int CPT>
__global__ void __launch_bounds__(kBT) k_btransform(Batch bt, int pass) {
  __shared__ float2 W[PMAX * PMAX];
  const int g = blockIdx.y;
  if (!bt.active[g]) return;
  const int j = *bt.jdev, p = bt.bp, N = (int)bt.N, G = bt.ngroups;
  const float2* Wg = bt.bw + ((size_t)g * 2 + pass) * p * p;
  for (int i = threadIdx.x; i < p * p; i += blockDim.x) W[i] = Wg[i];
  __syncthreads();
  const int cell0 = blockIdx.x * kBT * CPT + threadIdx.x;
#pragma unroll
  for (int c = 0; c < CPT; ++c) {
    const int cell = cell0 + c * kBT;
    if (cell >= N) continue;
    cdf x[PMAX];
#pragma unroll
    for (int l = 0; l < PMAX; ++l) {
      x[l] = {{0.f, 0.f}, {0.f, 0.f}};
      if (l < p) {
        const size_t b = (size_t)(l * G + g);
        const size_t off = pass == 0 ? b * bt.N : (b * (bt.maxit + 1) + j + 1) * bt.N;
        x[l] = pass == 0 ? load_cdf(bt.S_hi, bt.S_lo, off + cell) : load_cdf(bt.V_hi, bt.V_lo, off + cell);
      }
    }
#pragma unroll
    for (int q = 0; q < PMAX; ++q) {
      if (q >= p) continue;
      cdf acc = {{0.f, 0.f}, {0.f, 0.f}};
#pragma unroll
      for (int l = 0; l < PMAX; ++l)
        if (l <= q) {
          const float2 w = W[l * p + q];
          acc.re = df_fma2f(acc.re, x[l].re, w.x, x[l].im, -w.y);
          acc.im = df_fma2f(acc.im, x[l].re, w.y, x[l].im, w.x);
        }
      store_cdf(bt.V_hi, bt.V_lo, ((size_t)(q * G + g) * (bt.maxit + 1) + j + 1) * bt.N + cell, acc);
    }
  }
}

// Givens rotation zeroing b against a (a <- rho e^{i arg a}), the convention of the
// per-shift least squares: x_r' = c x_r + s x_r2, x_r2' = -conj(s) x_r + c x_r2, with
// c = |a| / rho, s = (a / |a|) conj(b) / rho, rho^2 = |a|^2 + |b|^2.  Formed from the squared moduli
// with two square roots and one reciprocal (the entries are far from the double range limits that
// hypot guards against); these rotations are computed one after another, so their latency counts.
__device__ __forceinline__ void bgivens(double2 a, double2 b, double& c, double2& s, double2& r) {
  const double na2 = a.x * a.x + a.y * a.y, nb2 = b.x * b.x + b.y * b.y;
  if (nb2 == 0.0) {   // nothing to eliminate (also a = b = 0)
    c = 1.0; s = make_double2(0.0, 0.0); r = a;
  } else if (na2 == 0.0) {
    const double nb = sqrt(nb2);
    c = 0.0; s = make_double2(b.x / nb, -b.y / nb); r = make_double2(nb, 0.0);
  } else {
    const double rho2 = na2 + nb2;
    const double inv = 1.0 / (sqrt(na2) * sqrt(rho2));   // 1 / (|a| rho)
    c = na2 * inv;
    const double2 ab = bz_mul(a, make_double2(b.x, -b.y));
    s = make_double2(ab.x * inv, ab.y * inv);
    const double f = rho2 * inv;                          // rho / |a|
    r = make_double2(a.x * f, a.y * f);
  }
}
__device__ __forceinline__ void brot(double2* x, int r1, int r2, double c, double2 s) {
  const double2 a = x[r1], b = x[r2];
  const double2 sb = bz_mul(s, b), sa = bz_cmul(s, a);
  x[r1] = make_double2(c * a.x + sb.x, c * a.y + sb.y);
  x[r2] = make_double2(c * b.x - sa.x, c * b.y - sa.y);
}
// the same on a row-major [row][p] right-hand-side block, column q
__device__ __forceinline__ void brot_g(double2* G, int p, int q, int r1, int r2, double c, double2 s) {
  const double2 a = G[(size_t)r1 * p + q], b = G[(size_t)r2 * p + q];
  const double2 sb = bz_mul(s, b), sa = bz_cmul(s, a);
  G[(size_t)r1 * p + q] = make_double2(c * a.x + sb.x, c * a.y + sb.y);
  G[(size_t)r2 * p + q] = make_double2(c * b.x - sa.x, c * b.y - sa.y);
}

// group of the member-0 shift bs (member-0 bases are 0..G-1, their shifts contiguous)
__device__ __forceinline__ int bshift_group(const Batch& bt, int bs) {
  int g = 0;
  while (g + 1 < bt.ngroups && bt.shift_off[g + 1] <= bs) ++g;
  return g;
}

// Block least squares of the shifts (one warp carries min(floor(32 / p), kBLsMaxSpw) of them):
// lane (slot, q) owns column q of its shift.  The new block column j of
// Hbar(z; T_j) = [I; 0] + Hbar_j (z - tau_j) gets every earlier rotation, then its own p rotations
// per column in column order, and the same lane applies them to column q of the rotated right-hand
// side E_1 (beta = I).  The rotated matrix R (upper triangular) and right-hand side are kept per
// shift for the back-substitution.  The rotations of an earlier column cc act on rows cc..cc+p only,
// so a lane walks its column down with a window of p+1 rows in registers: row cc leaves the window
// final, row cc+p+1 enters it from H; the earlier rotations of the warp's shifts come through shared
// memory, kBLsChunk columns at a time.
constexpr int kBLsChunk = 32;
// One shift per warp.  Measured on the 256x256 block step (48 launches): packing 2-4 shifts into a
// warp 62 ms against 57; the earlier columns taken four at a time in one unrolled block 49.4 against
// 50.1 ms, and the same with identity rotations padding each column to PMAX (branch-free) 60.7 ms --
// the time follows the FP64 work of the active lanes, not the dependency chains
constexpr int kBLsMaxSpw = 1;
__host__ __device__ __forceinline__ int ls_spw(int p) { return 32 / p > kBLsMaxSpw ? kBLsMaxSpw : 32 / p; }

template <int PMAX>
__global__ void __launch_bounds__(32) k_block_ls(Batch bt) {
  __shared__ double rc_s[kBLsMaxSpw][kBLsChunk * PMAX];
  __shared__ double2 rs_s[kBLsMaxSpw][kBLsChunk * PMAX];
  const int p = bt.bp, G = bt.ngroups, hld = bt.hld;
  const int spw = ls_spw(p);
  const int lane = threadIdx.x;
  const int sl = lane / p, q = lane - sl * p;
  const int bs = blockIdx.x * spw + sl;
  const int j = *bt.jdev, c0 = j * p;
  bool on = sl < spw && bs < bt.nbs;
  int g = 0, i_sh = 0;
  if (on) {
    g = bshift_group(bt, bs);
    on = bt.active[g] != 0;
    i_sh = bs - bt.shift_off[g];
  }
  if (on) {   // all right-hand sides of the shift converged: nothing left to do for it
    int open = 0;
    for (int r = 0; r < p; ++r) open |= bt.conv_it[bt.shift_off[r * G + g] + i_sh] == 0;
    on = open != 0;
  }
  double2 dz = make_double2(0.0, 0.0);
  if (on) {
    const double2 z = bt.zsh[bs], tau = bt.tau_cur[g];
    dz = make_double2(z.x - tau.x, z.y - tau.y);
  }
  double2* R = bt.bR + (size_t)(on ? bs : 0) * bt.bld * hld;
  double* rcs = bt.brc + (size_t)(on ? bs : 0) * bt.bld * p;
  double2* rss = bt.brs + (size_t)(on ? bs : 0) * bt.bld * p;
  double2* Gr = bt.bG + (size_t)(on ? bs : 0) * hld * p;
  const double2* H = bt.bH + (size_t)g * bt.bld * hld;
  const int c = c0 + q;
  double2* Rc = R + (size_t)c * hld;
  const double2* Hc = H + (size_t)c * hld;
  // row r of column c of Hbar(z; T_j); rows below c + p are zero (and never written in H)
  auto hz = [&](int r) {
    double2 v = make_double2(0.0, 0.0);
    if (r <= c + p) {
      v = bz_mul(dz, Hc[r]);
      if (r == c) v.x += 1.0;
    }
    return v;
  };
  double2 win[PMAX + 1];
#pragma unroll
  for (int r = 0; r <= PMAX; ++r) win[r] = (on && r <= p) ? hz(r) : make_double2(0.0, 0.0);
  for (int cb = 0; cb < c0; cb += kBLsChunk) {
    const int ce = min(cb + kBLsChunk, c0), nrot = (ce - cb) * p;
    __syncwarp();
    for (int idx = lane; idx < spw * nrot; idx += 32) {
      const int ss = idx / nrot, r = idx - ss * nrot, bss = blockIdx.x * spw + ss;
      if (bss < bt.nbs) {
        rc_s[ss][r] = bt.brc[(size_t)bss * bt.bld * p + (size_t)cb * p + r];
        rs_s[ss][r] = bt.brs[(size_t)bss * bt.bld * p + (size_t)cb * p + r];
      }
    }
    __syncwarp();
    if (on) {
      for (int cc = cb; cc < ce; ++cc) {
        const double* rcp = rc_s[sl] + (cc - cb) * p;
        const double2* rsp = rs_s[sl] + (cc - cb) * p;
        const double2 nv = hz(cc + p + 1);
#pragma unroll
        for (int k = 0; k < PMAX; ++k)
          if (k < p) {
            const double cs = rcp[k];
            const double2 sn = rsp[k], a = win[0], bq = win[1 + k];
            const double2 sb = bz_mul(sn, bq), sa = bz_cmul(sn, a);
            win[0] = make_double2(cs * a.x + sb.x, cs * a.y + sb.y);
            win[1 + k] = make_double2(cs * bq.x - sa.x, cs * bq.y - sa.y);
          }
        Rc[cc] = win[0];
#pragma unroll
        for (int r = 0; r < PMAX; ++r) win[r] = win[r + 1];
#pragma unroll
        for (int r = 0; r <= PMAX; ++r)
          if (r == p) win[r] = nv;
      }
    }
  }
  if (on) {
#pragma unroll
    for (int r = 0; r <= PMAX; ++r)
      if (r <= p) Rc[c0 + r] = win[r];
    for (int r = c0 + p + 1; r <= c + p; ++r) Rc[r] = hz(r);
    if (j == 0)
      for (int r = 0; r < p; ++r) Gr[(size_t)r * p + q] = make_double2(r == q ? 1.0 : 0.0, 0.0);
    for (int r = (j + 1) * p; r < (j + 2) * p; ++r) Gr[(size_t)r * p + q] = make_double2(0.0, 0.0);
  }
  __syncwarp();
  for (int qq = 0; qq < p; ++qq) {
    const int cn = c0 + qq;
    if (on && q == qq) {
      // the pivot and the p entries below it in registers: the rotations form one dependent chain
      double2 below[PMAX];
#pragma unroll
      for (int k = 0; k < PMAX; ++k) below[k] = k < p ? Rc[cn + 1 + k] : make_double2(0.0, 0.0);
      double2 top = Rc[cn];
#pragma unroll
      for (int k = 0; k < PMAX; ++k)
        if (k < p) {
          double cs;
          double2 sn, r;
          bgivens(top, below[k], cs, sn, r);
          top = r;
          rc_s[sl][k] = cs;
          rs_s[sl][k] = sn;
        }
      Rc[cn] = top;
      for (int k = 0; k < p; ++k) {
        Rc[cn + 1 + k] = make_double2(0.0, 0.0);
        rcs[(size_t)cn * p + k] = rc_s[sl][k];
        rss[(size_t)cn * p + k] = rs_s[sl][k];
      }
    }
    __syncwarp();
    if (on) {
      if (q > qq)
        for (int k = 0; k < p; ++k) brot(Rc, cn, cn + 1 + k, rc_s[sl][k], rs_s[sl][k]);
      for (int k = 0; k < p; ++k) brot_g(Gr, p, q, cn, cn + 1 + k, rc_s[sl][k], rs_s[sl][k]);
    }
    __syncwarp();
  }
  if (on) {
    double r2 = 0.0;
    for (int r = (j + 1) * p; r < (j + 2) * p; ++r) {
      const double2 v = Gr[(size_t)r * p + q];
      r2 += v.x * v.x + v.y * v.y;
    }
    const double res = sqrt(r2);
    const int sh = bt.shift_off[q * G + g] + i_sh;
    if (bt.conv_it[sh] == 0) {
      bt.pres[sh] = res;
      if (res <= 0.5 * bt.tol) {
        bt.conv_it[sh] = j + 1;
      } else {
        atomicOr(&bt.gany[g], 1);
        atomicMax(&bt.grmax[g], (unsigned long long)__double_as_longlong(res));
      }
    }
  }
}

// iteration counters, active flags and the largest open residual of every member basis
__global__ void k_block_flags(Batch bt) {
  const int j = *bt.jdev;
  for (int b = threadIdx.x; b < bt.nb; b += blockDim.x) {
    if (!bt.active[b]) continue;
    const int g = b % bt.ngroups;
    bt.nit[b] = j + 1;
    bt.active[b] = (bt.gany[g] && j + 1 < bt.maxit) ? 1 : 0;
    bt.rmax[b] = __longlong_as_double((long long)bt.grmax[g]);
  }
}

// y = R^{-1} g for every (shift, right-hand side): n = (iterations at convergence, else done) * p
// columns of the shift's rotated block system.  One warp per (shift, right-hand side), column by
// column from the last: y_i = g_i / R_ii, then g_l -= R_li y_i for l < i with the lanes splitting l
// (column i of R is contiguous); g sits in shared memory.  sh is the global shift of member q of
// group g.
__global__ void k_bbacksolve(Batch bt, const int* sh_basis) {
  extern __shared__ double2 gsm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int sh = blockIdx.x * (blockDim.x >> 5) + warp;
  if (sh >= bt.nsh) return;   // whole warps leave; the kernel has no block-wide barrier
  const int b = sh_basis[sh], G = bt.ngroups, p = bt.bp, hld = bt.hld;
  const int g = b % G, q = b / G;
  const int bs = bt.shift_off[g] + (sh - bt.shift_off[b]);
  const int m = bt.conv_it[sh] > 0 ? bt.conv_it[sh] : bt.nit[b];
  const int n = m * p;
  const double2* R = bt.bR + (size_t)bs * bt.bld * hld;
  const double2* Gr = bt.bG + (size_t)bs * hld * p;
  double2* y = bt.bY + (size_t)sh * bt.bld;
  double2* gw = gsm + (size_t)warp * bt.bld;
  for (int i = lane; i < n; i += 32) gw[i] = Gr[(size_t)i * p + q];
  for (int i = n + lane; i < bt.bld; i += 32) y[i] = make_double2(0.0, 0.0);
  __syncwarp();
  for (int i = n - 1; i >= 0; --i) {
    const double2* Rc = R + (size_t)i * hld;
    const double2 d = Rc[i];
    const double2 yi = (d.x != 0.0 || d.y != 0.0) ? bz_div(gw[i], d) : make_double2(0.0, 0.0);
    if (lane == 0) y[i] = yi;
    for (int l = lane; l < i; l += 32) {
      const double2 t = bz_mul(Rc[l], yi);
      gw[l].x -= t.x;
      gw[l].y -= t.y;
    }
    __syncwarp();
  }
}

constexpr int kBXS = 16;    // shifts per pass of the solution kernel
constexpr int kBXC = 128;   // coefficient columns staged per pass

// X[sh] = sum_c U_c y_sh[c] over the block's columns (every member's U), df32.  A chunk of kBXS
// shifts runs over the columns of its latest-converging shift only (the coefficients beyond a
// shift's own convergence are zero).
__global__ void __launch_bounds__(kBT) k_bxk(Batch bt, float2* X_hi, float2* X_lo) {
  __shared__ cdf ys[kBXS][kBXC];
  __shared__ int s_n;
  const int b = blockIdx.y;
  const int g = b % bt.ngroups;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int s0 = bt.shift_off[b], s1 = bt.shift_off[b + 1];
  for (int sa = s0; sa < s1; sa += kBXS) {
    __syncthreads();
    if (threadIdx.x == 0) {
      int m = 0;
      for (int sh = sa; sh < min(sa + kBXS, s1); ++sh) m = max(m, bt.conv_it[sh] > 0 ? bt.conv_it[sh] : bt.nit[b]);
      s_n = m * bt.bp;
    }
    __syncthreads();
    const int n = s_n;
    cdf acc[kBXS];
#pragma unroll
    for (int q = 0; q < kBXS; ++q) acc[q] = {{0.f, 0.f}, {0.f, 0.f}};
    for (int cb = 0; cb < n; cb += kBXC) {
      const int ce = min(cb + kBXC, n);
      __syncthreads();
      for (int idx = threadIdx.x; idx < kBXS * kBXC; idx += blockDim.x) {
        const int q = idx / kBXC, i = idx % kBXC;
        const int sh = sa + q;
        const double2 y = (sh < s1 && cb + i < ce) ? bt.bY[(size_t)sh * bt.bld + cb + i] : make_double2(0.0, 0.0);
        ys[q][i] = {df_from_double(y.x), df_from_double(y.y)};
      }
      __syncthreads();
      if (c < bt.N)
        for (int col = cb; col < ce; ++col) {
          const size_t off = ucol_off(bt, g, col);
          const cdf u = load_cdf(bt.U_hi + off, lo_at(bt.U_lo, off), c);
#pragma unroll
          for (int q = 0; q < kBXS; ++q) acc[q] = cdf_fma(acc[q], u, ys[q][col - cb]);
        }
    }
    if (c < bt.N)
#pragma unroll
      for (int q = 0; q < kBXS; ++q)
        if (sa + q < s1) store_cdf(X_hi, X_lo, (size_t)(sa + q) * bt.N + c, acc[q]);
  }
}

// quadrature coefficients over the block's columns: C[item][c] = sum_k w_k y_{sh0+k}[c]
__global__ void k_bquad_coef(Batch bt, const QuadItem* items, int nitems, const double2* wq, double2* C) {
  const int q = blockIdx.x;
  if (q >= nitems) return;
  const QuadItem it = items[q];
  for (int i = threadIdx.x; i < bt.bld; i += blockDim.x) {
    double2 acc = make_double2(0.0, 0.0);
    for (int k = 0; k < it.nk; ++k) {
      const double2 t = bz_mul(wq[it.sh0 + k], bt.bY[(size_t)(it.sh0 + k) * bt.bld + i]);
      acc.x += t.x; acc.y += t.y;
    }
    C[(size_t)q * bt.bld + i] = acc;
  }
}

__device__ __forceinline__ double bquad_dot(const Batch& bt, const QuadItem& it, const double2* C, int q, int64_t cell) {
  const int g = it.basis % bt.ngroups;
  const int n = bt.nit[it.basis] * bt.bp;
  double acc = 0.0;
  for (int col = 0; col < n; ++col) {
    const size_t ui = ucol_off(bt, g, col) + cell;
    const float2 hi = bt.U_hi[ui], lo = bt.U_lo ? bt.U_lo[ui] : make_float2(0.f, 0.f);
    const double2 cf = C[(size_t)q * bt.bld + col];
    acc += ((double)hi.x + (double)lo.x) * cf.x - ((double)hi.y + (double)lo.y) * cf.y;
  }
  return acc;
}

// h[s][r][t] = 2 Re (U_block[rcell] . C_{s,t})
__global__ void k_bmeasure(Batch bt, const QuadItem* items, const double2* C, int ns, int nr, int nt,
                           const int64_t* rcells, double* h) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= ns * nr * nt) return;
  const int t = idx % nt, r = (idx / nt) % nr, s = idx / (nt * nr);
  const int q = s * nt + t;
  h[idx] = 2.0 * bquad_dot(bt, items[q], C, q, rcells[r]);
}

// phi[q][c] for the items q = s * nt + t
__global__ void k_bfields(Batch bt, const QuadItem* items, const double2* C, double* phi) {
  const int q = blockIdx.y;
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= bt.N) return;
  phi[(size_t)q * bt.N + c] = 2.0 * bquad_dot(bt, items[q], C, q, c);
}

// ------------------------------------------------------------------ host launchers
static int device_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 148;
  }
  return sms;
}

// CTAs per group for the tile-looping kernels: about eight CTAs per SM over all groups (the update
// kernels hold up to three per SM; more CTAs than that keep the SMs full through the tail), every
// CTA with the same number of tiles
static unsigned tile_grid(int64_t N, int cpt, int groups) {
  const int64_t nt = (N + kBT * cpt - 1) / (kBT * cpt);
  const int64_t target = std::max<int64_t>(1, 8 * device_sms() / std::max(groups, 1));
  const int64_t per = (nt + target - 1) / target;
  return (unsigned)((nt + per - 1) / per);
}

// PMAX: register layout for up to PMAX right-hand sides; CPTD, CPTU: cells per thread of the dot
// kernels and of the update kernels
template <int PMAX, int CPTD, int CPTU>
static void block_arnoldi_t(const Batch& bt, const FineExact& fe, cudaStream_t st, Prof* pf) {
  const int G = bt.ngroups;
  const dim3 gd(tile_grid(fe.N, CPTD, G), G), gu(tile_grid(fe.N, CPTU, G), G);
  const dim3 gt((unsigned)((fe.N + kBT * CPTU - 1) / (kBT * CPTU)), G);
  k_bzero<<<G, 256, 0, st>>>(bt);
  prof_begin(pf, KC_DOTS, st);
  k_bdots<PMAX, CPTD><<<gd, kBT, 0, st>>>(bt, fe);
  prof_end(pf, KC_DOTS, st);
  for (int mode = 0; mode < 2; ++mode) {
    prof_begin(pf, KC_ORTHO, st);
    k_bupdate<PMAX, CPTU><<<gu, kBT, 0, st>>>(bt, fe, mode);
    prof_end(pf, KC_ORTHO, st);
  }
  prof_begin(pf, KC_NORMALIZE, st);
  for (int pass = 0; pass < 2; ++pass) {
    k_bgram<PMAX, CPTD><<<gd, kBT, 0, st>>>(bt, pass);
    k_bchol<<<G, 256, 0, st>>>(bt, pass);
    k_btransform<PMAX, CPTU><<<gt, kBT, 0, st>>>(bt, pass);
  }
  prof_end(pf, KC_NORMALIZE, st);
  prof_begin(pf, KC_SHIFT_LS, st);
  k_block_ls<PMAX><<<(bt.nbs + ls_spw(bt.bp) - 1) / ls_spw(bt.bp), 32, 0, st>>>(bt);
  prof_end(pf, KC_SHIFT_LS, st);
}

int launch_block_iteration(const Batch& bt, const FineExact& fe, cudaStream_t st, int* nlaunch, Prof* pf) {
  if (bt.bp <= 4) block_arnoldi_t<4, 4, 4>(bt, fe, st, pf);
  else if (bt.bp <= 8) block_arnoldi_t<8, 4, 2>(bt, fe, st, pf);
  else if (bt.bp <= 12) block_arnoldi_t<12, 2, 1>(bt, fe, st, pf);
  else if (bt.bp <= 16) block_arnoldi_t<16, 2, 1>(bt, fe, st, pf);
  else return 1;
  k_block_flags<<<1, 256, 0, st>>>(bt);
  *nlaunch += 12;
  return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

void launch_block_backsolve(const Batch& bt, const int* sh_basis, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_bbacksolve, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  const size_t per_warp = (size_t)bt.bld * sizeof(double2);
  const int warps = (int)std::max<size_t>(1, std::min<size_t>(8, (size_t)(200 * 1024) / per_warp));
  k_bbacksolve<<<(bt.nsh + warps - 1) / warps, 32 * warps, warps * per_warp, st>>>(bt, sh_basis);
}

void launch_block_xk(const Batch& bt, float2* X_hi, float2* X_lo, cudaStream_t st, Prof* pf) {
  const dim3 g((unsigned)((bt.N + kBT - 1) / kBT), bt.nb);
  prof_begin(pf, KC_XK, st);
  k_bxk<<<g, kBT, 0, st>>>(bt, X_hi, X_lo);
  prof_end(pf, KC_XK, st);
}

void launch_block_quad(const Batch& bt, const QuadItem* items, int nitems, const double2* wq, double2* C,
                       int ns, int nr, int nt, const int64_t* rcells, double* out, int fields, cudaStream_t st) {
  k_bquad_coef<<<nitems, 128, 0, st>>>(bt, items, nitems, wq, C);
  if (fields) {
    const dim3 g((unsigned)((bt.N + 255) / 256), ns * nt);
    k_bfields<<<g, 256, 0, st>>>(bt, items, C, out);
  } else {
    const int n = ns * nr * nt;
    k_bmeasure<<<(n + 127) / 128, 128, 0, st>>>(bt, items, C, ns, nr, nt, rcells, out);
  }
}

}  // namespace lt
