// exact.cuh -- df32 access to the Krylov vectors and the fine-level operator
// K + tau M applied in df32 (the "exact" residual of the preconditioner
// solves, Sec. 3), shared by the batched kernels and the cluster-resident
// inner solve.
#pragma once
#include "df32.cuh"
#include "lt_internal.h"

namespace lt {

// A vector is a hi plane and a lo plane of float2 (df32 complex).  With reduced precision
// (LT_PREC_FP32) the lo planes are not allocated: a null lo plane reads as zero and is not
// written, so the same kernels carry float32 vectors.
__device__ __forceinline__ cdf load_cdf(const float2* hi, const float2* lo, size_t idx) {
  float2 h = hi[idx], l = lo ? lo[idx] : make_float2(0.f, 0.f);
  return {{h.x, l.x}, {h.y, l.y}};
}
__device__ __forceinline__ void store_cdf(float2* hi, float2* lo, size_t idx, cdf v) {
  if (lo) {
    hi[idx] = make_float2(v.re.hi, v.im.hi);
    lo[idx] = make_float2(v.re.lo, v.im.lo);
  } else {
    hi[idx] = make_float2(v.re.hi + v.re.lo, v.im.hi + v.im.lo);
  }
}
__device__ __forceinline__ df ldf(const float* hi, const float* lo, int c) { return {hi[c], lo[c]}; }

// (K + tau M) u at cell c, df32; u given by hi/lo planes of one vector
__device__ __forceinline__ cdf apply_exact(const FineExact& fe, const float2* uhi, const float2* ulo, int c, df taur,
                                           df taui) {
  const int nx = fe.nx, ny = fe.ny, nz = fe.nz;
  int i = c % nx, j = (c / nx) % ny, k = c / (nx * ny);
  df D = ldf(fe.D_hi, fe.D_lo, c), m = ldf(fe.m_hi, fe.m_lo, c);
  cdf dg = {df_add(D, df_mul(taur, m)), df_mul(taui, m)};
  cdf acc = cdf_mul(dg, load_cdf(uhi, ulo, c));
  if (i + 1 < nx) acc = cdf_sub(acc, cdf_mul_r(load_cdf(uhi, ulo, c + 1), ldf(fe.Te_hi, fe.Te_lo, c)));
  if (i > 0) acc = cdf_sub(acc, cdf_mul_r(load_cdf(uhi, ulo, c - 1), ldf(fe.Te_hi, fe.Te_lo, c - 1)));
  if (j + 1 < ny) acc = cdf_sub(acc, cdf_mul_r(load_cdf(uhi, ulo, c + nx), ldf(fe.Tn_hi, fe.Tn_lo, c)));
  if (j > 0) acc = cdf_sub(acc, cdf_mul_r(load_cdf(uhi, ulo, c - nx), ldf(fe.Tn_hi, fe.Tn_lo, c - nx)));
  const int pl = nx * ny;
  if (k + 1 < nz) acc = cdf_sub(acc, cdf_mul_r(load_cdf(uhi, ulo, c + pl), ldf(fe.Tu_hi, fe.Tu_lo, c)));
  if (k > 0) acc = cdf_sub(acc, cdf_mul_r(load_cdf(uhi, ulo, c - pl), ldf(fe.Tu_hi, fe.Tu_lo, c - pl)));
  return acc;
}

}  // namespace lt
