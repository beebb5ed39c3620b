// mg_dev.cuh -- per-cell pieces of the float32 complex multigrid for
// K + tau M on the cell-centred grid (smoother, residual, restriction,
// prolongation), shared by the batched multigrid kernels and the
// cluster-resident inner solve.  u and f may point to global or shared memory.
#pragma once
#include "lt_internal.h"

namespace lt {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cinv(float2 d) {
  float inv = 1.f / (d.x * d.x + d.y * d.y);
  return make_float2(d.x * inv, -d.y * inv);
}
__device__ __forceinline__ float2 cdiv(float2 a, float2 d) {
  float inv = 1.f / (d.x * d.x + d.y * d.y);
  return make_float2((a.x * d.x + a.y * d.y) * inv, (a.y * d.x - a.x * d.y) * inv);
}

// sum_nb T u_nb and the cell's complex diagonal D + tau m
__device__ __forceinline__ float2 nb_sum(const Level& L, const float2* __restrict__ u, int i, int j, int k, int c) {
  float2 s = make_float2(0.f, 0.f);
  if (i + 1 < L.nx) { float t = L.Te[c]; float2 v = u[c + 1]; s.x += t * v.x; s.y += t * v.y; }
  if (i > 0) { float t = L.Te[c - 1]; float2 v = u[c - 1]; s.x += t * v.x; s.y += t * v.y; }
  if (j + 1 < L.ny) { float t = L.Tn[c]; float2 v = u[c + L.nx]; s.x += t * v.x; s.y += t * v.y; }
  if (j > 0) { float t = L.Tn[c - L.nx]; float2 v = u[c - L.nx]; s.x += t * v.x; s.y += t * v.y; }
  const int pl = L.nx * L.ny;
  if (k + 1 < L.nz) { float t = L.Tu[c]; float2 v = u[c + pl]; s.x += t * v.x; s.y += t * v.y; }
  if (k > 0) { float t = L.Tu[c - pl]; float2 v = u[c - pl]; s.x += t * v.x; s.y += t * v.y; }
  return s;
}

__device__ __forceinline__ float2 diag_of(const Level& L, int c, float2 tau) {
  float m = L.m[c];
  return make_float2(L.D[c] + tau.x * m, tau.y * m);
}

__device__ __forceinline__ void rbgs_cell(const Level& L, float2* u, const float2* f, int c, float2 tau) {
  int i = c % L.nx, j = (c / L.nx) % L.ny, k = c / (L.nx * L.ny);
  float2 s = nb_sum(L, u, i, j, k, c);
  float2 r = f[c];
  r.x += s.x; r.y += s.y;
  u[c] = cdiv(r, diag_of(L, c, tau));
}

__device__ __forceinline__ float2 resid_cell(const Level& L, const float2* u, const float2* f, int c, float2 tau) {
  int i = c % L.nx, j = (c / L.nx) % L.ny, k = c / (L.nx * L.ny);
  float2 s = nb_sum(L, u, i, j, k, c);
  float2 a = cmul(diag_of(L, c, tau), u[c]);
  float2 fc = f[c];
  return make_float2(fc.x - a.x + s.x, fc.y - a.y + s.y);
}

__device__ __forceinline__ void restrict_cell(const Level& Lf, const Level& Lc, const float2* uf, const float2* ff,
                                              float2* fc, float2* uc, int C, float2 tau) {
  int I = C % Lc.nx, J = (C / Lc.nx) % Lc.ny, K = C / (Lc.nx * Lc.ny);
  float2 acc = make_float2(0.f, 0.f);
  for (int dk = 0; dk < Lf.rz; ++dk)
    for (int dj = 0; dj < Lf.ry; ++dj)
      for (int di = 0; di < Lf.rx; ++di) {
        int c = ((K * Lf.rz + dk) * Lf.ny + (J * Lf.ry + dj)) * Lf.nx + (I * Lf.rx + di);
        float2 r = resid_cell(Lf, uf, ff, c, tau);
        acc.x += r.x; acc.y += r.y;
      }
  fc[C] = acc;
  uc[C] = make_float2(0.f, 0.f);
}

// multilinear interpolation weight setup along one axis
__device__ __forceinline__ void axis_interp(int i, int r, int nC, int lo_dir, int hi_dir, int& I0, int& I1,
                                            float& w0, float& w1, float& s1) {
  I0 = i / r;
  if (r == 1) { I1 = I0; w0 = 1.f; w1 = 0.f; s1 = 1.f; return; }
  int o = i - I0 * r;              // 0 or 1
  int nbI = o ? I0 + 1 : I0 - 1;
  w0 = 0.75f; w1 = 0.25f; s1 = 1.f;
  if (nbI < 0) { nbI = I0; s1 = lo_dir ? -1.f : 1.f; }
  else if (nbI >= nC) { nbI = I0; s1 = hi_dir ? -1.f : 1.f; }
  I1 = nbI;
}

__device__ __forceinline__ void prolong_cell(const Level& Lf, const Level& Lc, float2* uf, const float2* uc, int c,
                                             int dmask) {
  int i = c % Lf.nx, j = (c / Lf.nx) % Lf.ny, k = c / (Lf.nx * Lf.ny);
  int I[2], J[2], K[2];
  float wi[2], wj[2], wk[2], si, sj, sk;
  axis_interp(i, Lf.rx, Lc.nx, dmask & 1, dmask & 2, I[0], I[1], wi[0], wi[1], si);
  axis_interp(j, Lf.ry, Lc.ny, dmask & 4, dmask & 8, J[0], J[1], wj[0], wj[1], sj);
  axis_interp(k, Lf.rz, Lc.nz, dmask & 16, dmask & 32, K[0], K[1], wk[0], wk[1], sk);
  wi[1] *= si; wj[1] *= sj; wk[1] *= sk;
  float2 e = make_float2(0.f, 0.f);
  for (int a = 0; a < 2; ++a) {
    if (wk[a] == 0.f) continue;
    for (int bb = 0; bb < 2; ++bb) {
      if (wj[bb] == 0.f) continue;
      for (int cc = 0; cc < 2; ++cc) {
        if (wi[cc] == 0.f) continue;
        float w = wk[a] * wj[bb] * wi[cc];
        float2 v = uc[(K[a] * Lc.ny + J[bb]) * Lc.nx + I[cc]];
        e.x += w * v.x; e.y += w * v.y;
      }
    }
  }
  float2 u = uf[c];
  uf[c] = make_float2(u.x + e.x, u.y + e.y);
}

}  // namespace lt
