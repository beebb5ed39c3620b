// cn.cu -- Crank-Nicolson time stepping of M phi' + K phi = q_s(t) e_s on the GPU: the time-stepping
// method the paper compares the Laplace-transform approach against (Sec. 1, Sec. 5.3).
//
// One step of size dt:  (M + dt/2 K) phi' = (M - dt/2 K) phi + dt/2 (q(t) + q(t + dt)) e_s, i.e.
//   (K + tau M) phi' = tau M phi - K phi + (q(t) + q(t + dt)) e_s,   tau = 2 / dt;
// a backward-Euler step of size h (the Rannacher start):
//   (K + tau M) phi' = tau M phi + q(t + h) e_s,                      tau = 1 / h.
// Every step solves the real shifted system by iterative refinement: FP64 residuals of the
// fine operator, float32 multigrid V-cycles on them (the preconditioner of the Laplace path with a
// real shift), until ||f - (K + tau M) x|| <= tol ||f|| for every source (batched: one basis slot per
// source).  A step reads its index from a device counter so that one captured graph serves every
// step of an interval.
#include "lt_internal.h"
#include "lt_kernels.h"

namespace lt {

// (K phi)_c of the FP64 fine operator: D_c phi_c - sum over faces T_f phi_o
__device__ __forceinline__ double apply_k64(const CnArgs& a, const double* phi, int64_t c) {
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const int64_t pl = (int64_t)nx * ny;
  const int i = (int)(c % nx), j = (int)((c / nx) % ny), k = (int)(c / pl);
  double v = a.D[c] * phi[c];
  if (i + 1 < nx) v -= a.Te[c] * phi[c + 1];
  if (i > 0) v -= a.Te[c - 1] * phi[c - 1];
  if (j + 1 < ny) v -= a.Tn[c] * phi[c + nx];
  if (j > 0) v -= a.Tn[c - nx] * phi[c - nx];
  if (k + 1 < nz) v -= a.Tu[c] * phi[c + pl];
  if (k > 0) v -= a.Tu[c - pl] * phi[c - pl];
  return v;
}

__device__ __forceinline__ void block_add(double v, double* dst) {
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) atomicAdd(dst, v);
  }
}

// f = tau M phi - theta K phi + w_b e_{cell_b};  x = phi (initial guess); clears the round norms
__global__ void k_cn_rhs(CnArgs a, Batch bt) {
  const int b = blockIdx.y;
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int step = *a.step;
  const double* phi = a.phi + (size_t)b * a.N;
  double v = 0.0;
  if (c < a.N) {
    v = a.tau * a.m[c] * phi[c];
    if (a.theta != 0.0) v -= a.theta * apply_k64(a, phi, c);
    if (c == a.cell[b]) v += a.srcw[(size_t)step * a.nb + b];
    a.f[(size_t)b * a.N + c] = v;
    a.x[(size_t)b * a.N + c] = phi[c];
  }
  block_add(v * v, &a.fnorm2[b]);
  if (blockIdx.x == 0 && threadIdx.x == 0) bt.active[b] = 1;
}

// itol2 = tol^2 ||f||^2 once the norms of f are complete
__global__ void k_cn_tol(CnArgs a, Batch bt) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= a.nb) return;
  bt.itol2[b] = a.tol * a.tol * a.fnorm2[b];
  for (int r = 0; r <= bt.rounds; ++r) bt.rnorm2[b * (bt.rounds + 1) + r] = 0.0;
}

// r = f - (K + tau M) x  ->  float32 right-hand side of the V-cycles (imaginary part 0), u = 0;
// rnorm2[b][round] = ||r||^2.  A basis whose previous round already met its tolerance is left alone.
__global__ void k_cn_residual(CnArgs a, Batch bt, Level L0, int round) {
  const int b = blockIdx.y;
  if (round > 0 && bt.rnorm2[b * (bt.rounds + 1) + round - 1] <= bt.itol2[b]) {
    if (blockIdx.x == 0 && threadIdx.x == 0) bt.rnorm2[b * (bt.rounds + 1) + round] = 0.0;
    return;
  }
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const double* x = a.x + (size_t)b * a.N;
  double r = 0.0;
  if (c < a.N) {
    r = a.f[(size_t)b * a.N + c] - (apply_k64(a, x, c) + a.tau * a.m[c] * x[c]);
    L0.f[(size_t)b * L0.N + c] = make_float2((float)r, 0.f);
    L0.u[(size_t)b * L0.N + c] = make_float2(0.f, 0.f);
  }
  block_add(r * r, &bt.rnorm2[b * (bt.rounds + 1) + round]);
}

// x += the V-cycles' correction (where this round ran)
__global__ void k_cn_correct(CnArgs a, Batch bt, Level L0, int round) {
  const int b = blockIdx.y;
  if (bt.rnorm2[b * (bt.rounds + 1) + round] <= bt.itol2[b]) return;
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= a.N) return;
  a.x[(size_t)b * a.N + c] += (double)L0.u[(size_t)b * L0.N + c].x;
}

// phi = x; record the final residual norm; advance the step counter
__global__ void k_cn_finish(CnArgs a, Batch bt) {
  const int b = blockIdx.y;
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c < a.N) a.phi[(size_t)b * a.N + c] = a.x[(size_t)b * a.N + c];
  if (c == 0) {
    // largest relative residual of the step over the bases (the last round that ran)
    double worst = 0.0;
    for (int r = bt.rounds; r >= 0; --r) {
      const double v = bt.rnorm2[b * (bt.rounds + 1) + r];
      if (v > 0.0) { worst = v; break; }
    }
    const double rel2 = a.fnorm2[b] > 0.0 ? worst / a.fnorm2[b] : 0.0;
    atomicMax(reinterpret_cast<unsigned long long*>(a.maxres2), (unsigned long long)__double_as_longlong(rel2));
    a.fnorm2[b] = 0.0;
  }
  if (b == 0 && c == 0) *a.step += 1;
}

// h[s][r][t] = phi_s[cell_r]
__global__ void k_cn_measure(CnArgs a, const int64_t* rcells, int nr, int nt, int t, double* h) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= a.nb * nr) return;
  const int s = idx / nr, r = idx % nr;
  h[((size_t)s * nr + r) * nt + t] = a.phi[(size_t)s * a.N + rcells[r]];
}

int launch_cn_step(const MGHost& mg, const Batch& bt, const CnArgs& a, int cycles, cudaStream_t st, int* nl) {
  const Level& L0 = mg.h_levels[0];
  dim3 g((unsigned)((a.N + 255) / 256), a.nb);
  k_cn_rhs<<<g, 256, 0, st>>>(a, bt);
  k_cn_tol<<<(a.nb + 127) / 128, 128, 0, st>>>(a, bt);
  *nl += 2;
  for (int r = 0; r < bt.rounds; ++r) {
    k_cn_residual<<<g, 256, 0, st>>>(a, bt, L0, r);
    for (int cy = 0; cy < cycles; ++cy)
      if (launch_vcycle(mg, bt, r, st, nl, nullptr)) return 1;
    k_cn_correct<<<g, 256, 0, st>>>(a, bt, L0, r);
    *nl += 2;
  }
  k_cn_residual<<<g, 256, 0, st>>>(a, bt, L0, bt.rounds);
  k_cn_finish<<<g, 256, 0, st>>>(a, bt);
  *nl += 2;
  return cudaGetLastError() != cudaSuccess;
}

void launch_cn_measure(const CnArgs& a, const int64_t* rcells, int nr, int nt, int t, double* h, cudaStream_t st) {
  const int n = a.nb * nr;
  k_cn_measure<<<(n + 127) / 128, 128, 0, st>>>(a, rcells, nr, nt, t, h);
}

}  // namespace lt
