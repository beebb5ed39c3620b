// adjoint.cu -- Laplace-domain sensitivity assembly (Sec. 5.2).
//
// For a source s, receiver r and time t (shifts z_k, weights w_k):
//   J[s][r][t][0][c] = -2 Re sum_k w_k (Q_s / z_k) psi_{r,k}^T (dK/dlog kappa_c) x_{s,k}
//   J[s][r][t][1][c] = -2 Re sum_k w_k (Q_s / z_k) z_k m_c psi_{r,k}[c] x_{s,k}[c]
// with x_{s,k} = (K + z_k M)^{-1} e_{cell_s}, psi_{r,k} = (K + z_k M)^{-1} e_{cell_r}
// (K + zM is complex symmetric, so the adjoint uses a transpose), and
//   psi^T dK/dlog kappa_c x = sum_{faces f = (c, o)} W_co (psi_c - psi_o)(x_c - x_o) + Bd_c psi_c x_c,
//   W_co = T_f kappa_o / (kappa_c + kappa_o),  Bd_c = sum of the cell's Dirichlet face transmissibilities.
//
// One CTA per (tile of kTC consecutive cells, time t).  Per shift k it stages
//   A_f[s] = W_f omega_{s,k} (x_c - x_o)   (f = 6 faces),  A_b[s] = Bd_c omega x_c,  A_z[s] = m_c omega z_k x_c
//   B_f[r] = psi_c - psi_o,                                B_0[r] = psi_c
// in shared memory (df32), omega_{s,k} = w_k Q_s / z_k, and every thread
// accumulates Re sum A B in df32 (the quadrature sum cancels strongly, so
// float32 products would not reach 1e-8) for a block of kSB sources x kRB
// receivers of one cell: per face it loads kSB + kRB staged values and forms
// kSB kRB products (the per-cell sum is a small complex matrix product).
// mode 0 writes J; mode 1 accumulates grad[p][c] += sum g[s][r][t] J[s][r][t][p][c].
#include "df32.cuh"
#include "lt_internal.h"
#include "lt_kernels.h"

namespace lt {

constexpr int kTC = 8;       // cells per CTA
constexpr int kSB = 2;       // sources per thread block of pairs
constexpr int kRB = 6;       // receivers per thread block of pairs
constexpr int kSensThreads = 512;

struct SensArgs {
  int ns, nr, nt, Nk;
  int64_t N;
  int nx, ny, nz;
  const int* sh_src;      // [nt][ns] first shift of (s, t)
  const int* sh_rec;      // [nt][nr] first shift of (r, t)
  const double2* omega;   // [nt][ns][Nk] w_k Q_s / z_k
  const double2* zk;      // [nt][Nk]
  const float2 *X_hi, *X_lo;   // [nsh][N] x / psi per shift
  const double *Te, *Tn, *Tu, *kap, *Bd, *m;
  double* J;              // mode 0
  const double* g;        // mode 1 [ns][nr][nt]
  double* grad;           // mode 1 [2][N]
  int mode;
};

__device__ __forceinline__ cdf ldx(const SensArgs& a, int sh, int64_t c) {
  size_t i = (size_t)sh * a.N + c;
  float2 h = a.X_hi[i], l = a.X_lo ? a.X_lo[i] : make_float2(0.f, 0.f);
  return {{h.x, l.x}, {h.y, l.y}};
}
__device__ __forceinline__ cdf cdf_from_d2(double2 v) { return {df_from_double(v.x), df_from_double(v.y)}; }
__device__ __forceinline__ cdf cdf_zero() { return {{0.f, 0.f}, {0.f, 0.f}}; }

// acc += Re(a * b) in df32
__device__ __forceinline__ df re_mul_acc(df acc, const cdf& a, const cdf& b) {
  acc = df_add(acc, df_mul(a.re, b.re));
  return df_sub(acc, df_mul(a.im, b.im));
}

__global__ void __launch_bounds__(kSensThreads) k_sens(SensArgs a) {
  extern __shared__ cdf smem[];
  const int t = blockIdx.y;
  const int64_t c0 = (int64_t)blockIdx.x * kTC;
  const int ns = a.ns, nr = a.nr;
  // layout: A[cell][8][ns] then B[cell][7][nr]
  cdf* A = smem;
  cdf* B = smem + kTC * 8 * ns;
  const int plane = a.nx * a.ny;
  __shared__ double wf[kTC][6];
  __shared__ double bd[kTC], mm[kTC];
  __shared__ int64_t nb[kTC][6];
  if (threadIdx.x < kTC) {
    int q = threadIdx.x;
    int64_t c = c0 + q;
    for (int f = 0; f < 6; ++f) { wf[q][f] = 0.0; nb[q][f] = -1; }
    bd[q] = 0.0;
    mm[q] = 0.0;
    if (c < a.N) {
      int i = (int)(c % a.nx), j = (int)((c / a.nx) % a.ny), k = (int)(c / plane);
      double kc = a.kap[c];
      auto set = [&](int f, int64_t o, double T) {
        if (T != 0.0) { nb[q][f] = o; wf[q][f] = T * a.kap[o] / (kc + a.kap[o]); }
      };
      if (i + 1 < a.nx) set(0, c + 1, a.Te[c]);
      if (i > 0) set(1, c - 1, a.Te[c - 1]);
      if (j + 1 < a.ny) set(2, c + a.nx, a.Tn[c]);
      if (j > 0) set(3, c - a.nx, a.Tn[c - a.nx]);
      if (k + 1 < a.nz) set(4, c + plane, a.Tu[c]);
      if (k > 0) set(5, c - plane, a.Tu[c - plane]);
      bd[q] = a.Bd[c];
      mm[q] = a.m[c];
    }
  }
  __syncthreads();
  const int nsb = (ns + kSB - 1) / kSB, nrb = (nr + kRB - 1) / kRB;
  const int nblk = kTC * nsb * nrb;
  for (int p0 = 0; p0 < nblk; p0 += blockDim.x) {
    const int pb = p0 + threadIdx.x;
    const bool act = pb < nblk;
    const int rb = pb % nrb, sb = (pb / nrb) % nsb, cl = pb / (nrb * nsb);
    df acc0[kSB][kRB], acc1[kSB][kRB];
#pragma unroll
    for (int i = 0; i < kSB; ++i)
#pragma unroll
      for (int q = 0; q < kRB; ++q) { acc0[i][q] = {0.f, 0.f}; acc1[i][q] = {0.f, 0.f}; }
    for (int kk = 0; kk < a.Nk; ++kk) {
      __syncthreads();
      // stage A
      for (int idx = threadIdx.x; idx < kTC * 8 * ns; idx += blockDim.x) {
        int s = idx % ns, f = (idx / ns) % 8, q = idx / (8 * ns);
        int64_t c = c0 + q;
        cdf v = cdf_zero();
        if (c < a.N) {
          int sh = a.sh_src[t * ns + s] + kk;
          cdf om = cdf_from_d2(a.omega[((size_t)t * ns + s) * a.Nk + kk]);
          cdf xc = ldx(a, sh, c);
          if (f < 6) {
            if (nb[q][f] >= 0) {
              cdf d = cdf_sub(xc, ldx(a, sh, nb[q][f]));
              v = cdf_mul_r(cdf_mul(om, d), df_from_double(wf[q][f]));
            }
          } else if (f == 6) {
            v = cdf_mul_r(cdf_mul(om, xc), df_from_double(bd[q]));
          } else {
            cdf oz = cdf_mul(om, cdf_from_d2(a.zk[t * a.Nk + kk]));
            v = cdf_mul_r(cdf_mul(oz, xc), df_from_double(mm[q]));
          }
        }
        A[idx] = v;
      }
      // stage B
      for (int idx = threadIdx.x; idx < kTC * 7 * nr; idx += blockDim.x) {
        int r = idx % nr, f = (idx / nr) % 7, q = idx / (7 * nr);
        int64_t c = c0 + q;
        cdf v = cdf_zero();
        if (c < a.N) {
          int sh = a.sh_rec[t * nr + r] + kk;
          cdf pc = ldx(a, sh, c);
          if (f < 6) {
            if (nb[q][f] >= 0) v = cdf_sub(pc, ldx(a, sh, nb[q][f]));
          } else {
            v = pc;
          }
        }
        B[idx] = v;
      }
      __syncthreads();
      if (act) {
        const cdf* Ap = A + (size_t)cl * 8 * ns;
        const cdf* Bp = B + (size_t)cl * 7 * nr;
        for (int f = 0; f < 7; ++f) {
          cdf av[kSB], bv[kRB];
#pragma unroll
          for (int i = 0; i < kSB; ++i) {
            const int s = sb * kSB + i;
            av[i] = s < ns ? Ap[f * ns + s] : cdf_zero();
          }
#pragma unroll
          for (int q = 0; q < kRB; ++q) {
            const int r = rb * kRB + q;
            bv[q] = r < nr ? Bp[f * nr + r] : cdf_zero();
          }
#pragma unroll
          for (int i = 0; i < kSB; ++i)
#pragma unroll
            for (int q = 0; q < kRB; ++q) acc0[i][q] = re_mul_acc(acc0[i][q], av[i], bv[q]);
          if (f == 6) {   // storage term: A_z with the cell's own adjoint value (B_0 = bv here)
#pragma unroll
            for (int i = 0; i < kSB; ++i) {
              const int s = sb * kSB + i;
              const cdf az = s < ns ? Ap[7 * ns + s] : cdf_zero();
#pragma unroll
              for (int q = 0; q < kRB; ++q) acc1[i][q] = re_mul_acc(acc1[i][q], az, bv[q]);
            }
          }
        }
      }
    }
    // write / reduce
    if (act) {
      const int64_t c = c0 + cl;
      if (c < a.N) {
#pragma unroll
        for (int i = 0; i < kSB; ++i)
#pragma unroll
          for (int q = 0; q < kRB; ++q) {
            const int s = sb * kSB + i, r = rb * kRB + q;
            if (s >= ns || r >= nr) continue;
            double j0 = -2.0 * df_to_double(acc0[i][q]);
            double j1 = -2.0 * df_to_double(acc1[i][q]);
            if (a.mode == 0) {
              size_t row = ((size_t)s * nr + r) * a.nt + t;
              a.J[(row * 2 + 0) * a.N + c] = j0;
              a.J[(row * 2 + 1) * a.N + c] = j1;
            } else {
              double gv = a.g[((size_t)s * nr + r) * a.nt + t];
              atomicAdd(&a.grad[c], gv * j0);
              atomicAdd(&a.grad[a.N + c], gv * j1);
            }
          }
      }
    }
  }
}

size_t sens_smem_bytes(int ns, int nr) { return (size_t)kTC * (8 * ns + 7 * nr) * sizeof(cdf); }

int launch_sens2(const SensLaunch& L, cudaStream_t st) {
  SensArgs a;
  a.ns = L.ns; a.nr = L.nr; a.nt = L.nt; a.Nk = L.Nk; a.N = L.N;
  a.nx = L.nx; a.ny = L.ny; a.nz = L.nz;
  a.sh_src = L.sh_src; a.sh_rec = L.sh_rec; a.omega = L.omega; a.zk = L.zk;
  a.X_hi = L.X_hi; a.X_lo = L.X_lo;
  a.Te = L.Te; a.Tn = L.Tn; a.Tu = L.Tu; a.kap = L.kap; a.Bd = L.Bd; a.m = L.m;
  a.J = L.J; a.g = L.g; a.grad = L.grad; a.mode = L.mode;
  size_t smem = sens_smem_bytes(L.ns, L.nr);
  if (smem > 200 * 1024) return -1;
  cudaFuncSetAttribute(k_sens, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  dim3 g((unsigned)((L.N + kTC - 1) / kTC), L.nt);
  const int nblk = kTC * ((L.ns + kSB - 1) / kSB) * ((L.nr + kRB - 1) / kRB);
  const int threads = nblk >= kSensThreads ? kSensThreads : ((nblk + 31) / 32) * 32;
  k_sens<<<g, threads, smem, st>>>(a);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

}  // namespace lt
