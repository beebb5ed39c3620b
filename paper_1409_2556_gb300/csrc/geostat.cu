// geostat.cu -- one iteration of the quasi-linear geostatistical inversion (Sec. 5.1, Algorithm 2)
// on a 2D grid: Q J^T by FFT on the circulant embedding of the exponential covariance (the fast
// product Sec. 5.1 names for stationary kernels on regular grids), J Q J^T + R by an FP64 GEMM,
// the saddle-point system by a Cholesky factorisation of J Q J^T + R and the Schur complement of the
// drift, and s_{k+1} = X beta + Q J^T xi.
//
// Images are complex double [P1][P0] (P0, P1 powers of two >= twice the grid); a 2D transform is
// row FFTs, a transpose, row FFTs, so the spectrum and the products live in the transposed layout
// [P0][P1].  The covariance is embedded on the torus of that size, which makes the cropped circular
// convolution of a zero-padded field equal to the product with the dense covariance matrix.
#include <cuda_runtime.h>
#include <stdint.h>

namespace lt {

// ---------------------------------------------------------------- FFT (radix-2 Stockham)
// Every block transforms one row of length P (a power of two, <= 2048) in shared memory:
// log2(P) passes, each reading one buffer and writing the other in sorted order.  sign = -1
// forward, +1 inverse (unscaled).
__global__ void k_fft_rows(double2* data, int P, int sign) {
  extern __shared__ double2 sh[];
  double2* a = sh;
  double2* b = sh + P;
  double2* row = data + (size_t)blockIdx.x * P;
  for (int i = threadIdx.x; i < P; i += blockDim.x) a[i] = row[i];
  __syncthreads();
  const int half = P >> 1;
  for (int Ns = 1; Ns < P; Ns <<= 1) {
    for (int j = threadIdx.x; j < half; j += blockDim.x) {
      const int jm = j & (Ns - 1);
      double s, c;
      sincospi((double)sign * (double)jm / (double)Ns, &s, &c);   // e^{sign i pi jm / Ns}
      const double2 v0 = a[j], u = a[j + half];
      const double2 v1 = make_double2(u.x * c - u.y * s, u.x * s + u.y * c);
      const int idx = (j - jm) * 2 + jm;                           // (j / Ns) * 2 Ns + j mod Ns
      b[idx] = make_double2(v0.x + v1.x, v0.y + v1.y);
      b[idx + Ns] = make_double2(v0.x - v1.x, v0.y - v1.y);
    }
    __syncthreads();
    double2* t = a; a = b; b = t;
  }
  for (int i = threadIdx.x; i < P; i += blockDim.x) row[i] = a[i];
}

// out[b][c][r] = in[b][r][c] for images of R rows x C columns (32 x 32 tiles)
__global__ void k_transpose(const double2* in, double2* out, int R, int C) {
  __shared__ double2 tile[32][33];
  const size_t img = (size_t)blockIdx.z * R * C;
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
    const int r = r0 + dy, c = c0 + threadIdx.x;
    if (r < R && c < C) tile[dy][threadIdx.x] = in[img + (size_t)r * C + c];
  }
  __syncthreads();
  for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
    const int c = c0 + dy, r = r0 + threadIdx.x;
    if (r < R && c < C) out[img + (size_t)c * R + r] = tile[threadIdx.x][dy];
  }
}

// image q of the batch = row (row0 + q) of J (stride ldj between rows), zero-padded to [P1][P0]
__global__ void k_pad_rows(const double* J, size_t ldj, int row0, int nrows, int nx, int ny, int P0, int P1,
                           double2* img) {
  const int q = blockIdx.y;
  const size_t n = (size_t)P0 * P1;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % P0), y = (int)(i / P0);
    double v = 0.0;
    if (q < nrows && x < nx && y < ny) v = J[(size_t)(row0 + q) * ldj + (size_t)y * nx + x];
    img[(size_t)q * n + i] = make_double2(v, 0.0);
  }
}

// pointwise product with the (real) covariance spectrum, times the inverse transform's 1 / (P0 P1)
__global__ void k_spectrum_mul(double2* img, const double* lam, size_t n, double scale) {
  const int q = blockIdx.y;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double f = lam[i] * scale;
    double2 v = img[(size_t)q * n + i];
    img[(size_t)q * n + i] = make_double2(v.x * f, v.y * f);
  }
}

// G[row0 + q][c] = Re img[q][y][x] on the grid cells
__global__ void k_crop_rows(const double2* img, int row0, int nrows, int nx, int ny, int P0, int P1, double* G) {
  const int q = blockIdx.y;
  if (q >= nrows) return;
  const size_t n = (size_t)P0 * P1, N = (size_t)nx * ny;
  for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < N; c += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(c % nx), y = (int)(c / nx);
    G[(size_t)(row0 + q) * N + c] = img[(size_t)q * n + (size_t)y * P0 + x].x;
  }
}

// the real part of a transformed image (the covariance spectrum)
__global__ void k_real_part(const double2* img, double* out, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = img[i].x;
}

// ---------------------------------------------------------------- dense FP64 algebra
// C[i][j] = sum_k A[i][k] B[j][k] (+ R_i on the diagonal): 64 x 64 output tiles, 16 x 16 threads with
// 4 x 4 outputs each, k in steps of 16 through shared memory.
__global__ void __launch_bounds__(256) k_gemm_nt(const double* A, size_t lda, const double* B, size_t ldb, int M,
                                                 int Nn, int K, const double* R, double* C) {
  __shared__ double As[64][17], Bs[64][17];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int i0 = blockIdx.y * 64, j0 = blockIdx.x * 64;
  double acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += 16) {
    for (int e = threadIdx.x; e < 64 * 16; e += 256) {
      const int r = e >> 4, kk = e & 15;
      const int k = k0 + kk;
      As[r][kk] = (i0 + r < M && k < K) ? A[(size_t)(i0 + r) * lda + k] : 0.0;
      Bs[r][kk] = (j0 + r < Nn && k < K) ? B[(size_t)(j0 + r) * ldb + k] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) { a[u] = As[ty * 4 + u][kk]; b[u] = Bs[tx * 4 + u][kk]; }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int i = i0 + ty * 4 + u, j = j0 + tx * 4 + v;
      if (i < M && j < Nn) C[(size_t)i * Nn + j] = acc[u][v] + ((R && i == j) ? R[i] : 0.0);
    }
}

// Cholesky A = L L^T in place (lower triangle, row-major n x n), column k in two launches:
// scale the column below the diagonal by sqrt(A_kk), then update the trailing lower triangle
// (where the diagonal entry itself is replaced by its square root).  flag[0] = 1 if a pivot <= 0.
__global__ void k_chol_col(double* A, int n, int k, int* flag) {
  const double d = A[(size_t)k * n + k];
  if (d <= 0.0) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicExch(flag, 1);
    return;
  }
  const double inv = 1.0 / sqrt(d);
  for (int i = k + 1 + blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    A[(size_t)i * n + k] *= inv;
}

__global__ void k_chol_update(double* A, int n, int k) {
  const int i = k + 1 + blockIdx.y * blockDim.y + threadIdx.y;
  const int j = k + 1 + blockIdx.x * blockDim.x + threadIdx.x;
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0 && threadIdx.y == 0) {
    const double d = A[(size_t)k * n + k];
    if (d > 0.0) A[(size_t)k * n + k] = sqrt(d);
  }
  if (i >= n || j > i) return;
  A[(size_t)i * n + j] -= A[(size_t)i * n + k] * A[(size_t)j * n + k];
}

__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < nw; ++w) t += red[w];
  return t;
}

// L L^T z = rhs for two right-hand sides (columns of `rhs`, [n][2]) in one block: forward then
// backward substitution, each row's dot product spread over the block
__global__ void k_chol_solve2(const double* L, int n, const double* rhs, double* z) {
  __shared__ double red[32];
  for (int col = 0; col < 2; ++col) {
    for (int i = 0; i < n; ++i) {          // L y = rhs
      double p = 0.0;
      for (int j = threadIdx.x; j < i; j += blockDim.x) p += L[(size_t)i * n + j] * z[2 * j + col];
      const double sum = block_sum(p, red);
      if (threadIdx.x == 0) z[2 * i + col] = (rhs[2 * i + col] - sum) / L[(size_t)i * n + i];
      __syncthreads();
    }
    for (int i = n - 1; i >= 0; --i) {     // L^T x = y
      double p = 0.0;
      for (int j = i + 1 + threadIdx.x; j < n; j += blockDim.x) p += L[(size_t)j * n + i] * z[2 * j + col];
      const double sum = block_sum(p, red);
      if (threadIdx.x == 0) z[2 * i + col] = (z[2 * i + col] - sum) / L[(size_t)i * n + i];
      __syncthreads();
    }
  }
}

// per measurement row i of J (stride ldj): rhs[i][0] = y_i - h_i + J_i . s, rhs[i][1] = J_i . X (X = 1)
__global__ void k_gn_rows(const double* J, size_t ldj, int N, const double* s, const double* y, const double* h,
                          double* rhs) {
  __shared__ double red[32];
  const int i = blockIdx.x;
  double a = 0.0, b = 0.0;
  for (int c = threadIdx.x; c < N; c += blockDim.x) {
    const double v = J[(size_t)i * ldj + c];
    a += v * s[c];
    b += v;
  }
  const double js = block_sum(a, red);
  const double jx = block_sum(b, red);
  if (threadIdx.x == 0) {
    rhs[2 * i] = y[i] - h[i] + js;
    rhs[2 * i + 1] = jx;
  }
}

// drift beta = (JX . u) / (JX . w) and xi = u - beta w, from z = [u, w] = A^-1 [b, JX]
__global__ void k_gn_beta(const double* rhs, const double* z, int n, double* beta, double* xi) {
  __shared__ double red[32];
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    a += rhs[2 * i + 1] * z[2 * i];
    b += rhs[2 * i + 1] * z[2 * i + 1];
  }
  const double num = block_sum(a, red), den = block_sum(b, red);
  const double bt = num / den;
  if (threadIdx.x == 0) *beta = bt;
  for (int i = threadIdx.x; i < n; i += blockDim.x) xi[i] = z[2 * i] - bt * z[2 * i + 1];
}

// s_next[c] = beta + sum_j xi_j (Q J^T)[c][j]   (G holds the rows (Q J^T)^T)
__global__ void k_gn_update(const double* G, int ny, int N, const double* xi, const double* beta, double* s_next) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= N) return;
  double v = *beta;
  for (int j = 0; j < ny; ++j) v = fma(xi[j], G[(size_t)j * N + c], v);
  s_next[c] = v;
}

// ---------------------------------------------------------------- launchers
static int fft2_forward(double2* img, double2* tmp, int nimg, int P0, int P1, cudaStream_t st) {
  // rows of length P0, transpose to [P0][P1], rows of length P1: the spectrum in layout [P0][P1]
  const int t0 = P0 / 2 < 1024 ? P0 / 2 : 1024, t1 = P1 / 2 < 1024 ? P1 / 2 : 1024;
  k_fft_rows<<<nimg * P1, t0, 2 * P0 * sizeof(double2), st>>>(img, P0, -1);
  k_transpose<<<dim3((P0 + 31) / 32, (P1 + 31) / 32, nimg), dim3(32, 8), 0, st>>>(img, tmp, P1, P0);
  k_fft_rows<<<nimg * P0, t1, 2 * P1 * sizeof(double2), st>>>(tmp, P1, -1);
  return cudaGetLastError() != cudaSuccess;
}

static int fft2_inverse(double2* tmp, double2* img, int nimg, int P0, int P1, cudaStream_t st) {
  const int t0 = P0 / 2 < 1024 ? P0 / 2 : 1024, t1 = P1 / 2 < 1024 ? P1 / 2 : 1024;
  k_fft_rows<<<nimg * P0, t1, 2 * P1 * sizeof(double2), st>>>(tmp, P1, +1);
  k_transpose<<<dim3((P1 + 31) / 32, (P0 + 31) / 32, nimg), dim3(32, 8), 0, st>>>(tmp, img, P0, P1);
  k_fft_rows<<<nimg * P1, t0, 2 * P0 * sizeof(double2), st>>>(img, P0, +1);
  return cudaGetLastError() != cudaSuccess;
}

int geostat_prepare(int P0, int P1) {
  const int mx = (P0 > P1 ? P0 : P1);
  const size_t smem = 2 * (size_t)mx * sizeof(double2);
  return cudaFuncSetAttribute(k_fft_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess;
}

// covariance spectrum (layout [P0][P1]) from the embedded kernel image c[P1][P0] (device, overwritten)
int geostat_spectrum(double2* cimg, double2* tmp, int P0, int P1, double* lam, cudaStream_t st) {
  if (fft2_forward(cimg, tmp, 1, P0, P1, st)) return 1;
  k_real_part<<<256, 256, 0, st>>>(tmp, lam, (size_t)P0 * P1);
  return cudaGetLastError() != cudaSuccess;
}

// G[row0 .. row0 + nrows) = (Q J^T)^T for rows of J (stride ldj), nrows images at a time
int geostat_qjt(const double* J, size_t ldj, int row0, int nrows, int nx, int ny, int P0, int P1, const double* lam,
                double2* img, double2* tmp, double* G, cudaStream_t st) {
  const size_t n = (size_t)P0 * P1;
  k_pad_rows<<<dim3(64, nrows), 256, 0, st>>>(J, ldj, row0, nrows, nx, ny, P0, P1, img);
  if (fft2_forward(img, tmp, nrows, P0, P1, st)) return 1;
  k_spectrum_mul<<<dim3(64, nrows), 256, 0, st>>>(tmp, lam, n, 1.0 / (double)n);
  if (fft2_inverse(tmp, img, nrows, P0, P1, st)) return 1;
  k_crop_rows<<<dim3(64, nrows), 256, 0, st>>>(img, row0, nrows, nx, ny, P0, P1, G);
  return cudaGetLastError() != cudaSuccess;
}

// A = J G^T + diag(R), then A = L L^T; z = A^-1 [b, JX]; beta, xi; s_next = beta + G^T xi
int geostat_solve(const double* J, size_t ldj, const double* G, int ny, int N, const double* R, const double* s,
                  const double* y, const double* h, double* A, double* rhs, double* z, double* beta, double* xi,
                  double* s_next, int* flag, cudaStream_t st) {
  k_gemm_nt<<<dim3((ny + 63) / 64, (ny + 63) / 64), 256, 0, st>>>(J, ldj, G, (size_t)N, ny, ny, N, R, A);
  k_gn_rows<<<ny, 256, 0, st>>>(J, ldj, N, s, y, h, rhs);
  for (int k = 0; k < ny; ++k) {
    k_chol_col<<<(ny + 255) / 256, 256, 0, st>>>(A, ny, k, flag);
    const int m = ny - k - 1;
    k_chol_update<<<dim3((m + 15) / 16 > 0 ? (m + 15) / 16 : 1, (m + 15) / 16 > 0 ? (m + 15) / 16 : 1), dim3(16, 16),
                    0, st>>>(A, ny, k);
  }
  k_chol_solve2<<<1, 1024, 0, st>>>(A, ny, rhs, z);
  k_gn_beta<<<1, 1024, 0, st>>>(rhs, z, ny, beta, xi);
  k_gn_update<<<(N + 255) / 256, 256, 0, st>>>(G, ny, N, xi, beta, s_next);
  return cudaGetLastError() != cudaSuccess;
}

}  // namespace lt
