// lt_api.cu -- host side of the C ABI declared in include/lt.h.
//
// Builds the finite-volume operator and multigrid hierarchy, the Talbot
// contour tables (Sec. 2.2) and preconditioner-shift schedules (Sec. 3),
// and drives the batched flexible shifted-Krylov solve (Algorithm 1) on the
// context's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/lt.h"
#include "df32.cuh"
#include "lt_internal.h"
#include "lt_kernels.h"

using cplx = std::complex<double>;

// ------------------------------------------------------------------ contour (Sec. 2.2)
// z(theta) = (Nz/t) (sigma + mu theta cot(alpha theta) + i nu theta), the
// modified Talbot contour with the parameters of Trefethen, Weideman and
// Schmelzer (BIT 2006); midpoint nodes theta_k = (2k - 1) pi / Nz in (0, pi);
// weights w_k = -(i / Nz) e^{z_k t} z'(theta_k) for phi = 2 Re sum_k w_k F(z_k).
static const double kSigma = -0.6122, kMu = 0.5017, kAlpha = 0.6407, kNu = 0.2645;

static void talbot_half(double t, int Nz, std::vector<cplx>& z, std::vector<cplx>& w) {
  z.resize(Nz / 2);
  w.resize(Nz / 2);
  for (int k = 0; k < Nz / 2; ++k) {
    double th = (2.0 * (k + 1) - 1.0) * M_PI / Nz;
    double a = kAlpha * th;
    double cot = std::cos(a) / std::sin(a);
    double s = std::sin(a);
    cplx zz = (Nz / t) * cplx(kSigma + kMu * th * cot, kNu * th);
    cplx dz = (Nz / t) * cplx(kMu * (cot - a / (s * s)), kNu);
    z[k] = zz;
    w[k] = cplx(0.0, -1.0 / Nz) * std::exp(zz * t) * dz;
  }
}

// ------------------------------------------------------------------ context
struct HostLevel {
  int nx, ny, nz, N, rx, ry, rz;
  std::vector<double> Te, Tn, Tu, D, m;
};

struct Workspace {
  int nb = 0, maxit = 0, nsh = 0, rounds = 0, ngroups = 0, nc2 = 0, prec = -1;
  int64_t N = 0;
  std::vector<void*> allocs;
  lt::Batch bt{};
  float2* X_hi = nullptr;
  float2* X_lo = nullptr;
  size_t x_elems = 0;
  float4* l0q = nullptr;          // [nb][N] finest-level scratch of the cluster-resident solve
  float2* l0u = nullptr;          // [nb][N] finest-level iterates of the cluster-resident solve (mg_cluster = 3)
  // block flexible GMRES arrays (Batch::bdot .. grmax), sized for (p, groups, maxit, block shifts, shifts)
  std::vector<void*> block_allocs;
  int bk_p = 0, bk_G = 0, bk_M = 0, bk_nbs = 0, bk_nsh = 0;
  // small per-call buffers of the forward path, kept between calls (slot = kScr*)
  void* scr[8] = {};
  size_t scr_bytes[8] = {};
};
enum { kScrShb = 0, kScrRes2, kScrItems, kScrWq, kScrC, kScrRc, kScrOut };

struct lt_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  lt_opts opts{};
  // grid
  bool have_grid = false;
  int nx = 0, ny = 0, nz = 0;
  int64_t N = 0;
  double dx = 0, dy = 0, dz = 0;
  int bc[6] = {0, 0, 0, 0, 1, 1};
  std::vector<double> kappa, Ss;
  std::vector<HostLevel> hl;
  lt::MGHost mg{};
  lt::InnerPlan inner{};          // cluster-resident preconditioner solve on this grid (inner.ok = 0: not possible)
  // other shapes of the same solve, by lt_opts.mg_cluster: [2] 16-CTA clusters of 256 threads with half-height
  // strips; [3] 8-CTA clusters of 256 threads and [4] 4-CTA clusters of 512 threads, both with the finest
  // level's iterate in global memory ([1] is `inner`)
  lt::InnerPlan inner_alt[5]{};
  std::vector<void*> grid_allocs;
  lt::FineExact fe{};
  // float64 fine-level geometry for the sensitivity assembly
  double *g_Te = nullptr, *g_Tn = nullptr, *g_Tu = nullptr, *g_kap = nullptr, *g_Bd = nullptr, *g_m = nullptr;
  // wells
  std::vector<int64_t> src, rec;
  std::vector<double> Q;
  // per source: rate q_s(t) = sum_j rate_a[s][j] exp(-rate_l[s][j] t) (empty: the constant Q[s])
  std::vector<std::vector<double>> rate_a, rate_l;
  // initial head phi_0 (empty: zero)
  std::vector<double> phi0;
  Workspace ws;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  lt::Prof prof;
  std::vector<cudaEvent_t> prof_events;
  // set only for the duration of an lt_forward_noalloc call: device buffers are
  // carved from this region instead of being allocated
  char* arena_base = nullptr;
  size_t arena_cap = 0, arena_off = 0;
  // non-blocking stream on which the per-iteration CUDA graph is captured and replayed
  cudaStream_t cap_stream = nullptr;
  cudaStream_t part_stream[7] = {};     // the streams of parts 1-7 when the bases run decoupled
  cudaEvent_t ev_tail = nullptr;        // end-of-solve buffers ready (decoupled parts queue their own tails)
  cudaEvent_t ev_a = nullptr, ev_b = nullptr;
  // second branch of an outer iteration whose bases are split in two (cluster-resident solves)
  cudaStream_t side_stream = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // learned initial guess (opts.precond = 1)
  lt_unet* net = nullptr;
  float *d_lk = nullptr, *d_mD = nullptr, *d_xin = nullptr, *d_gn2 = nullptr, *d_D32 = nullptr;
  // the last solve's bases (lt_krylov_vectors): group, outer iterations, shifts per group, tau pattern
  std::vector<int> last_group, last_nit;
  std::vector<cplx> last_tau;
  int last_single = 0;
  size_t xin_cap = 0;
  // workspace of lt_precond_apply
  std::vector<void*> pc_allocs;
  int pc_nb = 0;
  lt::Batch pc_bt{};
  lt::MGHost pc_mg{};
};

static int fail(lt_ctx* ctx, int code, const char* fmt, ...) {
  if (ctx) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    ctx->err = buf;
  }
  return code;
}

#define CK(call)                                                                         \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) {                                                             \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? LT_ERR_OOM : LT_ERR_CUDA,       \
                  "%s failed: %s", #call, cudaGetErrorString(e_));                       \
    }                                                                                    \
  } while (0)

static size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

// the cluster-resident solve selected by lt_opts.mg_cluster (its ok flag says whether the grid allows it;
// mg_cluster = 0 selects none)
static const lt::InnerPlan& cluster_plan(const lt_ctx* ctx) {
  static const lt::InnerPlan none{};
  const int m = ctx->opts.mg_cluster;
  return m == 1 ? ctx->inner : (m >= 2 && m <= 4) ? ctx->inner_alt[m] : none;
}
static bool any_cluster_plan(const lt_ctx* ctx) {
  for (const lt::InnerPlan& q : ctx->inner_alt)
    if (q.ok) return true;
  return false;
}

template <typename T>
static int dalloc(lt_ctx* ctx, std::vector<void*>& list, T** p, size_t n) {
  if (ctx->arena_base) {
    size_t bytes = round256(std::max<size_t>(n, 1) * sizeof(T));
    if (ctx->arena_off + bytes > ctx->arena_cap)
      return fail(ctx, LT_ERR_INVALID_ARG, "problem needs more than the %zu-byte static scratch of lt_forward_noalloc",
                  ctx->arena_cap);
    *p = (T*)(ctx->arena_base + ctx->arena_off);
    ctx->arena_off += bytes;
    return LT_OK;
  }
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(T));
  if (e != cudaSuccess)
    return fail(ctx, e == cudaErrorMemoryAllocation ? LT_ERR_OOM : LT_ERR_CUDA, "cudaMalloc of %zu bytes: %s",
                n * sizeof(T), cudaGetErrorString(e));
  list.push_back(q);
  *p = (T*)q;
  return LT_OK;
}

// A per-call device buffer of the forward path, kept in the workspace between calls (grown when a
// call needs more; cudaMalloc / cudaFree synchronise the device, which the steady state avoids).  In
// lt_forward_noalloc it is carved from the static region like every other buffer.
template <typename T>
static int scratch(lt_ctx* ctx, int slot, T** p, size_t n) {
  if (ctx->arena_base) {
    std::vector<void*> none;
    return dalloc(ctx, none, p, n);
  }
  Workspace& ws = ctx->ws;
  const size_t bytes = std::max<size_t>(n, 1) * sizeof(T);
  if (ws.scr_bytes[slot] < bytes) {
    if (ws.scr[slot]) cudaFree(ws.scr[slot]);
    ws.scr[slot] = nullptr;
    ws.scr_bytes[slot] = 0;
    const cudaError_t e = cudaMalloc(&ws.scr[slot], bytes);
    if (e != cudaSuccess)
      return fail(ctx, e == cudaErrorMemoryAllocation ? LT_ERR_OOM : LT_ERR_CUDA, "cudaMalloc of %zu bytes: %s", bytes,
                  cudaGetErrorString(e));
    ws.scr_bytes[slot] = bytes;
  }
  *p = reinterpret_cast<T*>(ws.scr[slot]);
  return LT_OK;
}

static void free_list(std::vector<void*>& list) {
  for (void* p : list) cudaFree(p);
  list.clear();
}

extern "C" {

int lt_default_options(lt_opts* o) {
  if (!o) return LT_ERR_INVALID_ARG;
  o->Nz = 16;
  o->tol = 1e-8;
  o->maxit = 160;
  o->tau_policy = LT_TAU_FLEXIBLE;
  o->tau_project = 1;
  o->groups = 1;
  o->mg_pre = 2;
  o->mg_post = 2;
  o->inner_cycles = 6;
  o->inner_rounds = 6;
  o->inner_tol = 0.0;
  o->true_residual = 1;
  o->check_every = 4;
  o->timing_class = -1;
  o->inner_relax = 0.0;
  o->graphs = 1;
  o->mg_tile = 2;
  o->precond = 0;
  o->mg_tma = 1;
  o->mg_cluster = 1;
  o->precision = LT_PREC_FP64;
  o->krylov = LT_KRYLOV_GMRES;
  o->stop_rule = LT_STOP_SHIFT;
  o->tma_wait_polls = 1 << 26;
  o->gram_schmidt = 2;
  o->block = 0;
  return LT_OK;
}

const char* lt_strerror(int s) {
  switch (s) {
    case LT_OK: return "ok";
    case LT_ERR_INVALID_ARG: return "invalid argument";
    case LT_ERR_OOM: return "device out of memory";
    case LT_ERR_CUDA: return "CUDA runtime error";
    case LT_ERR_NOT_CONVERGED: return "not all shifted systems reached the tolerance";
    case LT_ERR_TIMEOUT: return "device wait timed out";
    case LT_ERR_STATE: return "call order violated";
    default: return "unknown status";
  }
}

const char* lt_last_error(lt_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int lt_create(lt_ctx** out, int device) {
  if (!out) return LT_ERR_INVALID_ARG;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) return LT_ERR_CUDA;
  if (device < 0 || device >= n) return LT_ERR_INVALID_ARG;
  lt_ctx* ctx = new lt_ctx();
  ctx->device = device;
  lt_default_options(&ctx->opts);
  if (cudaSetDevice(device) != cudaSuccess || cudaEventCreate(&ctx->ev0) != cudaSuccess ||
      cudaEventCreate(&ctx->ev1) != cudaSuccess) {
    delete ctx;
    return LT_ERR_CUDA;
  }
  *out = ctx;
  return LT_OK;
}

int lt_set_stream(lt_ctx* ctx, void* stream) {
  if (!ctx) return LT_ERR_INVALID_ARG;
  ctx->stream = (cudaStream_t)stream;
  return LT_OK;
}

static void free_ws(lt_ctx* ctx) {
  free_list(ctx->ws.allocs);
  free_list(ctx->ws.block_allocs);
  for (void*& q : ctx->ws.scr)
    if (q) cudaFree(q);
  ctx->ws = Workspace();
}

void lt_destroy(lt_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  free_ws(ctx);
  free_list(ctx->grid_allocs);
  if (ctx->mg.d_levels) cudaFree(ctx->mg.d_levels);
  if (ctx->ev0) cudaEventDestroy(ctx->ev0);
  if (ctx->ev1) cudaEventDestroy(ctx->ev1);
  for (cudaEvent_t e : ctx->prof_events) cudaEventDestroy(e);
  if (ctx->ev_a) cudaEventDestroy(ctx->ev_a);
  if (ctx->ev_b) cudaEventDestroy(ctx->ev_b);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  if (ctx->ev_tail) cudaEventDestroy(ctx->ev_tail);
  for (cudaStream_t& q : ctx->part_stream)
    if (q) cudaStreamDestroy(q);
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
  if (ctx->side_stream) cudaStreamDestroy(ctx->side_stream);
  lt::tma_cache_free(ctx->mg);
  lt::tma_cache_free(ctx->pc_mg);
  free_list(ctx->pc_allocs);          // also holds pc_mg.d_levels
  ctx->pc_mg.d_levels = nullptr;
  for (float* p : {ctx->d_lk, ctx->d_mD, ctx->d_xin, ctx->d_gn2, ctx->d_D32})
    if (p) cudaFree(p);
  cudaGetLastError();                  // leave no error state behind for other users of the runtime
  delete ctx;
}

int lt_set_options(lt_ctx* ctx, const lt_opts* o) {
  if (!ctx || !o) return LT_ERR_INVALID_ARG;
  if (o->Nz < 4 || o->Nz > 128 || (o->Nz & 1)) return fail(ctx, LT_ERR_INVALID_ARG, "Nz=%d must be even in [4,128]", o->Nz);
  if (!(o->tol > 0.0 && o->tol < 1.0)) return fail(ctx, LT_ERR_INVALID_ARG, "tol=%g must be in (0,1)", o->tol);
  if (o->maxit < 1 || o->maxit > 250) return fail(ctx, LT_ERR_INVALID_ARG, "maxit=%d must be in [1,250]", o->maxit);
  if (o->tau_policy != LT_TAU_SINGLE && o->tau_policy != LT_TAU_FLEXIBLE)
    return fail(ctx, LT_ERR_INVALID_ARG, "tau_policy=%d", o->tau_policy);
  if (o->groups < 1 || o->groups > 64) return fail(ctx, LT_ERR_INVALID_ARG, "groups=%d must be in [1,64]", o->groups);
  if (o->mg_pre < 0 || o->mg_pre > 8 || o->mg_post < 0 || o->mg_post > 8 || o->mg_pre + o->mg_post == 0)
    return fail(ctx, LT_ERR_INVALID_ARG, "mg_pre/mg_post must be in [0,8], not both 0");
  if (o->inner_cycles < 1 || o->inner_cycles > 64 || o->inner_rounds < 1 || o->inner_rounds > 16)
    return fail(ctx, LT_ERR_INVALID_ARG, "inner_cycles in [1,64], inner_rounds in [1,16]");
  if (o->inner_tol < 0.0 || o->inner_tol >= 1.0) return fail(ctx, LT_ERR_INVALID_ARG, "inner_tol=%g", o->inner_tol);
  if (o->check_every < 1) return fail(ctx, LT_ERR_INVALID_ARG, "check_every=%d", o->check_every);
  if (o->mg_tile < 0 || o->mg_tile > 2) return fail(ctx, LT_ERR_INVALID_ARG, "mg_tile=%d must be 0, 1 or 2", o->mg_tile);
  if (o->precond != 0 && o->precond != 1) return fail(ctx, LT_ERR_INVALID_ARG, "precond=%d must be 0 or 1", o->precond);
  if (o->mg_tma != 0 && o->mg_tma != 1) return fail(ctx, LT_ERR_INVALID_ARG, "mg_tma=%d must be 0 or 1", o->mg_tma);
  if (o->graphs != 0 && o->graphs != 1) return fail(ctx, LT_ERR_INVALID_ARG, "graphs=%d must be 0 or 1", o->graphs);
  if (o->mg_cluster < 0 || o->mg_cluster > 4)
    return fail(ctx, LT_ERR_INVALID_ARG, "mg_cluster=%d must be 0 .. 4", o->mg_cluster);
  if (!(o->inner_relax >= 0.0 && o->inner_relax < 1.0))
    return fail(ctx, LT_ERR_INVALID_ARG, "inner_relax=%g must be in [0,1)", o->inner_relax);
  if (o->timing_class < -1 || o->timing_class >= LT_KC_COUNT)
    return fail(ctx, LT_ERR_INVALID_ARG, "timing_class=%d", o->timing_class);
  if (o->precision != LT_PREC_FP64 && o->precision != LT_PREC_FP32)
    return fail(ctx, LT_ERR_INVALID_ARG, "precision=%d must be LT_PREC_FP64 or LT_PREC_FP32", o->precision);
  if (o->precision == LT_PREC_FP32 && o->tol < 2e-6)
    return fail(ctx, LT_ERR_INVALID_ARG, "tol=%g is below the float32 floor (2e-6) of LT_PREC_FP32", o->tol);
  if (o->krylov != LT_KRYLOV_GMRES && o->krylov != LT_KRYLOV_FOM)
    return fail(ctx, LT_ERR_INVALID_ARG, "krylov=%d must be LT_KRYLOV_GMRES or LT_KRYLOV_FOM", o->krylov);
  if (o->stop_rule != LT_STOP_SHIFT && o->stop_rule != LT_STOP_QUADRATURE)
    return fail(ctx, LT_ERR_INVALID_ARG, "stop_rule=%d must be LT_STOP_SHIFT or LT_STOP_QUADRATURE", o->stop_rule);
  if (o->tma_wait_polls < 0) return fail(ctx, LT_ERR_INVALID_ARG, "tma_wait_polls=%d must be >= 0", o->tma_wait_polls);
  if (o->gram_schmidt != 1 && o->gram_schmidt != 2)
    return fail(ctx, LT_ERR_INVALID_ARG, "gram_schmidt=%d must be 1 or 2", o->gram_schmidt);
  if (o->block != 0 && o->block != 1) return fail(ctx, LT_ERR_INVALID_ARG, "block=%d must be 0 or 1", o->block);
  if (o->block && (o->krylov != LT_KRYLOV_GMRES || o->stop_rule != LT_STOP_SHIFT || o->precision != LT_PREC_FP64))
    return fail(ctx, LT_ERR_INVALID_ARG, "block = 1 needs LT_KRYLOV_GMRES, LT_STOP_SHIFT and LT_PREC_FP64");
  ctx->opts = *o;
  ctx->mg.npre = o->mg_pre;
  ctx->mg.npost = o->mg_post;
  ctx->mg.tile = o->mg_tile;
  ctx->mg.tma = o->mg_tma;
  ctx->pc_mg.tma = o->mg_tma;
  return LT_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ grid + multigrid hierarchy
// Coarse level by series-parallel upscaling of the transmissibilities: along
// the face normal (ratio r = 2) every fine row of cells is a series path
// centre -> face -> centre crossing half the coarse cell's internal face, the
// crossing face and half the neighbour's internal face; the parallel rows of
// the coarse face add.  With r = 1 the coarse face is the parallel sum of the
// fine faces.  m_coarse = sum of the children.  (For a uniform kappa this
// reproduces the transmissibility of the coarse grid; for strongly varying
// kappa it keeps the series resistance inside coarse cells, which the
// multigrid coarse correction needs.)  The Dirichlet part is coarsened by
// coarsen_bfaces and the diagonal rebuilt by level_diag.
static HostLevel coarsen(const HostLevel& f) {
  HostLevel c;
  c.nx = f.nx / f.rx; c.ny = f.ny / f.ry; c.nz = f.nz / f.rz;
  c.N = c.nx * c.ny * c.nz;
  c.rx = c.ry = c.rz = 1;
  c.Te.assign(c.N, 0.0); c.Tn.assign(c.N, 0.0); c.Tu.assign(c.N, 0.0); c.D.assign(c.N, 0.0); c.m.assign(c.N, 0.0);
  auto fi = [&](int i, int j, int k) { return ((size_t)k * f.ny + j) * f.nx + i; };
  for (int K = 0; K < c.nz; ++K)
    for (int J = 0; J < c.ny; ++J)
      for (int I = 0; I < c.nx; ++I) {
        size_t C = ((size_t)K * c.ny + J) * c.nx + I;
        double mm = 0, te = 0, tn = 0, tu = 0;
        for (int dk = 0; dk < f.rz; ++dk)
          for (int dj = 0; dj < f.ry; ++dj)
            for (int di = 0; di < f.rx; ++di) mm += f.m[fi(I * f.rx + di, J * f.ry + dj, K * f.rz + dk)];
        // x faces: paths over (dj, dk)
        if (I + 1 < c.nx)
          for (int dk = 0; dk < f.rz; ++dk)
            for (int dj = 0; dj < f.ry; ++dj) {
              int j = J * f.ry + dj, k = K * f.rz + dk;
              if (f.rx == 1) { te += f.Te[fi(I, j, k)]; continue; }
              double a = f.Te[fi(2 * I, j, k)], x = f.Te[fi(2 * I + 1, j, k)], b = f.Te[fi(2 * I + 2, j, k)];
              te += 1.0 / (0.5 / a + 1.0 / x + 0.5 / b);
            }
        if (J + 1 < c.ny)
          for (int dk = 0; dk < f.rz; ++dk)
            for (int di = 0; di < f.rx; ++di) {
              int i = I * f.rx + di, k = K * f.rz + dk;
              if (f.ry == 1) { tn += f.Tn[fi(i, J, k)]; continue; }
              double a = f.Tn[fi(i, 2 * J, k)], x = f.Tn[fi(i, 2 * J + 1, k)], b = f.Tn[fi(i, 2 * J + 2, k)];
              tn += 1.0 / (0.5 / a + 1.0 / x + 0.5 / b);
            }
        if (K + 1 < c.nz)
          for (int dj = 0; dj < f.ry; ++dj)
            for (int di = 0; di < f.rx; ++di) {
              int i = I * f.rx + di, j = J * f.ry + dj;
              if (f.rz == 1) { tu += f.Tu[fi(i, j, K)]; continue; }
              double a = f.Tu[fi(i, j, 2 * K)], x = f.Tu[fi(i, j, 2 * K + 1)], b = f.Tu[fi(i, j, 2 * K + 2)];
              tu += 1.0 / (0.5 / a + 1.0 / x + 0.5 / b);
            }
        c.Te[C] = te; c.Tn[C] = tn; c.Tu[C] = tu; c.m[C] = mm;
      }
  return c;
}

// per-face Dirichlet transmissibility arrays on each level (built alongside the levels)
struct BFaces {
  std::vector<double> b[6];   // per cell: transmissibility of the face on side d (0 if none/Neumann)
};

static void level_diag(HostLevel& L, const BFaces& bf) {
  for (int k = 0; k < L.nz; ++k)
    for (int j = 0; j < L.ny; ++j)
      for (int i = 0; i < L.nx; ++i) {
        size_t q = ((size_t)k * L.ny + j) * L.nx + i;
        double s = L.Te[q] + L.Tn[q] + L.Tu[q];
        if (i > 0) s += L.Te[q - 1];
        if (j > 0) s += L.Tn[q - L.nx];
        if (k > 0) s += L.Tu[q - (size_t)L.nx * L.ny];
        for (int d = 0; d < 6; ++d) s += bf.b[d][q];
        L.D[q] = s;
      }
}

// Dirichlet boundary faces of the coarse level: per parallel fine row, the
// fine boundary transmissibility in series with half the internal face of the
// coarse cell along the normal (ratio 2), or the fine face itself (ratio 1).
static BFaces coarsen_bfaces(const HostLevel& f, const HostLevel& c, const BFaces& bf) {
  BFaces out;
  for (int d = 0; d < 6; ++d) out.b[d].assign(c.N, 0.0);
  auto fi = [&](int i, int j, int k) { return ((size_t)k * f.ny + j) * f.nx + i; };
  const int r[3] = {f.rx, f.ry, f.rz};
  for (int k = 0; k < f.nz; ++k)
    for (int j = 0; j < f.ny; ++j)
      for (int i = 0; i < f.nx; ++i) {
        size_t q = fi(i, j, k);
        size_t C = ((size_t)(k / f.rz) * c.ny + j / f.ry) * c.nx + i / f.rx;
        for (int d = 0; d < 6; ++d) {
          double tb = bf.b[d][q];
          if (tb == 0.0) continue;
          int ax = d / 2;
          if (r[ax] == 1) { out.b[d][C] += tb; continue; }
          // internal face of the coarse cell along axis ax, in this fine row
          double tint;
          if (ax == 0) tint = f.Te[fi((i / 2) * 2, j, k)];
          else if (ax == 1) tint = f.Tn[fi(i, (j / 2) * 2, k)];
          else tint = f.Tu[fi(i, j, (k / 2) * 2)];
          out.b[d][C] += 1.0 / (1.0 / tb + 0.5 / tint);
        }
      }
  return out;
}

static int upload_f32(lt_ctx* ctx, std::vector<void*>& list, float** dst, const std::vector<double>& src) {
  std::vector<float> tmp(src.size());
  for (size_t i = 0; i < src.size(); ++i) tmp[i] = (float)src[i];
  int rc = dalloc(ctx, list, dst, tmp.size());
  if (rc) return rc;
  CK(cudaMemcpy(*dst, tmp.data(), tmp.size() * sizeof(float), cudaMemcpyHostToDevice));
  return LT_OK;
}

static int upload_df(lt_ctx* ctx, std::vector<void*>& list, const float** hi, const float** lo,
                     const std::vector<double>& src) {
  std::vector<float> th(src.size()), tl(src.size());
  for (size_t i = 0; i < src.size(); ++i) {
    lt::df v = lt::df_from_double(src[i]);
    th[i] = v.hi;
    tl[i] = v.lo;
  }
  float *dh, *dl;
  int rc = dalloc(ctx, list, &dh, th.size());
  if (rc) return rc;
  rc = dalloc(ctx, list, &dl, tl.size());
  if (rc) return rc;
  CK(cudaMemcpy(dh, th.data(), th.size() * sizeof(float), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(dl, tl.data(), tl.size() * sizeof(float), cudaMemcpyHostToDevice));
  *hi = dh;
  *lo = dl;
  return LT_OK;
}

extern "C" int lt_setup_grid(lt_ctx* ctx, int nx, int ny, int nz, double dx, double dy, double dz,
                             const double* kappa, const double* Ss, const int* bc, const double* Sy) {
  if (!ctx) return LT_ERR_INVALID_ARG;
  if (nx < 1 || ny < 1 || nz < 1) return fail(ctx, LT_ERR_INVALID_ARG, "grid dims %d x %d x %d must be >= 1", nx, ny, nz);
  if ((int64_t)nx * ny * nz > (1LL << 30)) return fail(ctx, LT_ERR_INVALID_ARG, "grid too large");
  if (!(dx > 0 && dy > 0 && dz > 0) || !std::isfinite(dx) || !std::isfinite(dy) || !std::isfinite(dz))
    return fail(ctx, LT_ERR_INVALID_ARG, "cell sizes must be positive and finite");
  if (!kappa || !Ss || !bc) return fail(ctx, LT_ERR_INVALID_ARG, "kappa, Ss and bc are required");
  bool any_wt = false;
  for (int d = 0; d < 6; ++d) {
    if (bc[d] != LT_BC_DIRICHLET && bc[d] != LT_BC_NEUMANN && bc[d] != LT_BC_WATERTABLE)
      return fail(ctx, LT_ERR_INVALID_ARG, "bc[%d]=%d: must be Dirichlet (0), Neumann (1) or water table (2)", d, bc[d]);
    any_wt |= bc[d] == LT_BC_WATERTABLE;
  }
  if (any_wt && !Sy) return fail(ctx, LT_ERR_INVALID_ARG, "a water-table face needs the specific yield Sy");
  const int64_t N = (int64_t)nx * ny * nz;
  if (any_wt)
    for (int64_t c = 0; c < N; ++c)
      if (!(Sy[c] >= 0.0) || !std::isfinite(Sy[c]))
        return fail(ctx, LT_ERR_INVALID_ARG, "Sy[%lld]=%g must be finite and >= 0", (long long)c, Sy[c]);
  for (int64_t c = 0; c < N; ++c) {
    if (!(kappa[c] > 0.0) || !std::isfinite(kappa[c]))
      return fail(ctx, LT_ERR_INVALID_ARG, "kappa[%lld]=%g must be positive and finite", (long long)c, kappa[c]);
    if (!(Ss[c] > 0.0) || !std::isfinite(Ss[c]))
      return fail(ctx, LT_ERR_INVALID_ARG, "Ss[%lld]=%g must be positive and finite", (long long)c, Ss[c]);
  }
  bool any_dirichlet = false;
  for (int d = 0; d < 6; ++d) any_dirichlet |= (bc[d] == LT_BC_DIRICHLET);
  if (!any_dirichlet) return fail(ctx, LT_ERR_INVALID_ARG, "at least one Dirichlet face is required (K must be nonsingular)");
  CK(cudaSetDevice(ctx->device));
  CK(cudaStreamSynchronize(ctx->stream));
  // A new aquifer on a grid of the same dimensions keeps the Krylov workspace (its sizes depend only
  // on the dimensions, the level structure and the plan): only the coefficients are replaced.
  const bool keep_ws = ctx->have_grid && ctx->ws.nb > 0 && nx == ctx->nx && ny == ctx->ny && nz == ctx->nz;
  float2* keep_u[lt::kMaxLevels] = {};
  float2* keep_f[lt::kMaxLevels] = {};
  const int keep_nlev = ctx->mg.nlev;
  if (keep_ws)
    for (int l = 0; l < keep_nlev; ++l) { keep_u[l] = ctx->mg.h_levels[l].u; keep_f[l] = ctx->mg.h_levels[l].f; }
  else
    free_ws(ctx);
  free_list(ctx->grid_allocs);
  if (ctx->mg.d_levels) { cudaFree(ctx->mg.d_levels); ctx->mg.d_levels = nullptr; }
  ctx->have_grid = false;
  lt::tma_cache_free(ctx->mg);
  lt::tma_cache_free(ctx->pc_mg);
  for (float** p : {&ctx->d_lk, &ctx->d_mD, &ctx->d_D32}) {
    if (*p) cudaFree(*p);
    *p = nullptr;
  }
  ctx->last_group.clear(); ctx->last_nit.clear(); ctx->last_tau.clear();
  free_list(ctx->pc_allocs);
  ctx->pc_mg.d_levels = nullptr;
  ctx->pc_nb = 0;
  ctx->nx = nx; ctx->ny = ny; ctx->nz = nz; ctx->N = N;
  ctx->dx = dx; ctx->dy = dy; ctx->dz = dz;
  for (int d = 0; d < 6; ++d) ctx->bc[d] = bc[d];
  ctx->kappa.assign(kappa, kappa + N);
  ctx->Ss.assign(Ss, Ss + N);

  // fine level, float64 (Sec. 2.1 restated as two-point-flux finite volumes)
  HostLevel L0;
  L0.nx = nx; L0.ny = ny; L0.nz = nz; L0.N = (int)N;
  L0.Te.assign(N, 0.0); L0.Tn.assign(N, 0.0); L0.Tu.assign(N, 0.0); L0.D.assign(N, 0.0); L0.m.assign(N, 0.0);
  const double ax = dy * dz / dx, ay = dx * dz / dy, az = dx * dy / dz, vol = dx * dy * dz;
  auto harm = [](double a, double b) { return 2.0 * a * b / (a + b); };
  BFaces bf;
  for (int d = 0; d < 6; ++d) bf.b[d].assign(N, 0.0);
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        size_t q = ((size_t)k * ny + j) * nx + i;
        double kc = kappa[q];
        if (i + 1 < nx) L0.Te[q] = ax * harm(kc, kappa[q + 1]);
        if (j + 1 < ny) L0.Tn[q] = ay * harm(kc, kappa[q + nx]);
        if (k + 1 < nz) L0.Tu[q] = az * harm(kc, kappa[q + (size_t)nx * ny]);
        if (i == 0 && bc[0] == 0) bf.b[0][q] = 2.0 * kc * ax;
        if (i == nx - 1 && bc[1] == 0) bf.b[1][q] = 2.0 * kc * ax;
        if (j == 0 && bc[2] == 0) bf.b[2][q] = 2.0 * kc * ay;
        if (j == ny - 1 && bc[3] == 0) bf.b[3][q] = 2.0 * kc * ay;
        if (k == 0 && bc[4] == 0) bf.b[4][q] = 2.0 * kc * az;
        if (k == nz - 1 && bc[5] == 0) bf.b[5][q] = 2.0 * kc * az;
        // storage: Ss V, plus S_y times the face area on water-table faces (Sec. 2.1, the boundary
        // term (S_y d phi / dt, psi) of the weak form; no flux through those faces)
        double m = Ss[q] * vol;
        if (any_wt) {
          const double sy = Sy[q];
          if (i == 0 && bc[0] == LT_BC_WATERTABLE) m += sy * dy * dz;
          if (i == nx - 1 && bc[1] == LT_BC_WATERTABLE) m += sy * dy * dz;
          if (j == 0 && bc[2] == LT_BC_WATERTABLE) m += sy * dx * dz;
          if (j == ny - 1 && bc[3] == LT_BC_WATERTABLE) m += sy * dx * dz;
          if (k == 0 && bc[4] == LT_BC_WATERTABLE) m += sy * dx * dy;
          if (k == nz - 1 && bc[5] == LT_BC_WATERTABLE) m += sy * dx * dy;
        }
        L0.m[q] = m;
      }
  level_diag(L0, bf);
  ctx->hl.clear();
  std::vector<BFaces> bfs;
  ctx->hl.push_back(L0);
  bfs.push_back(bf);
  for (;;) {
    HostLevel& f = ctx->hl.back();
    f.rx = (f.nx % 2 == 0 && f.nx >= 2) ? 2 : 1;
    f.ry = (f.ny % 2 == 0 && f.ny >= 2) ? 2 : 1;
    f.rz = (f.nz % 2 == 0 && f.nz >= 2) ? 2 : 1;
    bool can = (f.rx * f.ry * f.rz > 1);
    if (f.N <= 64 || !can || (int)ctx->hl.size() >= lt::kMaxLevels) {
      f.rx = f.ry = f.rz = 1;
      break;
    }
    HostLevel c = coarsen(f);
    BFaces cb = coarsen_bfaces(f, c, bfs.back());
    level_diag(c, cb);
    ctx->hl.push_back(c);
    bfs.push_back(cb);
  }
  const int nlev = (int)ctx->hl.size();
  if (ctx->hl.back().N > 1024)
    return fail(ctx, LT_ERR_INVALID_ARG,
                "grid %d x %d x %d coarsens only to %d cells (> 1024): use dimensions with more factors of 2", nx,
                ny, nz, ctx->hl.back().N);
  lt::MGHost& mg = ctx->mg;
  mg.nlev = nlev;
  mg.npre = ctx->opts.mg_pre;
  mg.npost = ctx->opts.mg_post;
  mg.tile = ctx->opts.mg_tile;
  mg.tma = ctx->opts.mg_tma;
  mg.dmask = 0;
  for (int d = 0; d < 6; ++d)
    if (bc[d] == 0) mg.dmask |= (1 << d);
  mg.coarse_direct = ctx->hl.back().N <= lt::kDirectCells ? 1 : 0;
  mg.lc = nlev - 1;
  while (mg.lc > 0 && ctx->hl[mg.lc - 1].N <= lt::kCoarseCells) --mg.lc;
  for (int l = 0; l < nlev; ++l) {
    const HostLevel& h = ctx->hl[l];
    lt::Level& L = mg.h_levels[l];
    L.nx = h.nx; L.ny = h.ny; L.nz = h.nz; L.N = h.N;
    L.rx = h.rx; L.ry = h.ry; L.rz = h.rz;
    int rc;
    if ((rc = upload_f32(ctx, ctx->grid_allocs, &L.Te, h.Te))) return rc;
    if ((rc = upload_f32(ctx, ctx->grid_allocs, &L.Tn, h.Tn))) return rc;
    if ((rc = upload_f32(ctx, ctx->grid_allocs, &L.Tu, h.Tu))) return rc;
    if ((rc = upload_f32(ctx, ctx->grid_allocs, &L.D, h.D))) return rc;
    if ((rc = upload_f32(ctx, ctx->grid_allocs, &L.m, h.m))) return rc;
    L.u = L.f = nullptr;   // per-batch vectors, set when a workspace is sized
  }
  if (keep_ws) {
    if (nlev == keep_nlev) {
      for (int l = 0; l < nlev; ++l) { mg.h_levels[l].u = keep_u[l]; mg.h_levels[l].f = keep_f[l]; }
    } else {
      free_ws(ctx);   // (cannot happen for equal dimensions; kept as a guard)
    }
  }
  lt::FineExact& fe = ctx->fe;
  fe.nx = nx; fe.ny = ny; fe.nz = nz; fe.N = (int)N;
  int rc;
  if ((rc = upload_df(ctx, ctx->grid_allocs, &fe.Te_hi, &fe.Te_lo, L0.Te))) return rc;
  if ((rc = upload_df(ctx, ctx->grid_allocs, &fe.Tn_hi, &fe.Tn_lo, L0.Tn))) return rc;
  if ((rc = upload_df(ctx, ctx->grid_allocs, &fe.Tu_hi, &fe.Tu_lo, L0.Tu))) return rc;
  if ((rc = upload_df(ctx, ctx->grid_allocs, &fe.D_hi, &fe.D_lo, ctx->hl[0].D))) return rc;
  if ((rc = upload_df(ctx, ctx->grid_allocs, &fe.m_hi, &fe.m_lo, L0.m))) return rc;
  {
    std::vector<double> Bd(N, 0.0), mss(N);
    for (int64_t c = 0; c < N; ++c) {
      for (int d = 0; d < 6; ++d) Bd[c] += bfs[0].b[d][c];
      mss[c] = Ss[c] * vol;      // dM / dlog Ss_c: the water-table storage S_y A does not depend on Ss
    }
    auto up = [&](double** dst, const std::vector<double>& v) -> int {
      int r = dalloc(ctx, ctx->grid_allocs, dst, v.size());
      if (r) return r;
      CK(cudaMemcpy(*dst, v.data(), v.size() * sizeof(double), cudaMemcpyHostToDevice));
      return LT_OK;
    };
    if ((rc = up(&ctx->g_Te, L0.Te)) || (rc = up(&ctx->g_Tn, L0.Tn)) || (rc = up(&ctx->g_Tu, L0.Tu)) ||
        (rc = up(&ctx->g_kap, ctx->kappa)) || (rc = up(&ctx->g_Bd, Bd)) || (rc = up(&ctx->g_m, mss)))
      return rc;
  }
  CK(cudaMalloc(&mg.d_levels, sizeof(lt::Level) * lt::kMaxLevels));
  if (ctx->ws.nb > 0)   // kept workspace: the device level table must point at the new coefficients
    CK(cudaMemcpy(mg.d_levels, mg.h_levels, sizeof(lt::Level) * nlev, cudaMemcpyHostToDevice));
  lt::inner_cluster_plan(mg, ctx->inner_alt[2], 16, 256);
  lt::inner_cluster_plan(mg, ctx->inner_alt[3], 8, 256, 1);
  lt::inner_cluster_plan(mg, ctx->inner_alt[4], 4, 512, 1);
  if (lt::inner_cluster_plan(mg, ctx->inner) || any_cluster_plan(ctx)) {
    // the four faces of every finest-level cell in one 16-byte record (zero across domain edges),
    // in red-black order: colour (x + y) & 1 first, then row by row, x / 2 within the row
    const HostLevel& h0 = ctx->hl[0];
    std::vector<float4> p4(N);
    for (int64_t c = 0; c < N; ++c) {
      const int x = (int)(c % nx), y = (int)(c / nx);
      p4[((x + y) & 1) * (N / 2) + (int64_t)y * (nx / 2) + x / 2] = make_float4(x + 1 < nx ? (float)h0.Te[c] : 0.f, x > 0 ? (float)h0.Te[c - 1] : 0.f,
                          y + 1 < ny ? (float)h0.Tn[c] : 0.f, y > 0 ? (float)h0.Tn[c - nx] : 0.f);
    }
    float4* d4 = nullptr;
    if ((rc = dalloc(ctx, ctx->grid_allocs, &d4, (size_t)N))) return rc;
    CK(cudaMemcpy(d4, p4.data(), N * sizeof(float4), cudaMemcpyHostToDevice));
    ctx->inner.p4 = d4;
    for (lt::InnerPlan& q : ctx->inner_alt) q.p4 = d4;
  }
  ctx->have_grid = true;
  ctx->src.clear(); ctx->Q.clear(); ctx->rec.clear();
  ctx->rate_a.clear(); ctx->rate_l.clear(); ctx->phi0.clear();
  return LT_OK;
}

extern "C" int lt_set_sources(lt_ctx* ctx, int ns, const int64_t* cells, const double* Q) {
  if (!ctx) return LT_ERR_INVALID_ARG;
  if (!ctx->have_grid) return fail(ctx, LT_ERR_STATE, "lt_setup_grid must come first");
  if (ns < 0 || (ns > 0 && (!cells || !Q))) return fail(ctx, LT_ERR_INVALID_ARG, "ns=%d with null arrays", ns);
  for (int s = 0; s < ns; ++s) {
    if (cells[s] < 0 || cells[s] >= ctx->N)
      return fail(ctx, LT_ERR_INVALID_ARG, "source %d cell %lld out of range [0,%lld)", s, (long long)cells[s],
                  (long long)ctx->N);
    if (!std::isfinite(Q[s])) return fail(ctx, LT_ERR_INVALID_ARG, "source %d rate not finite", s);
  }
  ctx->src.assign(cells, cells + ns);
  ctx->Q.assign(Q, Q + ns);
  ctx->rate_a.clear(); ctx->rate_l.clear();
  return LT_OK;
}

extern "C" int lt_set_source_rates(lt_ctx* ctx, int ns, const int* nterm, const double* a, const double* lambda) {
  if (!ctx) return LT_ERR_INVALID_ARG;
  if (!ctx->have_grid) return fail(ctx, LT_ERR_STATE, "lt_setup_grid must come first");
  if (!nterm) {
    ctx->rate_a.clear(); ctx->rate_l.clear();
    return LT_OK;
  }
  if (ns != (int)ctx->src.size())
    return fail(ctx, LT_ERR_INVALID_ARG, "ns=%d must equal the %d sources set by lt_set_sources", ns,
                (int)ctx->src.size());
  if (!a || !lambda) return fail(ctx, LT_ERR_INVALID_ARG, "a and lambda must not be null");
  std::vector<std::vector<double>> A(ns), L(ns);
  size_t off = 0;
  for (int s = 0; s < ns; ++s) {
    if (nterm[s] < 1 || nterm[s] > 64) return fail(ctx, LT_ERR_INVALID_ARG, "nterm[%d]=%d must be in [1,64]", s, nterm[s]);
    for (int j = 0; j < nterm[s]; ++j, ++off) {
      if (!std::isfinite(a[off])) return fail(ctx, LT_ERR_INVALID_ARG, "a[%zu] is not finite", off);
      if (!(lambda[off] >= 0.0) || !std::isfinite(lambda[off]))
        return fail(ctx, LT_ERR_INVALID_ARG, "lambda[%zu]=%g must be finite and >= 0", off, lambda[off]);
      A[s].push_back(a[off]);
      L[s].push_back(lambda[off]);
    }
  }
  ctx->rate_a.swap(A);
  ctx->rate_l.swap(L);
  return LT_OK;
}

extern "C" int lt_set_initial_state(lt_ctx* ctx, const double* phi0) {
  if (!ctx) return LT_ERR_INVALID_ARG;
  if (!ctx->have_grid) return fail(ctx, LT_ERR_STATE, "lt_setup_grid must come first");
  if (!phi0) {
    ctx->phi0.clear();
    return LT_OK;
  }
  bool any = false;
  for (int64_t c = 0; c < ctx->N; ++c) {
    if (!std::isfinite(phi0[c])) return fail(ctx, LT_ERR_INVALID_ARG, "phi0[%lld] is not finite", (long long)c);
    any |= phi0[c] != 0.0;
  }
  if (any) ctx->phi0.assign(phi0, phi0 + ctx->N);
  else ctx->phi0.clear();
  return LT_OK;
}

// Laplace transform of source s's rate at z (Sec. 2.1-2.2): sum_j a_j / (z + lambda_j), or Q_s / z
static cplx qhat(const lt_ctx* ctx, int s, cplx z) {
  if (ctx->rate_a.empty()) return ctx->Q[s] / z;
  cplx v(0.0, 0.0);
  for (size_t j = 0; j < ctx->rate_a[s].size(); ++j) v += ctx->rate_a[s][j] / (z + ctx->rate_l[s][j]);
  return v;
}

extern "C" int lt_set_receivers(lt_ctx* ctx, int nr, const int64_t* cells) {
  if (!ctx) return LT_ERR_INVALID_ARG;
  if (!ctx->have_grid) return fail(ctx, LT_ERR_STATE, "lt_setup_grid must come first");
  if (nr < 0 || (nr > 0 && !cells)) return fail(ctx, LT_ERR_INVALID_ARG, "nr=%d with null array", nr);
  for (int r = 0; r < nr; ++r)
    if (cells[r] < 0 || cells[r] >= ctx->N)
      return fail(ctx, LT_ERR_INVALID_ARG, "receiver %d cell %lld out of range", r, (long long)cells[r]);
  ctx->rec.assign(cells, cells + nr);
  return LT_OK;
}

// ------------------------------------------------------------------ solve plan
struct Plan {
  int nt = 0, G = 0, Nk = 0;
  std::vector<double> times;            // caller order
  std::vector<int> tgroup;              // time -> group
  std::vector<int> tpos;                // time -> position inside its group
  std::vector<int> gcount;              // times per group
  std::vector<std::vector<cplx>> z, w;  // per time: Nk nodes / weights
  std::vector<cplx> tau;                // [G][2]
  // bases
  int nb = 0, nsh = 0;
  std::vector<int64_t> rhs_cell;        // per basis
  std::vector<int> group;               // per basis
  std::vector<int> shift_off;           // nb + 1
  std::vector<int> sh_basis;
  std::vector<cplx> zsh;
  // bases [dense_b0, nb) (one per group) solve for the dense right-hand side M phi_0 / beta0
  int dense_b0 = -1;
  double beta0 = 0.0;
  std::vector<double> wabs;             // [nsh] |w_k qhat(z_k)| (quadrature stopping rule)
  bool block = false;                   // block flexible GMRES over the sources of each group
};

// rhs: one point right-hand side per entry; the first n_src of them are sources (weights of the
// quadrature stopping rule use their rate transforms).  dense: one more basis per group for the
// initial-state right-hand side M phi_0.
static int make_plan(lt_ctx* ctx, int nt, const double* times, const std::vector<int64_t>& rhs, Plan& P,
                     int n_src = 0, bool dense = false) {
  const lt_opts& o = ctx->opts;
  P.nt = nt;
  P.times.assign(times, times + nt);
  P.Nk = o.Nz / 2;
  P.G = std::min(o.groups, nt);
  std::vector<int> order(nt);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return times[a] < times[b]; });
  P.tgroup.assign(nt, 0);
  P.tpos.assign(nt, 0);
  P.gcount.assign(P.G, 0);
  for (int q = 0; q < nt; ++q) {
    int t = order[q];
    int g = (int)((int64_t)q * P.G / nt);
    P.tgroup[t] = g;
    P.tpos[t] = P.gcount[g]++;
  }
  P.z.resize(nt);
  P.w.resize(nt);
  for (int t = 0; t < nt; ++t) talbot_half(times[t], o.Nz, P.z[t], P.w[t]);
  // group shift lists in position order
  std::vector<std::vector<int>> gtimes(P.G);
  for (int q = 0; q < nt; ++q) gtimes[P.tgroup[order[q]]].push_back(order[q]);
  P.tau.assign(2 * P.G, cplx(0, 0));
  for (int g = 0; g < P.G; ++g) {
    cplx lo(1e300, 0), hi(-1e300, 0);
    for (int t : gtimes[g])
      for (const cplx& z : P.z[t]) {
        if (z.real() < lo.real()) lo = z;
        if (z.real() > hi.real()) hi = z;
      }
    if (o.tau_project) {
      lo = cplx(std::max(lo.real(), 0.0), lo.imag());
      hi = cplx(std::max(hi.real(), 0.0), hi.imag());
    }
    P.tau[2 * g] = lo;
    P.tau[2 * g + 1] = (o.tau_policy == LT_TAU_SINGLE) ? lo : hi;
  }
  const int nrhs = (int)rhs.size() + (dense ? 1 : 0);
  P.nb = nrhs * P.G;
  P.dense_b0 = dense ? (int)rhs.size() * P.G : -1;
  P.beta0 = 0.0;
  if (dense) {   // beta0 = ||M phi_0||_2
    for (int64_t c = 0; c < ctx->N; ++c) P.beta0 += std::pow(ctx->hl[0].m[c] * ctx->phi0[c], 2);
    P.beta0 = std::sqrt(P.beta0);
  }
  P.rhs_cell.resize(P.nb);
  P.group.resize(P.nb);
  P.shift_off.assign(P.nb + 1, 0);
  P.zsh.clear();
  P.sh_basis.clear();
  P.wabs.clear();
  for (int s = 0; s < nrhs; ++s)
    for (int g = 0; g < P.G; ++g) {
      int b = s * P.G + g;
      P.rhs_cell[b] = s < (int)rhs.size() ? rhs[s] : -1;
      P.group[b] = g;
      for (int t : gtimes[g])
        for (int k = 0; k < P.Nk; ++k) {
          const cplx z = P.z[t][k];
          P.zsh.push_back(z);
          P.sh_basis.push_back(b);
          P.wabs.push_back(std::abs(P.w[t][k] * (s < n_src ? qhat(ctx, s, z) : cplx(1.0, 0.0))));
        }
      P.shift_off[b + 1] = (int)P.zsh.size();
    }
  P.nsh = (int)P.zsh.size();
  for (int g = 0; g < P.G; ++g) std::sort(gtimes[g].begin(), gtimes[g].end(), [&](int a, int b) { return P.tpos[a] < P.tpos[b]; });
  return LT_OK;
}

// first global shift index of time t inside basis b
static int shift_of(const Plan& P, int b, int t) { return P.shift_off[b] + P.tpos[t] * P.Nk; }

// dense inverse of the coarsest operator K_c + tau M_c (complex LU with partial pivoting)
static bool dense_inverse(const HostLevel& L, cplx tau, std::vector<cplx>& inv) {
  const int n = L.N;
  std::vector<cplx> A((size_t)n * n, 0.0);
  for (int k = 0; k < L.nz; ++k)
    for (int j = 0; j < L.ny; ++j)
      for (int i = 0; i < L.nx; ++i) {
        int q = (k * L.ny + j) * L.nx + i;
        A[(size_t)q * n + q] = L.D[q] + tau * L.m[q];
        auto off = [&](int p, double t) {
          A[(size_t)q * n + p] -= t;
        };
        if (i + 1 < L.nx) off(q + 1, L.Te[q]);
        if (i > 0) off(q - 1, L.Te[q - 1]);
        if (j + 1 < L.ny) off(q + L.nx, L.Tn[q]);
        if (j > 0) off(q - L.nx, L.Tn[q - L.nx]);
        if (k + 1 < L.nz) off(q + L.nx * L.ny, L.Tu[q]);
        if (k > 0) off(q - L.nx * L.ny, L.Tu[q - L.nx * L.ny]);
      }
  inv.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) inv[(size_t)i * n + i] = 1.0;
  for (int col = 0; col < n; ++col) {
    int piv = col;
    double best = std::abs(A[(size_t)col * n + col]);
    for (int r = col + 1; r < n; ++r)
      if (std::abs(A[(size_t)r * n + col]) > best) { best = std::abs(A[(size_t)r * n + col]); piv = r; }
    if (best == 0.0) return false;
    if (piv != col)
      for (int c = 0; c < n; ++c) {
        std::swap(A[(size_t)piv * n + c], A[(size_t)col * n + c]);
        std::swap(inv[(size_t)piv * n + c], inv[(size_t)col * n + c]);
      }
    cplx d = 1.0 / A[(size_t)col * n + col];
    for (int c = 0; c < n; ++c) { A[(size_t)col * n + c] *= d; inv[(size_t)col * n + c] *= d; }
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      cplx f = A[(size_t)r * n + col];
      if (f == 0.0) continue;
      for (int c = 0; c < n; ++c) {
        A[(size_t)r * n + c] -= f * A[(size_t)col * n + c];
        inv[(size_t)r * n + c] -= f * inv[(size_t)col * n + c];
      }
    }
  }
  return true;
}

static int ensure_ws(lt_ctx* ctx, const Plan& P) {
  Workspace& ws = ctx->ws;
  const lt_opts& o = ctx->opts;
  const int nc = ctx->hl.back().N;
  const int nc2 = ctx->mg.coarse_direct ? nc * nc : 0;
  if (ws.nb >= P.nb && ws.maxit == o.maxit && ws.nsh >= P.nsh && ws.rounds == o.inner_rounds && ws.N == ctx->N &&
      ws.ngroups >= P.G && ws.nc2 >= nc2 && ws.prec == o.precision &&
      (ws.l0u != nullptr) == cluster_plan(ctx).u0_global)
    return LT_OK;
  CK(cudaStreamSynchronize(ctx->stream));
  free_ws(ctx);
  lt::tma_cache_free(ctx->mg);
  lt::Batch& bt = ws.bt;
  const int nb = P.nb, M = o.maxit, R = o.inner_rounds, nsh = P.nsh;
  const size_t N = (size_t)ctx->N;
  auto& A = ws.allocs;
  int rc = 0;
#define AL(p, n) if ((rc = dalloc(ctx, A, &p, (size_t)(n)))) return rc
  // reduced precision keeps one float32 plane per vector (the lo planes stay null)
  const bool df = o.precision == LT_PREC_FP64;
  AL(bt.V_hi, (size_t)nb * (M + 1) * N);
  AL(bt.U_hi, (size_t)nb * M * N);
  AL(bt.S_hi, (size_t)nb * N);
  bt.V_lo = bt.U_lo = bt.S_lo = nullptr;
  if (df) {
    AL(bt.V_lo, (size_t)nb * (M + 1) * N);
    AL(bt.U_lo, (size_t)nb * M * N);
    AL(bt.S_lo, (size_t)nb * N);
  }
  AL(bt.tau_grp, 2 * P.G); AL(bt.group, nb); AL(bt.tau_pattern, 5); AL(bt.tau_cur, nb); AL(bt.tau_slot, nb);
  AL(bt.rnorm2, (size_t)nb * (R + 1)); AL(bt.dot, (size_t)nb * 2 * (M + 1)); AL(bt.H, (size_t)nb * M * (M + 1));
  AL(bt.snorm2, nb); AL(bt.active, nb); AL(bt.nit, nb); AL(bt.inner_max, nb); AL(bt.rhs_cell, nb);
  AL(bt.shift_off, nb + 1); AL(bt.zsh, nsh); AL(bt.R, (size_t)nsh * M * M); AL(bt.rc, (size_t)nsh * M);
  AL(bt.rs, (size_t)nsh * M); AL(bt.g, (size_t)nsh * (M + 1)); AL(bt.conv_it, nsh); AL(bt.pres, nsh);
  AL(bt.Y, (size_t)nsh * M);
  AL(bt.work, lt::kWorkSlots);
  AL(bt.itol2, nb);
  AL(bt.rmax, nb);
  AL(bt.jdev, 8);
  {
    double* w = nullptr;
    float *rh = nullptr, *rl = nullptr;
    AL(w, nsh); AL(rh, N); AL(rl, N);
    bt.wabs = w; bt.rhs_hi = rh; bt.rhs_lo = rl;
  }
  if (nc2) AL(bt.coarse_inv, (size_t)2 * P.G * nc2);
  if (ctx->inner.ok || any_cluster_plan(ctx)) AL(ws.l0q, (size_t)nb * N);
  if (cluster_plan(ctx).u0_global) AL(ws.l0u, (size_t)nb * N);
  // multigrid vectors
  for (int l = 0; l < ctx->mg.nlev; ++l) {
    lt::Level& L = ctx->mg.h_levels[l];
    AL(L.u, (size_t)nb * L.N);
    AL(L.f, (size_t)nb * L.N);
  }
#undef AL
  CK(cudaMemcpy(ctx->mg.d_levels, ctx->mg.h_levels, sizeof(lt::Level) * ctx->mg.nlev, cudaMemcpyHostToDevice));
  ws.nb = nb; ws.maxit = M; ws.nsh = nsh; ws.rounds = R; ws.N = ctx->N; ws.ngroups = P.G; ws.nc2 = nc2;
  ws.prec = o.precision;
  bt.nb = nb; bt.maxit = M; bt.N = ctx->N; bt.rounds = R; bt.nsh = nsh;
  return LT_OK;
}

// Arrays of the block flexible GMRES (block = 1): the bases q * G + g of group g form one block of
// p = nb / G right-hand sides; the member-0 shifts [shift_off[0], shift_off[G]) index the block shifts.
static int ensure_block_ws(lt_ctx* ctx, const Plan& P) {
  Workspace& ws = ctx->ws;
  lt::Batch& bt = ws.bt;
  const int p = P.nb / P.G, G = P.G, M = ctx->opts.maxit, nbs = P.shift_off[G], nsh = P.nsh;
  const size_t bld = (size_t)M * p, hld = (size_t)(M + 1) * p;
  if (!(ws.bk_p == p && ws.bk_G == G && ws.bk_M == M && ws.bk_nbs == nbs && ws.bk_nsh == nsh)) {
    CK(cudaStreamSynchronize(ctx->stream));
    free_list(ws.block_allocs);
    ws.bk_p = ws.bk_G = ws.bk_M = ws.bk_nbs = ws.bk_nsh = 0;
    auto& A = ws.block_allocs;
    int rc = 0;
#define AL(ptr, n) if ((rc = dalloc(ctx, A, &ptr, (size_t)(n)))) return rc
    AL(bt.bdot, (size_t)G * 2 * bld * p);
    AL(bt.bgram, (size_t)G * 2 * p * p);
    AL(bt.bw, (size_t)G * 2 * p * p);
    AL(bt.bH, (size_t)G * bld * hld);
    AL(bt.bR, (size_t)nbs * bld * hld);
    AL(bt.brc, (size_t)nbs * bld * p);
    AL(bt.brs, (size_t)nbs * bld * p);
    AL(bt.bG, (size_t)nbs * hld * p);
    AL(bt.bY, (size_t)nsh * bld);
    AL(bt.gany, G);
    AL(bt.grmax, G);
#undef AL
    ws.bk_p = p; ws.bk_G = G; ws.bk_M = M; ws.bk_nbs = nbs; ws.bk_nsh = nsh;
  }
  bt.block = 1;
  bt.bp = p;
  bt.ngroups = G;
  bt.bld = (int)bld;
  bt.hld = (int)hld;
  bt.nbs = nbs;
  return LT_OK;
}

// State of the batched flexible shifted Krylov solves of one context between
// the stages below (begin: tables, workspace, graph capture; launch: enqueue
// outer iterations; poll: read the active flags; end: back-substitution, x_k,
// true residuals, statistics).  run_solves chains them for one context;
// lt_forward_batch interleaves them over several contexts.
struct SolveState {
  int j = 0, cycles = 0, per_iter = 0;
  bool use_graph = false, done = false;
  cudaGraphExec_t gexec = nullptr;
  cudaStream_t q = nullptr;
  lt::Prof* pf = nullptr;
  std::vector<int> act;
  // decoupled parts (nbr > 0): bases [bb0[p], bb0[p] + bbn[p]) with their own iteration counter,
  // graph and stream, so that one part's solves run while another part orthogonalises
  int nbr = 0;
  cudaGraphExec_t bgx[8] = {};
  cudaStream_t bq[8] = {};
  int bj[8] = {}, bb0[8] = {}, bbn[8] = {}, bper[8] = {};
  bool bdone[8] = {};
  // the end-of-solve work (y_k, x_k, true residuals) already queued part by part, as each finished
  bool tail_done = false, tail_x = false;
  int* d_shb = nullptr;      // [nsh] basis of each shift
  double* d_res2 = nullptr;  // [nsh] squared true residuals
};

// the whole preconditioner solve of each basis runs in one thread-block cluster
static bool uses_cluster_solve(const lt_ctx* ctx) {
  return ctx->opts.precond == 0 && ctx->opts.mg_cluster >= 1 && cluster_plan(ctx).ok;
}

// The bases [b0, b0 + n) of a batch as a batch of their own: per-basis arrays
// offset by b0; shift indices (shift_off) stay global, so per-shift arrays
// are shared; the outer-iteration counter is shared too.
static lt::Batch sub_batch(const lt::Batch& bt, int b0, int n, int jslot = 0) {
  lt::Batch v = bt;
  v.jdev = bt.jdev + jslot;
  const size_t N = (size_t)bt.N, M = (size_t)bt.maxit;
  v.nb = n;
  v.itol2 += b0; v.rmax += b0;
  v.V_hi += b0 * (M + 1) * N; v.V_lo = lt::lo_at(bt.V_lo, b0 * (M + 1) * N);
  v.U_hi += b0 * M * N; v.U_lo = lt::lo_at(bt.U_lo, b0 * M * N);
  v.S_hi += b0 * N; v.S_lo = lt::lo_at(bt.S_lo, b0 * N);
  v.group += b0; v.tau_cur += b0; v.tau_slot += b0;
  v.rnorm2 += (size_t)b0 * (bt.rounds + 1);
  v.dot += (size_t)b0 * 2 * (M + 1);
  v.H += (size_t)b0 * M * (M + 1);
  v.snorm2 += b0; v.active += b0; v.nit += b0; v.inner_max += b0; v.rhs_cell += b0;
  v.shift_off += b0;
  return v;
}

// One outer iteration with cluster-resident preconditioner solves.  When the
// bases outnumber the clusters the device holds at once, they are split in
// two halves issued as two independent branches (the second on side_stream):
// while one half's second wave of clusters runs, the other half's
// Gram-Schmidt and least squares use the SMs the clusters leave idle.
static int launch_iteration_cluster(lt_ctx* ctx, cudaStream_t q, int jj, int* nlq, lt::Prof* pf) {
  const lt_opts& o = ctx->opts;
  lt::Batch& bt = ctx->ws.bt;
  const int nb = bt.nb;
  // (not inside lt_forward_noalloc, which creates no streams or events)
  // (nor in block mode, whose Arnoldi process couples the bases of a group)
  const lt::InnerPlan& ip = cluster_plan(ctx);
  if (ip.u0_global && !ctx->ws.l0u) return fail(ctx, LT_ERR_STATE, "finest-level iterate array missing");
  const int parts = (!bt.block && nb > ip.max_clusters && nb >= 2 && ctx->arena_base == nullptr) ? 2 : 1;
  if (parts == 2) {
    if (!ctx->side_stream) CK(cudaStreamCreateWithFlags(&ctx->side_stream, cudaStreamNonBlocking));
    if (!ctx->ev_fork) CK(cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming));
    if (!ctx->ev_join) CK(cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming));
    CK(cudaEventRecord(ctx->ev_fork, q));
    CK(cudaStreamWaitEvent(ctx->side_stream, ctx->ev_fork, 0));
  }
  const int half = (nb + 1) / 2;
  for (int part = 0; part < parts; ++part) {
    const int b0 = part == 0 ? 0 : half;
    const int n = parts == 1 ? nb : (part == 0 ? half : nb - half);
    // with per-launch CUDA-event timing on, both halves go to one stream so that the timed
    // windows of different launches never overlap
    const bool timing = pf && pf->cls >= 0;
    cudaStream_t qs = (part == 0 || timing) ? q : ctx->side_stream;
    const lt::Batch v = parts == 1 ? bt : sub_batch(bt, b0, n);
    lt::launch_prep_iter(v, jj, qs);
    if (lt::launch_inner_cluster(ctx->mg, ip, v, ctx->fe, ctx->ws.l0q + (size_t)b0 * ctx->N,
                                 ctx->ws.l0u ? ctx->ws.l0u + (size_t)b0 * ctx->N : nullptr,
                                 o.inner_cycles, qs, pf))
      return LT_ERR_CUDA;
    lt::launch_inner_record(v, qs);
    if (bt.block) {
      if (lt::launch_block_iteration(v, ctx->fe, qs, nlq, pf)) return LT_ERR_CUDA;
      *nlq += 2;
      continue;
    }
    lt::launch_arnoldi(v, ctx->fe, jj, qs, nlq, pf);
    lt::launch_shift_ls_only(v, jj, qs);
    *nlq += 4;
  }
  if (parts == 2) {
    CK(cudaEventRecord(ctx->ev_join, ctx->side_stream));
    CK(cudaStreamWaitEvent(q, ctx->ev_join, 0));
  }
  lt::launch_next_iter(bt, q);
  *nlq += 1;
  return LT_OK;
}

// parts of a decoupled cluster-resident solve (each its own counter slot, graph and stream; up to 8)
constexpr int kDecoupledParts = 4;

// One outer iteration of the bases [b0, b0 + n) on the cluster-resident path with iteration counter
// slot jslot: each half of a decoupled solve replays a graph of this on its own stream
static int launch_half_iteration(lt_ctx* ctx, cudaStream_t q, int b0, int n, int jslot, int* nlq) {
  const lt_opts& o = ctx->opts;
  const lt::Batch v = sub_batch(ctx->ws.bt, b0, n, jslot);
  lt::launch_prep_iter(v, 0, q);
  if (lt::launch_inner_cluster(ctx->mg, cluster_plan(ctx), v, ctx->fe, ctx->ws.l0q + (size_t)b0 * ctx->N,
                               ctx->ws.l0u ? ctx->ws.l0u + (size_t)b0 * ctx->N : nullptr, o.inner_cycles, q,
                               nullptr))
    return LT_ERR_CUDA;
  lt::launch_inner_record(v, q);
  lt::launch_arnoldi(v, ctx->fe, 0, q, nlq, nullptr);
  lt::launch_shift_ls(v, 0, q);   // the least squares, then this half's iteration counter
  *nlq += 5;
  return LT_OK;
}

// one outer iteration of every active basis (kernels read j from bt.jdev)
static int launch_iteration(lt_ctx* ctx, cudaStream_t q, int jj, int* nlq, lt::Prof* pf) {
  const lt_opts& o = ctx->opts;
  lt::Batch& bt = ctx->ws.bt;
  const lt::Level& L0 = ctx->mg.h_levels[0];
  if (uses_cluster_solve(ctx)) return launch_iteration_cluster(ctx, q, jj, nlq, pf);
  lt::launch_prep_iter(bt, jj, q);
  ++*nlq;
  for (int r = 0; r < o.inner_rounds; ++r) {
    lt::launch_exact_residual(bt, ctx->fe, L0, jj, r, 0, q, pf);
    ++*nlq;
    if (o.precond == 1 && r == 0) {   // first round: the residual is the Krylov vector v_j itself
      learned_guess(ctx->net, bt, L0, r, ctx->d_lk, ctx->d_mD, ctx->d_xin, ctx->d_gn2, q);
      *nlq += 24;
    }
    // the round's correction starts at zero (unless the learned guess seeded it), and each later
    // cycle follows the previous one's post-smoothing
    for (int cy = 0; cy < o.inner_cycles; ++cy)
      if (lt::launch_vcycle(ctx->mg, bt, r, q, nlq, pf, cy > 0 ? 0 : (o.precond == 1 && r == 0) ? -1 : 1))
        return LT_ERR_CUDA;
    lt::launch_update_u(bt, L0, jj, r, q);
    ++*nlq;
  }
  lt::launch_exact_residual(bt, ctx->fe, L0, jj, o.inner_rounds, 1, q, pf);
  lt::launch_inner_record(bt, q);
  *nlq += 2;
  if (bt.block) {
    if (lt::launch_block_iteration(bt, ctx->fe, q, nlq, pf)) return LT_ERR_CUDA;
    lt::launch_next_iter(bt, q);
    ++*nlq;
    return LT_OK;
  }
  lt::launch_arnoldi(bt, ctx->fe, jj, q, nlq, pf);
  lt::launch_shift_ls(bt, jj, q);
  *nlq += 2;
  return LT_OK;
}

// per-cell tables of the learned preconditioner's input channels (normalised log kappa, m / D) and
// the float32 diagonal D of the fine operator; built once per grid
static int learned_tables(lt_ctx* ctx) {
  if (ctx->d_lk) return LT_OK;
  std::vector<float> lk(ctx->N), mD(ctx->N), D(ctx->N);
  double mu = 0, var = 0;
  for (int64_t c = 0; c < ctx->N; ++c) mu += std::log(ctx->kappa[c]);
  mu /= ctx->N;
  for (int64_t c = 0; c < ctx->N; ++c) var += std::pow(std::log(ctx->kappa[c]) - mu, 2);
  double sd = std::sqrt(var / ctx->N);
  if (sd < 1e-12) sd = 1.0;
  for (int64_t c = 0; c < ctx->N; ++c) {
    lk[c] = (float)((std::log(ctx->kappa[c]) - mu) / sd);
    mD[c] = (float)(ctx->hl[0].m[c] / ctx->hl[0].D[c]);
    D[c] = (float)ctx->hl[0].D[c];
  }
  CK(cudaMalloc(&ctx->d_lk, ctx->N * sizeof(float)));
  CK(cudaMalloc(&ctx->d_mD, ctx->N * sizeof(float)));
  CK(cudaMalloc(&ctx->d_D32, ctx->N * sizeof(float)));
  CK(cudaMemcpy(ctx->d_lk, lk.data(), ctx->N * sizeof(float), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->d_mD, mD.data(), ctx->N * sizeof(float), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->d_D32, D.data(), ctx->N * sizeof(float), cudaMemcpyHostToDevice));
  return LT_OK;
}

static int solve_begin(lt_ctx* ctx, const Plan& P, SolveState& S, int* nl, bool decouple = false) {
  const lt_opts& o = ctx->opts;
  if (o.block && !P.block)
    return fail(ctx, LT_ERR_INVALID_ARG, "block = 1 applies to lt_forward and lt_forward_fields only");
  int rc = ensure_ws(ctx, P);
  if (rc) return rc;
  if (P.block) {
    if ((rc = ensure_block_ws(ctx, P))) return rc;
  } else {
    ctx->ws.bt.block = 0;
  }
  lt::Batch& bt = ctx->ws.bt;
  bt.nb = P.nb;
  bt.nsh = P.nsh;
  bt.tol = o.tol;
  double itol = o.inner_tol > 0 ? o.inner_tol : 0.01 * o.tol;
  // float32 solution vectors: the residual of a rounded u_j stalls near 2e-7 (relative), so
  // refinement rounds below that would not make progress
  if (o.precision == LT_PREC_FP32) itol = std::max(itol, 3e-7);
  bt.inner_tol2 = itol * itol;
  bt.inner_relax_max = o.inner_relax;
  bt.tma_polls = (unsigned)o.tma_wait_polls;
  bt.krylov = o.krylov;
  bt.stop_rule = o.stop_rule;
  bt.gs_passes = o.gram_schmidt;
  bt.nk = P.Nk;
  cudaStream_t s = ctx->stream;
  CK(cudaMemcpyAsync(const_cast<double*>(bt.wabs), P.wabs.data(), P.nsh * sizeof(double), cudaMemcpyHostToDevice, s));
  if (P.dense_b0 >= 0) {
    // dense right-hand side M phi_0 / beta0 (Sec. 3: the second system [b, M phi_0]), df32 split
    std::vector<float> hi(ctx->N), lo(ctx->N);
    for (int64_t c = 0; c < ctx->N; ++c) {
      const double x = ctx->hl[0].m[c] * ctx->phi0[c] / P.beta0;
      hi[c] = (float)x;
      lo[c] = (float)(x - (double)hi[c]);
    }
    CK(cudaMemcpyAsync(const_cast<float*>(bt.rhs_hi), hi.data(), ctx->N * sizeof(float), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(const_cast<float*>(bt.rhs_lo), lo.data(), ctx->N * sizeof(float), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));    // host vectors go out of scope
  }
  // tables
  std::vector<double2> taug(2 * P.G);
  for (int i = 0; i < 2 * P.G; ++i) taug[i] = make_double2(P.tau[i].real(), P.tau[i].imag());
  int pat_flex[5] = {0, 0, 0, 1, 1}, pat_single[5] = {0, 0, 0, 0, 0};
  std::vector<double2> zsh(P.nsh);
  for (int i = 0; i < P.nsh; ++i) zsh[i] = make_double2(P.zsh[i].real(), P.zsh[i].imag());
  CK(cudaMemcpyAsync(bt.tau_grp, taug.data(), taug.size() * sizeof(double2), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(bt.tau_pattern, o.tau_policy == LT_TAU_SINGLE ? pat_single : pat_flex, 5 * sizeof(int),
                     cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(bt.group, P.group.data(), P.nb * sizeof(int), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(bt.rhs_cell, P.rhs_cell.data(), P.nb * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(bt.shift_off, P.shift_off.data(), (P.nb + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(bt.zsh, zsh.data(), P.nsh * sizeof(double2), cudaMemcpyHostToDevice, s));
  bt.coarse_direct = ctx->mg.coarse_direct;
  if (ctx->mg.coarse_direct) {
    const HostLevel& Lc = ctx->hl.back();
    const size_t nc2 = (size_t)Lc.N * Lc.N;
    std::vector<float2> inv32(2 * P.G * nc2);
    for (int q = 0; q < 2 * P.G; ++q) {
      std::vector<cplx> inv;
      if (!dense_inverse(Lc, P.tau[q], inv)) return fail(ctx, LT_ERR_INVALID_ARG, "singular coarsest operator");
      for (size_t i = 0; i < nc2; ++i) inv32[q * nc2 + i] = make_float2((float)inv[i].real(), (float)inv[i].imag());
    }
    CK(cudaMemcpyAsync(bt.coarse_inv, inv32.data(), inv32.size() * sizeof(float2), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
  }
  CK(cudaMemsetAsync(bt.work, 0, lt::kWorkSlots * sizeof(unsigned long long), s));
  lt::Prof* pf = nullptr;
  if (o.timing_class >= 0) {
    const int cap = 16384;
    while ((int)ctx->prof_events.size() < 2 * cap) {
      cudaEvent_t e;
      CK(cudaEventCreate(&e));
      ctx->prof_events.push_back(e);
    }
    ctx->prof.cls = o.timing_class;
    ctx->prof.n = 0;
    ctx->prof.cap = cap;
    ctx->prof.ev = ctx->prof_events.data();
    pf = &ctx->prof;
  }
  lt::launch_init_batch(bt, s);
  *nl += 2;
  if (o.precond == 1) {
    if (!ctx->net) return fail(ctx, LT_ERR_STATE, "precond = 1 needs lt_set_learned_preconditioner");
    if (ctx->arena_base) return fail(ctx, LT_ERR_INVALID_ARG, "the learned preconditioner allocates; not available here");
    if (ctx->nz != 1 || ctx->nx % 8 || ctx->ny % 8)
      return fail(ctx, LT_ERR_INVALID_ARG, "the learned preconditioner needs a 2D grid with nx, ny multiples of 8");
    if (learned_prepare(ctx->net, P.nb, ctx->ny, ctx->nx)) return fail(ctx, LT_ERR_OOM, "network workspace");
    size_t need = (size_t)P.nb * ctx->N * 5;
    if (ctx->xin_cap < need) {
      if (ctx->d_xin) cudaFree(ctx->d_xin);
      if (ctx->d_gn2) cudaFree(ctx->d_gn2);
      CK(cudaMalloc(&ctx->d_xin, need * sizeof(float)));
      CK(cudaMalloc(&ctx->d_gn2, (size_t)P.nb * 64 * sizeof(float)));
      ctx->xin_cap = need;
    }
    if ((rc = learned_tables(ctx))) return rc;
    // every basis starts the solve with the network's guess switched on (int 0x01010101)
    CK(cudaMemsetAsync(ctx->d_gn2 + 4 * (size_t)P.nb, 0x01, (size_t)P.nb * sizeof(int), s));
  }
  S = SolveState();
  S.act.assign(P.nb, 1);
  S.pf = pf;
  // CUDA graph replay (not while timing individual launches, and not inside
  // lt_forward_noalloc, whose contract excludes any device allocation)
  S.use_graph = o.graphs && pf == nullptr && ctx->arena_base == nullptr;
  S.q = s;
  if (S.use_graph) {
    if (!ctx->cap_stream) CK(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
    if (!ctx->ev_a) CK(cudaEventCreateWithFlags(&ctx->ev_a, cudaEventDisableTiming));
    if (!ctx->ev_b) CK(cudaEventCreateWithFlags(&ctx->ev_b, cudaEventDisableTiming));
    S.q = ctx->cap_stream;
    CK(cudaEventRecord(ctx->ev_a, s));
    CK(cudaStreamWaitEvent(S.q, ctx->ev_a, 0));
    // Decoupled halves: with more bases than resident clusters, the two halves of the cluster-resident
    // path each get their own iteration counter, graph and stream, and run without a join per outer
    // iteration (one half's solves fill the clusters while the other half orthogonalises).
    if (decouple && uses_cluster_solve(ctx) && !bt.block && P.nb >= kDecoupledParts &&
        P.nb > cluster_plan(ctx).max_clusters) {
      S.nbr = kDecoupledParts;
      for (int h = 0; h < S.nbr; ++h) {
        if (h == 0) {
          S.bq[h] = ctx->cap_stream;
        } else {
          if (!ctx->part_stream[h - 1]) CK(cudaStreamCreateWithFlags(&ctx->part_stream[h - 1], cudaStreamNonBlocking));
          S.bq[h] = ctx->part_stream[h - 1];
          CK(cudaStreamWaitEvent(S.bq[h], ctx->ev_a, 0));
        }
        S.bb0[h] = (int)((int64_t)P.nb * h / S.nbr);
        S.bbn[h] = (int)((int64_t)P.nb * (h + 1) / S.nbr) - S.bb0[h];
      }
      for (int h = 0; h < S.nbr; ++h) {
        cudaGraph_t graph = nullptr;
        CK(cudaStreamBeginCapture(S.bq[h], cudaStreamCaptureModeThreadLocal));
        const int rc2 = launch_half_iteration(ctx, S.bq[h], S.bb0[h], S.bbn[h], h, &S.bper[h]);
        const cudaError_t ec = cudaStreamEndCapture(S.bq[h], &graph);
        if (rc2 || ec != cudaSuccess) {
          if (graph) cudaGraphDestroy(graph);
          return fail(ctx, LT_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(ec));
        }
        const cudaError_t ei = cudaGraphInstantiate(&S.bgx[h], graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) return fail(ctx, LT_ERR_CUDA, "graph instantiate failed: %s", cudaGetErrorString(ei));
      }
      return LT_OK;
    }
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(S.q, cudaStreamCaptureModeThreadLocal));
    int rc2 = launch_iteration(ctx, S.q, 0, &S.per_iter, nullptr);
    cudaError_t ec = cudaStreamEndCapture(S.q, &graph);
    if (rc2 || ec != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return fail(ctx, LT_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(ec));
    }
    ec = cudaGraphInstantiate(&S.gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (ec != cudaSuccess) return fail(ctx, LT_ERR_CUDA, "graph instantiate failed: %s", cudaGetErrorString(ec));
  }
  return LT_OK;
}

// enqueue up to n outer iterations (no host synchronisation)
static int solve_launch(lt_ctx* ctx, SolveState& S, int n, int* nl) {
  const lt_opts& o = ctx->opts;
  for (int k = 0; k < n && S.j < o.maxit && !S.done; ++k) {
    if (S.use_graph) {
      CK(cudaGraphLaunch(S.gexec, S.q));
      *nl += S.per_iter;
    } else if (launch_iteration(ctx, S.q, S.j, nl, S.pf)) {
      return fail(ctx, LT_ERR_CUDA, "kernel launch failed");
    }
    S.cycles += o.inner_rounds * o.inner_cycles;
    ++S.j;
  }
  CK(cudaGetLastError());
  return LT_OK;
}

// read the active flags (waits for the context's queued iterations)
static int solve_poll(lt_ctx* ctx, const Plan& P, SolveState& S) {
  CK(cudaMemcpyAsync(S.act.data(), ctx->ws.bt.active, P.nb * sizeof(int), cudaMemcpyDeviceToHost, S.q));
  CK(cudaStreamSynchronize(S.q));
  bool any = false;
  for (int b = 0; b < P.nb; ++b) any |= S.act[b] != 0;
  if (!any || S.j >= ctx->opts.maxit) S.done = true;
  return LT_OK;
}

// Which shifted systems count as solved.  Per-shift rule: the shift's true relative residual is at
// most tol (without true residuals: it stopped on its projected residual).  Quadrature rule: the
// shifts of one output time of a basis count together when their |w_k qhat(z_k)|-weighted true
// residual is at most tol times the sum of the weights.
static void converged_flags(const lt_ctx* ctx, const Plan& P, const std::vector<double>& tres, const int* conv,
                            std::vector<char>& ok) {
  const lt_opts& o = ctx->opts;
  ok.assign(P.nsh, 0);
  for (int i = 0; i < P.nsh; ++i) ok[i] = o.true_residual ? (tres[i] >= 0 && tres[i] <= o.tol) : (conv && conv[i] > 0);
  if (o.stop_rule != LT_STOP_QUADRATURE || !o.true_residual) return;
  for (int b = 0; b < P.nb; ++b)
    for (int t0 = P.shift_off[b]; t0 < P.shift_off[b + 1]; t0 += P.Nk) {
      double num = 0.0, den = 0.0;
      for (int i = t0; i < t0 + P.Nk; ++i) {
        num += P.wabs[i] * (tres[i] >= 0 ? tres[i] : INFINITY);
        den += P.wabs[i];
      }
      const char v = num <= o.tol * den;
      for (int i = t0; i < t0 + P.Nk; ++i) ok[i] = v;
    }
}

static int solve_end(lt_ctx* ctx, const Plan& P, SolveState& S, std::vector<double>& true_res, lt_stats* st,
                     int* nl, bool need_x) {
  const lt_opts& o = ctx->opts;
  lt::Batch& bt = ctx->ws.bt;
  cudaStream_t s = ctx->stream;
  lt::Prof* pf = S.pf;
  int rc = LT_OK;
  const int cycles = S.cycles;
  if (S.nbr) {
    for (int h = 0; h < S.nbr; ++h) {
      CK(cudaEventRecord(ctx->ev_b, S.bq[h]));
      CK(cudaStreamWaitEvent(s, ctx->ev_b, 0));
      cudaGraphExecDestroy(S.bgx[h]);
      S.bgx[h] = nullptr;
    }
  } else if (S.use_graph) {
    CK(cudaEventRecord(ctx->ev_b, S.q));
    CK(cudaStreamWaitEvent(s, ctx->ev_b, 0));
    cudaGraphExecDestroy(S.gexec);
    S.gexec = nullptr;
  }
  std::vector<void*> tmp;
  true_res.assign(P.nsh, -1.0);
  if (S.tail_done) {   // queued by the parts as they finished: only the true residuals to read back
    if (o.true_residual)
      CK(cudaMemcpyAsync(true_res.data(), S.d_res2, P.nsh * sizeof(double), cudaMemcpyDeviceToHost, s));
  } else {
  // y per shift
  int* d_shb = nullptr;
  if ((rc = scratch(ctx, kScrShb, &d_shb, P.nsh))) return rc;
  CK(cudaMemcpyAsync(d_shb, P.sh_basis.data(), P.nsh * sizeof(int), cudaMemcpyHostToDevice, s));
  if (bt.block) lt::launch_block_backsolve(bt, d_shb, s);
  else lt::launch_backsolve_map(bt, d_shb, s);
  ++*nl;
  if (o.true_residual || need_x) {
    Workspace& ws = ctx->ws;
    size_t need = (size_t)P.nsh * ctx->N;
    if (ws.x_elems < need) {
      // X buffers live in the workspace list
      if ((rc = dalloc(ctx, ws.allocs, &ws.X_hi, need))) { free_list(tmp); return rc; }
      ws.X_lo = nullptr;
      if (o.precision == LT_PREC_FP64 && (rc = dalloc(ctx, ws.allocs, &ws.X_lo, need))) { free_list(tmp); return rc; }
      ws.x_elems = need;
    }
    if (bt.block) lt::launch_block_xk(bt, ws.X_hi, ws.X_lo, s, pf);
    else lt::launch_xk(bt, ws.X_hi, ws.X_lo, s, pf);
    ++*nl;
    if (o.true_residual) {
      double* d_res2 = nullptr;
      if ((rc = scratch(ctx, kScrRes2, &d_res2, P.nsh))) { free_list(tmp); return rc; }
      CK(cudaMemsetAsync(d_res2, 0, P.nsh * sizeof(double), s));
      lt::launch_true_res(bt, ctx->fe, d_shb, ws.X_hi, ws.X_lo, d_res2, s, pf);
      ++*nl;
      CK(cudaMemcpyAsync(true_res.data(), d_res2, P.nsh * sizeof(double), cudaMemcpyDeviceToHost, s));
    }
  }
  }
  // stats
  std::vector<int> nit(P.nb), conv(P.nsh);
  std::vector<double> pres(P.nsh), inner(P.nb);
  CK(cudaMemcpyAsync(nit.data(), bt.nit, P.nb * sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(conv.data(), bt.conv_it, P.nsh * sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(pres.data(), bt.pres, P.nsh * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(inner.data(), bt.inner_max, P.nb * sizeof(double), cudaMemcpyDeviceToHost, s));
  unsigned long long work[lt::kWorkSlots];
  CK(cudaMemcpyAsync(work, bt.work, sizeof(work), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  free_list(tmp);
  for (auto& r : true_res)
    if (r >= 0) r = std::sqrt(r);
  if (work[lt::kTimeoutSlot] > 0)
    return fail(ctx, LT_ERR_TIMEOUT, "a bulk tensor copy did not complete within its bounded wait (%llu tiles)",
                (unsigned long long)work[lt::kTimeoutSlot]);
  if (st) {
    for (int c = 0; c < LT_KC_COUNT; ++c) st->work[c] += work[c];
    if (pf) {
      float tot = 0.f;
      for (int q = 0; q < pf->n; ++q) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, pf->ev[2 * q], pf->ev[2 * q + 1]);
        tot += ms;
      }
      st->timed_ms += tot;
      st->timed_launches += pf->n;
    }
    st->n_bases += P.nb;
    st->n_shift_solves += P.nsh;
    int conv_count = 0;
    std::vector<char> okv;
    converged_flags(ctx, P, true_res, conv.data(), okv);
    for (int i = 0; i < P.nsh; ++i) {
      conv_count += okv[i];
      st->max_proj_residual = std::max(st->max_proj_residual, pres[i]);
      if (o.true_residual) st->max_true_residual = std::max(st->max_true_residual, true_res[i]);
    }
    st->n_converged += conv_count;
    for (int b = 0; b < P.nb; ++b) {
      st->outer_iters_max = std::max(st->outer_iters_max, nit[b]);
      st->outer_iters_sum += nit[b];
      st->max_inner_residual = std::max(st->max_inner_residual, inner[b]);
    }
    st->inner_cycles_total += cycles;
  }
  ctx->last_group = P.group;
  ctx->last_nit = nit;
  ctx->last_tau = P.tau;
  ctx->last_single = o.tau_policy == LT_TAU_SINGLE;
  return LT_OK;
}

// The buffers of the end-of-solve work, set up on the context stream before the decoupled parts
// finish (each part then queues its own y_k, x_k and true residuals on its stream)
static int prepare_tail(lt_ctx* ctx, const Plan& P, SolveState& S, bool need_x) {
  const lt_opts& o = ctx->opts;
  Workspace& ws = ctx->ws;
  cudaStream_t s = ctx->stream;
  int rc = LT_OK;
  if ((rc = scratch(ctx, kScrShb, &S.d_shb, P.nsh))) return rc;
  CK(cudaMemcpyAsync(S.d_shb, P.sh_basis.data(), P.nsh * sizeof(int), cudaMemcpyHostToDevice, s));
  S.tail_x = o.true_residual || need_x;
  if (S.tail_x) {
    const size_t need = (size_t)P.nsh * ctx->N;
    if (ws.x_elems < need) {
      if ((rc = dalloc(ctx, ws.allocs, &ws.X_hi, need))) return rc;
      ws.X_lo = nullptr;
      if (o.precision == LT_PREC_FP64 && (rc = dalloc(ctx, ws.allocs, &ws.X_lo, need))) return rc;
      ws.x_elems = need;
    }
  }
  if (o.true_residual) {
    if ((rc = scratch(ctx, kScrRes2, &S.d_res2, P.nsh))) return rc;
    CK(cudaMemsetAsync(S.d_res2, 0, P.nsh * sizeof(double), s));
  }
  if (!ctx->ev_tail) CK(cudaEventCreateWithFlags(&ctx->ev_tail, cudaEventDisableTiming));
  CK(cudaEventRecord(ctx->ev_tail, s));
  return LT_OK;
}

// y_k, x_k and the true residuals of part h's shifts, on its stream, once the part has finished
static int launch_part_tail(lt_ctx* ctx, const Plan& P, SolveState& S, int h, int* nl) {
  const lt_opts& o = ctx->opts;
  const lt::Batch& bt = ctx->ws.bt;
  Workspace& ws = ctx->ws;
  cudaStream_t q = S.bq[h];
  const int s0 = P.shift_off[S.bb0[h]], s1 = P.shift_off[S.bb0[h] + S.bbn[h]];
  CK(cudaStreamWaitEvent(q, ctx->ev_tail, 0));
  lt::launch_backsolve_map(bt, S.d_shb, q, s0, s1);
  ++*nl;
  if (S.tail_x) {
    lt::launch_xk(sub_batch(bt, S.bb0[h], S.bbn[h], h), ws.X_hi, ws.X_lo, q, nullptr);
    ++*nl;
  }
  if (o.true_residual) {
    lt::launch_true_res(bt, ctx->fe, S.d_shb, ws.X_hi, ws.X_lo, S.d_res2, q, nullptr, s0, s1);
    ++*nl;
  }
  CK(cudaGetLastError());
  return LT_OK;
}

static int run_solves(lt_ctx* ctx, const Plan& P, std::vector<double>& true_res, lt_stats* st, int* nl,
                      bool need_x = false) {
  SolveState S;
  int rc = solve_begin(ctx, P, S, nl, true);
  if (rc) return rc;
  if (S.nbr) {
    // decoupled parts: fill every part's queue, then refill each part as soon as its own queue drains
    // (only that part's stream is waited on, so the others keep running); a finished part queues its
    // own end-of-solve work at once, next to the parts still iterating
    const lt_opts& o = ctx->opts;
    if ((rc = prepare_tail(ctx, P, S, need_x))) return rc;
    auto enqueue = [&](int h) -> int {
      for (int k = 0; k < o.check_every && S.bj[h] < o.maxit; ++k) {
        if (cudaGraphLaunch(S.bgx[h], S.bq[h]) != cudaSuccess) return fail(ctx, LT_ERR_CUDA, "graph launch failed");
        *nl += S.bper[h];
        if (h == 0) S.cycles += o.inner_rounds * o.inner_cycles;   // (per outer iteration, as joined)
        ++S.bj[h];
      }
      return LT_OK;
    };
    for (int h = 0; h < S.nbr; ++h)
      if ((rc = enqueue(h))) return rc;
    auto all_done = [&]() {
      for (int h = 0; h < S.nbr; ++h)
        if (!S.bdone[h]) return false;
      return true;
    };
    while (!all_done()) {
      for (int h = 0; h < S.nbr; ++h) {
        if (S.bdone[h]) continue;
        CK(cudaMemcpyAsync(S.act.data() + S.bb0[h], ctx->ws.bt.active + S.bb0[h], S.bbn[h] * sizeof(int),
                           cudaMemcpyDeviceToHost, S.bq[h]));
        CK(cudaStreamSynchronize(S.bq[h]));
        bool any = false;
        for (int b = S.bb0[h]; b < S.bb0[h] + S.bbn[h]; ++b) any |= S.act[b] != 0;
        if (!any || S.bj[h] >= o.maxit) {
          S.bdone[h] = true;
          if ((rc = launch_part_tail(ctx, P, S, h, nl))) return rc;
        } else if ((rc = enqueue(h))) {
          return rc;
        }
      }
    }
    for (int h = 0; h < S.nbr; ++h) S.j = std::max(S.j, S.bj[h]);
    S.done = true;
    S.tail_done = true;
  }
  while (!S.done) {
    if ((rc = solve_launch(ctx, S, ctx->opts.check_every, nl))) return rc;
    if ((rc = solve_poll(ctx, P, S))) return rc;
  }
  return solve_end(ctx, P, S, true_res, st, nl, need_x);
}

static void stats_reset(lt_stats* st, bool tr) {
  if (!st) return;
  memset(st, 0, sizeof(*st));
  st->max_true_residual = tr ? 0.0 : -1.0;
}

static int check_times(lt_ctx* ctx, int nt, const double* times) {
  if (!ctx->have_grid) return fail(ctx, LT_ERR_STATE, "lt_setup_grid must come first");
  if (nt < 1 || !times) return fail(ctx, LT_ERR_INVALID_ARG, "nt=%d must be >= 1", nt);
  for (int t = 0; t < nt; ++t)
    if (!(times[t] > 0.0) || !std::isfinite(times[t]))
      return fail(ctx, LT_ERR_INVALID_ARG, "times[%d]=%g must be positive and finite", t, times[t]);
  return LT_OK;
}

// forward driver shared by lt_forward and lt_forward_fields
static int forward_finish(lt_ctx* ctx, const Plan& P, const std::vector<double>& tres, double* out, int on_device,
                          int fields, lt_stats* st, int nl);

static int forward_impl(lt_ctx* ctx, int nt, const double* times, double* out, int on_device, int fields,
                        lt_stats* st) {
  if (!ctx) return LT_ERR_INVALID_ARG;
  int rc = check_times(ctx, nt, times);
  if (rc) return rc;
  if (ctx->src.empty()) return fail(ctx, LT_ERR_STATE, "no sources set");
  if (!fields && ctx->rec.empty()) return fail(ctx, LT_ERR_STATE, "no receivers set");
  if (!out) return fail(ctx, LT_ERR_INVALID_ARG, "output pointer is null");
  CK(cudaSetDevice(ctx->device));
  stats_reset(st, ctx->opts.true_residual);
  Plan P;
  make_plan(ctx, nt, times, ctx->src, P, (int)ctx->src.size(), !ctx->phi0.empty());
  if (ctx->opts.block) {
    if (ctx->arena_base) return fail(ctx, LT_ERR_INVALID_ARG, "lt_forward_noalloc does not support block = 1");
    if (ctx->src.size() > 16) return fail(ctx, LT_ERR_INVALID_ARG, "block = 1 takes at most 16 sources");
    if (!ctx->phi0.empty()) return fail(ctx, LT_ERR_INVALID_ARG, "block = 1 does not take an initial state");
    for (size_t a = 0; a < ctx->src.size(); ++a)
      for (size_t b = 0; b < a; ++b)
        if (ctx->src[a] == ctx->src[b])
          return fail(ctx, LT_ERR_INVALID_ARG, "block = 1 needs sources in distinct cells (%zu and %zu share one)", b, a);
    P.block = true;
  }
  int nl = 0;
  CK(cudaEventRecord(ctx->ev0, ctx->stream));
  std::vector<double> tres;
  rc = run_solves(ctx, P, tres, st, &nl);
  if (rc) return rc;
  return forward_finish(ctx, P, tres, out, on_device, fields, st, nl);
}

// quadrature-fused measurements (or fields) after the solves of a forward plan
static int forward_finish(lt_ctx* ctx, const Plan& P, const std::vector<double>& tres, double* out, int on_device,
                          int fields, lt_stats* st, int nl) {
  int rc = LT_OK;
  const int nt = P.nt;
  const int ns = (int)ctx->src.size(), nr = (int)ctx->rec.size();
  cudaStream_t s = ctx->stream;
  // quadrature items (s, t) and weights w_k qhat_s(z_k); with an initial state, items
  // (dense, t) with weights beta0 w_k (its basis solves for M phi_0 / beta0)
  const int dense_q0 = P.dense_b0 >= 0 ? ns * nt : -1;
  std::vector<lt::QuadItem> items(ns * nt + (dense_q0 >= 0 ? nt : 0));
  std::vector<double2> wq(P.nsh);
  for (int si = 0; si < ns; ++si)
    for (int t = 0; t < nt; ++t) {
      int b = si * P.G + P.tgroup[t];
      int sh0 = shift_of(P, b, t);
      items[si * nt + t] = {b, sh0, P.Nk};
      for (int k = 0; k < P.Nk; ++k) {
        cplx v = P.w[t][k] * qhat(ctx, si, P.z[t][k]);
        wq[sh0 + k] = make_double2(v.real(), v.imag());
      }
    }
  if (dense_q0 >= 0)
    for (int t = 0; t < nt; ++t) {
      int b = P.dense_b0 + P.tgroup[t];
      int sh0 = shift_of(P, b, t);
      items[dense_q0 + t] = {b, sh0, P.Nk};
      for (int k = 0; k < P.Nk; ++k) {
        cplx v = P.w[t][k] * P.beta0;
        wq[sh0 + k] = make_double2(v.real(), v.imag());
      }
    }
  std::vector<void*> tmp;
  lt::QuadItem* d_items;
  double2 *d_wq, *d_C;
  int64_t* d_rc;
  double* d_out = nullptr;
  const size_t out_n = fields ? (size_t)ns * nt * ctx->N : (size_t)ns * nr * nt;
  if ((rc = scratch(ctx, kScrItems, &d_items, items.size())) || (rc = scratch(ctx, kScrWq, &d_wq, wq.size())) ||
      (rc = scratch(ctx, kScrC, &d_C, items.size() * (P.block ? (size_t)ctx->ws.bt.bld : (size_t)ctx->opts.maxit))) ||
      (rc = scratch(ctx, kScrRc, &d_rc, std::max(nr, 1)))) {
    free_list(tmp);
    return rc;
  }
  if (on_device) d_out = out;
  else if ((rc = scratch(ctx, kScrOut, &d_out, out_n))) { free_list(tmp); return rc; }
  CK(cudaMemcpyAsync(d_items, items.data(), items.size() * sizeof(lt::QuadItem), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(d_wq, wq.data(), wq.size() * sizeof(double2), cudaMemcpyHostToDevice, s));
  if (nr) CK(cudaMemcpyAsync(d_rc, ctx->rec.data(), nr * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  if (P.block) {
    lt::launch_block_quad(ctx->ws.bt, d_items, (int)items.size(), d_wq, d_C, ns, nr, nt, d_rc, d_out, fields, s);
  } else {
    lt::launch_quad_coef(ctx->ws.bt, d_items, (int)items.size(), d_wq, d_C, s);
    if (fields) lt::launch_fields(ctx->ws.bt, d_items, d_C, ns * nt, d_out, s, nt, dense_q0);
    else lt::launch_measure(ctx->ws.bt, d_items, d_C, ns, nr, nt, d_rc, d_out, s, dense_q0);
  }
  nl += 2;
  CK(cudaGetLastError());
  CK(cudaEventRecord(ctx->ev1, s));
  if (!on_device) CK(cudaMemcpyAsync(out, d_out, out_n * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  free_list(tmp);
  if (st) {
    cudaEventElapsedTime(&st->ms_total, ctx->ev0, ctx->ev1);
    st->kernel_launches = nl;
  }
  if (ctx->opts.true_residual) {
    std::vector<char> ok;
    converged_flags(ctx, P, tres, nullptr, ok);
    for (char c : ok)
      if (!c) return fail(ctx, LT_ERR_NOT_CONVERGED, "some shifted systems did not reach tol");
  }
  return LT_OK;
}

extern "C" int lt_forward(lt_ctx* ctx, int nt, const double* times, double* h, int h_on_device, lt_stats* st) {
  return forward_impl(ctx, nt, times, h, h_on_device, 0, st);
}

extern "C" int lt_forward_fields(lt_ctx* ctx, int nt, const double* times, double* phi, int on_device,
                                 lt_stats* st) {
  return forward_impl(ctx, nt, times, phi, on_device, 1, st);
}

// Forward solves of several independent contexts (one aquifer each) driven
// together: every context replays its outer-iteration graph on its own
// non-blocking stream, and the host enqueues a slab of iterations for every
// unfinished context before it polls any of them, so the GPU overlaps the
// aquifers' latency-bound kernel chains.
extern "C" int lt_forward_batch(int n, lt_ctx* const* ctxs, const int* nt, const double* const* times,
                                double* const* h, int h_on_device, lt_stats* stats) {
  if (n < 1 || !ctxs || !nt || !times || !h) return LT_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i) {
    lt_ctx* ctx = ctxs[i];
    if (!ctx) return LT_ERR_INVALID_ARG;
    for (int k = 0; k < i; ++k)
      if (ctxs[k] == ctx) return fail(ctx, LT_ERR_INVALID_ARG, "context %d appears twice in the batch", i);
    int rc = check_times(ctx, nt[i], times[i]);
    if (rc) return rc;
    if (ctx->src.empty() || ctx->rec.empty()) return fail(ctx, LT_ERR_STATE, "context %d: sources and receivers must be set", i);
    if (!h[i]) return fail(ctx, LT_ERR_INVALID_ARG, "context %d: output pointer is null", i);
  }
  std::vector<Plan> P(n);
  std::vector<SolveState> S(n);
  std::vector<int> nl(n, 0);
  for (int i = 0; i < n; ++i) {
    lt_ctx* ctx = ctxs[i];
    CK(cudaSetDevice(ctx->device));
    stats_reset(stats ? &stats[i] : nullptr, ctx->opts.true_residual);
    make_plan(ctx, nt[i], times[i], ctx->src, P[i], (int)ctx->src.size(), !ctx->phi0.empty());
    CK(cudaEventRecord(ctx->ev0, ctx->stream));
    int rc = solve_begin(ctx, P[i], S[i], &nl[i]);
    if (rc) return rc;
  }
  for (;;) {
    bool any = false;
    for (int i = 0; i < n; ++i) {
      if (S[i].done) continue;
      lt_ctx* ctx = ctxs[i];
      CK(cudaSetDevice(ctx->device));
      int rc = solve_launch(ctx, S[i], ctx->opts.check_every, &nl[i]);
      if (rc) return rc;
      any = true;
    }
    if (!any) break;
    for (int i = 0; i < n; ++i) {
      if (S[i].done) continue;
      lt_ctx* ctx = ctxs[i];
      CK(cudaSetDevice(ctx->device));
      int rc = solve_poll(ctx, P[i], S[i]);
      if (rc) return rc;
    }
  }
  int worst = LT_OK;
  for (int i = 0; i < n; ++i) {
    lt_ctx* ctx = ctxs[i];
    CK(cudaSetDevice(ctx->device));
    std::vector<double> tres;
    lt_stats* st = stats ? &stats[i] : nullptr;
    int rc = solve_end(ctx, P[i], S[i], tres, st, &nl[i], false);
    if (rc) return rc;
    rc = forward_finish(ctx, P[i], tres, h[i], h_on_device, 0, st, nl[i]);
    if (rc == LT_ERR_NOT_CONVERGED) worst = rc;
    else if (rc) return rc;
  }
  return worst;
}

// Adjoint path (Sec. 5.2): one batch of bases for the sources and the
// receivers, solutions per shift, then the sensitivity assembly (mode 0: J,
// mode 1: vector-Jacobian product).  h (optional) = forward measurements.
static int adjoint_check(lt_ctx* ctx, int nt, const double* times, double* J, const double* g, double* grad,
                         int mode) {
  if (!ctx) return LT_ERR_INVALID_ARG;
  int rc = check_times(ctx, nt, times);
  if (rc) return rc;
  if (ctx->src.empty() || ctx->rec.empty()) return fail(ctx, LT_ERR_STATE, "sources and receivers must be set");
  if (mode == 0 && !J) return fail(ctx, LT_ERR_INVALID_ARG, "J is null");
  if (mode == 1 && (!g || !grad)) return fail(ctx, LT_ERR_INVALID_ARG, "g and grad are required");
  if (!ctx->phi0.empty())
    return fail(ctx, LT_ERR_STATE, "the adjoint Jacobian is implemented for phi_0 = 0; clear the initial state "
                                   "(lt_set_initial_state(ctx, NULL))");
  return LT_OK;
}

// the adjoint plan: one basis per (source or receiver, time group)
static void adjoint_plan(lt_ctx* ctx, int nt, const double* times, Plan& P) {
  std::vector<int64_t> rhs(ctx->src);
  rhs.insert(rhs.end(), ctx->rec.begin(), ctx->rec.end());
  make_plan(ctx, nt, times, rhs, P, (int)ctx->src.size(), false);
}

static int adjoint_finish(lt_ctx* ctx, const Plan& P, const std::vector<double>& tres, double* J, const double* g,
                          double* grad, double* h, int on_device, int mode, lt_stats* st, int nl);

static int adjoint_impl(lt_ctx* ctx, int nt, const double* times, double* J, const double* g, double* grad,
                        double* h, int on_device, int mode, lt_stats* st) {
  int rc = adjoint_check(ctx, nt, times, J, g, grad, mode);
  if (rc) return rc;
  CK(cudaSetDevice(ctx->device));
  stats_reset(st, ctx->opts.true_residual);
  Plan P;
  adjoint_plan(ctx, nt, times, P);
  int nl = 0;
  CK(cudaEventRecord(ctx->ev0, ctx->stream));
  std::vector<double> tres;
  rc = run_solves(ctx, P, tres, st, &nl, true);
  if (rc) return rc;
  return adjoint_finish(ctx, P, tres, J, g, grad, h, on_device, mode, st, nl);
}

// sensitivity assembly (J or the VJP) and the measurements, after the solves of an adjoint plan
static int adjoint_finish(lt_ctx* ctx, const Plan& P, const std::vector<double>& tres, double* J, const double* g,
                          double* grad, double* h, int on_device, int mode, lt_stats* st, int nl) {
  int rc = LT_OK;
  const int ns = (int)ctx->src.size(), nr = (int)ctx->rec.size(), nt = P.nt;
  cudaStream_t s = ctx->stream;
  const int Nk = P.Nk;
  std::vector<int> sh_src(nt * ns), sh_rec(nt * nr);
  std::vector<double2> omega((size_t)nt * ns * Nk), zk((size_t)nt * Nk);
  for (int t = 0; t < nt; ++t) {
    for (int si = 0; si < ns; ++si) {
      sh_src[t * ns + si] = shift_of(P, si * P.G + P.tgroup[t], t);
      for (int k = 0; k < Nk; ++k) {
        cplx v = P.w[t][k] * qhat(ctx, si, P.z[t][k]);
        omega[((size_t)t * ns + si) * Nk + k] = make_double2(v.real(), v.imag());
      }
    }
    for (int r = 0; r < nr; ++r) sh_rec[t * nr + r] = shift_of(P, (ns + r) * P.G + P.tgroup[t], t);
    for (int k = 0; k < Nk; ++k) zk[t * Nk + k] = make_double2(P.z[t][k].real(), P.z[t][k].imag());
  }
  std::vector<void*> tmp;
  int *d_ss, *d_sr;
  double2 *d_om, *d_zk;
  double *d_g = nullptr, *d_grad = nullptr, *d_h = nullptr;
  if ((rc = dalloc(ctx, tmp, &d_ss, sh_src.size())) || (rc = dalloc(ctx, tmp, &d_sr, sh_rec.size())) ||
      (rc = dalloc(ctx, tmp, &d_om, omega.size())) || (rc = dalloc(ctx, tmp, &d_zk, zk.size()))) {
    free_list(tmp);
    return rc;
  }
  CK(cudaMemcpyAsync(d_ss, sh_src.data(), sh_src.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(d_sr, sh_rec.data(), sh_rec.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(d_om, omega.data(), omega.size() * sizeof(double2), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(d_zk, zk.data(), zk.size() * sizeof(double2), cudaMemcpyHostToDevice, s));
  const size_t nrow = (size_t)ns * nr * nt;
  if (mode == 1) {
    if (on_device) {
      d_g = const_cast<double*>(g);
      d_grad = grad;
    } else {
      if ((rc = dalloc(ctx, tmp, &d_g, nrow)) || (rc = dalloc(ctx, tmp, &d_grad, 2 * (size_t)ctx->N))) {
        free_list(tmp);
        return rc;
      }
      CK(cudaMemcpyAsync(d_g, g, nrow * sizeof(double), cudaMemcpyHostToDevice, s));
    }
    CK(cudaMemsetAsync(d_grad, 0, 2 * (size_t)ctx->N * sizeof(double), s));
  }
  lt::SensLaunch L;
  L.ns = ns; L.nr = nr; L.nt = nt; L.Nk = Nk; L.N = ctx->N;
  L.nx = ctx->nx; L.ny = ctx->ny; L.nz = ctx->nz;
  L.sh_src = d_ss; L.sh_rec = d_sr; L.omega = d_om; L.zk = d_zk;
  L.X_hi = ctx->ws.X_hi; L.X_lo = ctx->ws.X_lo;
  L.Te = ctx->g_Te; L.Tn = ctx->g_Tn; L.Tu = ctx->g_Tu; L.kap = ctx->g_kap; L.Bd = ctx->g_Bd; L.m = ctx->g_m;
  L.J = J; L.g = d_g; L.grad = d_grad; L.mode = mode;
  if (lt::launch_sens2(L, s)) {
    free_list(tmp);
    return fail(ctx, LT_ERR_INVALID_ARG, "sensitivity launch failed (too many sources/receivers for shared memory?)");
  }
  ++nl;
  if (h) {   // forward measurements from the source bases
    std::vector<lt::QuadItem> items(ns * nt);
    std::vector<double2> wq(P.nsh, make_double2(0.0, 0.0));
    for (int si = 0; si < ns; ++si)
      for (int t = 0; t < nt; ++t) {
        int b = si * P.G + P.tgroup[t];
        int sh0 = shift_of(P, b, t);
        items[si * nt + t] = {b, sh0, Nk};
        for (int k = 0; k < Nk; ++k) wq[sh0 + k] = omega[((size_t)t * ns + si) * Nk + k];
      }
    lt::QuadItem* d_items;
    double2 *d_wq, *d_C;
    int64_t* d_rc;
    if ((rc = dalloc(ctx, tmp, &d_items, items.size())) || (rc = dalloc(ctx, tmp, &d_wq, wq.size())) ||
        (rc = dalloc(ctx, tmp, &d_C, items.size() * ctx->opts.maxit)) || (rc = dalloc(ctx, tmp, &d_rc, nr))) {
      free_list(tmp);
      return rc;
    }
    if (on_device) d_h = h;
    else if ((rc = dalloc(ctx, tmp, &d_h, nrow))) { free_list(tmp); return rc; }
    CK(cudaMemcpyAsync(d_items, items.data(), items.size() * sizeof(lt::QuadItem), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(d_wq, wq.data(), wq.size() * sizeof(double2), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(d_rc, ctx->rec.data(), nr * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    lt::launch_quad_coef(ctx->ws.bt, d_items, (int)items.size(), d_wq, d_C, s);
    lt::launch_measure(ctx->ws.bt, d_items, d_C, ns, nr, nt, d_rc, d_h, s);
    nl += 2;
  }
  CK(cudaGetLastError());
  CK(cudaEventRecord(ctx->ev1, s));
  if (mode == 1 && !on_device) CK(cudaMemcpyAsync(grad, d_grad, 2 * (size_t)ctx->N * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (h && !on_device) CK(cudaMemcpyAsync(h, d_h, nrow * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  free_list(tmp);
  if (st) {
    cudaEventElapsedTime(&st->ms_total, ctx->ev0, ctx->ev1);
    st->kernel_launches = nl;
  }
  if (ctx->opts.true_residual) {
    std::vector<char> ok;
    converged_flags(ctx, P, tres, nullptr, ok);
    for (char c : ok)
      if (!c) return fail(ctx, LT_ERR_NOT_CONVERGED, "some shifted systems did not reach tol");
  }
  return LT_OK;
}

extern "C" int lt_adjoint_batch(int n, lt_ctx* const* ctxs, const int* nt, const double* const* times,
                                double* const* J, const double* const* g, double* const* grad, double* const* h,
                                lt_stats* stats) {
  if (n < 1 || !ctxs || !nt || !times) return LT_ERR_INVALID_ARG;
  std::vector<int> mode(n);
  for (int i = 0; i < n; ++i) {
    lt_ctx* ctx = ctxs[i];
    if (!ctx) return LT_ERR_INVALID_ARG;
    for (int k = 0; k < i; ++k)
      if (ctxs[k] == ctx) return fail(ctx, LT_ERR_INVALID_ARG, "context %d appears twice in the batch", i);
    mode[i] = (J && J[i]) ? 0 : 1;
    int rc = adjoint_check(ctx, nt[i], times[i], J ? J[i] : nullptr, g ? g[i] : nullptr, grad ? grad[i] : nullptr,
                           mode[i]);
    if (rc) return rc;
  }
  std::vector<Plan> P(n);
  std::vector<SolveState> S(n);
  std::vector<int> nl(n, 0);
  for (int i = 0; i < n; ++i) {
    lt_ctx* ctx = ctxs[i];
    CK(cudaSetDevice(ctx->device));
    stats_reset(stats ? &stats[i] : nullptr, ctx->opts.true_residual);
    adjoint_plan(ctx, nt[i], times[i], P[i]);
    CK(cudaEventRecord(ctx->ev0, ctx->stream));
    int rc = solve_begin(ctx, P[i], S[i], &nl[i]);
    if (rc) return rc;
  }
  for (;;) {
    bool any = false;
    for (int i = 0; i < n; ++i) {
      if (S[i].done) continue;
      lt_ctx* ctx = ctxs[i];
      CK(cudaSetDevice(ctx->device));
      int rc = solve_launch(ctx, S[i], ctx->opts.check_every, &nl[i]);
      if (rc) return rc;
      any = true;
    }
    if (!any) break;
    for (int i = 0; i < n; ++i) {
      if (S[i].done) continue;
      lt_ctx* ctx = ctxs[i];
      CK(cudaSetDevice(ctx->device));
      int rc = solve_poll(ctx, P[i], S[i]);
      if (rc) return rc;
    }
  }
  int worst = LT_OK;
  for (int i = 0; i < n; ++i) {
    lt_ctx* ctx = ctxs[i];
    CK(cudaSetDevice(ctx->device));
    std::vector<double> tres;
    lt_stats* st = stats ? &stats[i] : nullptr;
    int rc = solve_end(ctx, P[i], S[i], tres, st, &nl[i], true);
    if (rc) return rc;
    rc = adjoint_finish(ctx, P[i], tres, mode[i] == 0 ? J[i] : nullptr, mode[i] == 1 ? g[i] : nullptr,
                        mode[i] == 1 ? grad[i] : nullptr, h ? h[i] : nullptr, 1, mode[i], st, nl[i]);
    if (rc == LT_ERR_NOT_CONVERGED) worst = rc;
    else if (rc) return rc;
  }
  return worst;
}

extern "C" int lt_adjoint_jacobian(lt_ctx* ctx, int nt, const double* times, double* J, lt_stats* st) {
  return adjoint_impl(ctx, nt, times, J, nullptr, nullptr, nullptr, 1, 0, st);
}

extern "C" int lt_adjoint_vjp(lt_ctx* ctx, int nt, const double* times, const double* g, double* grad, double* h,
                              int on_device, lt_stats* st) {
  return adjoint_impl(ctx, nt, times, nullptr, g, grad, h, on_device, 1, st);
}

// ------------------------------------------------------------------ preconditioner apply (training pairs)
extern "C" int lt_set_learned_preconditioner(lt_ctx* ctx, lt_unet* net) {
  if (!ctx) return LT_ERR_INVALID_ARG;
  ctx->net = net;
  return LT_OK;
}

extern "C" int lt_precond_apply(lt_ctx* ctx, int nimg, const double* tau, const float* r, float* e, int cycles) {
  if (!ctx) return LT_ERR_INVALID_ARG;
  if (!ctx->have_grid) return fail(ctx, LT_ERR_STATE, "lt_setup_grid must come first");
  if (nimg < 1 || nimg > 4096 || !tau || !r || !e || cycles < 1 || cycles > 1000)
    return fail(ctx, LT_ERR_INVALID_ARG, "bad lt_precond_apply arguments");
  CK(cudaSetDevice(ctx->device));
  cudaStream_t s = ctx->stream;
  const HostLevel& Lc = ctx->hl.back();
  const size_t nc2 = ctx->mg.coarse_direct ? (size_t)Lc.N * Lc.N : 0;
  lt::Batch& bt = ctx->pc_bt;
  lt::MGHost& mg = ctx->pc_mg;
  if (ctx->pc_nb < nimg) {
    CK(cudaStreamSynchronize(s));
    free_list(ctx->pc_allocs);
    ctx->pc_mg.d_levels = nullptr;
    int rc;
    auto& A = ctx->pc_allocs;
#define AL(p, n) if ((rc = dalloc(ctx, A, &p, (size_t)(n)))) return rc
    AL(bt.active, nimg); AL(bt.rnorm2, nimg); AL(bt.itol2, nimg); AL(bt.tau_cur, nimg); AL(bt.tau_slot, nimg);
    AL(bt.work, lt::kWorkSlots);
    if (nc2) AL(bt.coarse_inv, nimg * nc2);
    lt::tma_cache_free(mg);
    void* keep_none = nullptr;
    mg = ctx->mg;
    mg.tma_cache = keep_none;
    for (int l = 0; l < mg.nlev; ++l) {
      AL(mg.h_levels[l].u, (size_t)nimg * mg.h_levels[l].N);
      AL(mg.h_levels[l].f, (size_t)nimg * mg.h_levels[l].N);
    }
    lt::Level* dl = nullptr;
    AL(dl, lt::kMaxLevels);
#undef AL
    mg.d_levels = nullptr;
    CK(cudaMemcpy(dl, mg.h_levels, sizeof(lt::Level) * mg.nlev, cudaMemcpyHostToDevice));
    mg.d_levels = dl;
    ctx->pc_nb = nimg;
  }
  mg.npre = ctx->opts.mg_pre; mg.npost = ctx->opts.mg_post; mg.tile = ctx->opts.mg_tile; mg.tma = ctx->opts.mg_tma;
  bt.nb = nimg;
  bt.rounds = 0;
  bt.tma_polls = (unsigned)ctx->opts.tma_wait_polls;
  bt.coarse_direct = ctx->mg.coarse_direct;
  std::vector<int> ones(nimg, 1), slots(nimg);
  std::vector<double> big(nimg, 1e300), zero(nimg, 0.0);
  std::vector<double2> t2(nimg);
  std::vector<float2> inv32(nimg * nc2);
  for (int i = 0; i < nimg; ++i) {
    t2[i] = make_double2(tau[2 * i], tau[2 * i + 1]);
    slots[i] = i;
    if (nc2) {
      std::vector<cplx> inv;
      if (!dense_inverse(Lc, cplx(tau[2 * i], tau[2 * i + 1]), inv)) return fail(ctx, LT_ERR_INVALID_ARG, "singular coarse operator");
      for (size_t q = 0; q < nc2; ++q) inv32[i * nc2 + q] = make_float2((float)inv[q].real(), (float)inv[q].imag());
    }
  }
  CK(cudaMemcpyAsync(bt.active, ones.data(), nimg * sizeof(int), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(bt.rnorm2, big.data(), nimg * sizeof(double), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(bt.itol2, zero.data(), nimg * sizeof(double), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(bt.tau_cur, t2.data(), nimg * sizeof(double2), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(bt.tau_slot, slots.data(), nimg * sizeof(int), cudaMemcpyHostToDevice, s));
  if (nc2) CK(cudaMemcpyAsync(bt.coarse_inv, inv32.data(), inv32.size() * sizeof(float2), cudaMemcpyHostToDevice, s));
  const lt::Level& L0 = mg.h_levels[0];
  CK(cudaMemcpyAsync(L0.f, r, (size_t)nimg * L0.N * sizeof(float2), cudaMemcpyDeviceToDevice, s));
  CK(cudaMemsetAsync(L0.u, 0, (size_t)nimg * L0.N * sizeof(float2), s));
  CK(cudaMemsetAsync(bt.work, 0, lt::kWorkSlots * sizeof(unsigned long long), s));
  int nl = 0;
  for (int c = 0; c < cycles; ++c)
    if (lt::launch_vcycle(mg, bt, 0, s, &nl, nullptr)) return fail(ctx, LT_ERR_CUDA, "V-cycle launch failed");
  CK(cudaMemcpyAsync(e, L0.u, (size_t)nimg * L0.N * sizeof(float2), cudaMemcpyDeviceToDevice, s));
  unsigned long long flag = 0;
  CK(cudaMemcpyAsync(&flag, bt.work + lt::kTimeoutSlot, sizeof(flag), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (flag) return fail(ctx, LT_ERR_TIMEOUT, "a bulk tensor copy did not complete within its bounded wait");
  return LT_OK;
}

// ------------------------------------------------------------------ Crank-Nicolson (comparison method)
// rate of source s at time t: sum_j a_j exp(-lambda_j t), or the constant Q_s
static double qtime(const lt_ctx* ctx, int s, double t) {
  if (ctx->rate_a.empty()) return ctx->Q[s];
  double v = 0.0;
  for (size_t j = 0; j < ctx->rate_a[s].size(); ++j) v += ctx->rate_a[s][j] * std::exp(-ctx->rate_l[s][j] * t);
  return v;
}

extern "C" int lt_crank_nicolson(lt_ctx* ctx, int nt, const double* times, int steps, double* h, int h_on_device,
                                 lt_stats* st) {
  if (!ctx) return LT_ERR_INVALID_ARG;
  int rc = check_times(ctx, nt, times);
  if (rc) return rc;
  for (int t = 1; t < nt; ++t)
    if (!(times[t] > times[t - 1])) return fail(ctx, LT_ERR_INVALID_ARG, "times must increase strictly");
  if (steps < 2 || steps > 1000000) return fail(ctx, LT_ERR_INVALID_ARG, "steps=%d must be in [2, 1e6]", steps);
  if (ctx->src.empty() || ctx->rec.empty()) return fail(ctx, LT_ERR_STATE, "sources and receivers must be set");
  if (!h) return fail(ctx, LT_ERR_INVALID_ARG, "h is null");
  if (ctx->arena_base) return fail(ctx, LT_ERR_STATE, "not available inside lt_forward_noalloc");
  CK(cudaSetDevice(ctx->device));
  stats_reset(st, true);
  const lt_opts& o = ctx->opts;
  const int ns = (int)ctx->src.size(), nr = (int)ctx->rec.size();
  const int64_t N = ctx->N;
  const int R = o.inner_rounds, cycles = o.inner_cycles;
  cudaStream_t s = ctx->stream;
  CK(cudaEventRecord(ctx->ev0, s));
  // schedule: interval i covers (t_{i-1}, t_i] with `steps` uniform steps; the first interval opens
  // with four backward-Euler quarter steps in place of its first step (Rannacher start)
  struct Seg { double tau, theta; int count, slot; };
  std::vector<Seg> segs;
  std::vector<double> srcw;
  double tprev = 0.0;
  for (int i = 0; i < nt; ++i) {
    const double dt = (times[i] - tprev) / steps;
    double tc = tprev;
    if (i == 0) {
      segs.push_back({4.0 / dt, 0.0, 4, 0});
      for (int q = 0; q < 4; ++q) {
        tc += dt / 4;
        for (int b = 0; b < ns; ++b) srcw.push_back(qtime(ctx, b, tc));
      }
    }
    const int ncn = i == 0 ? steps - 1 : steps;
    segs.push_back({2.0 / dt, 1.0, ncn, i + 1});
    for (int q = 0; q < ncn; ++q, tc += dt)
      for (int b = 0; b < ns; ++b) srcw.push_back(qtime(ctx, b, tc) + qtime(ctx, b, tc + dt));
    tprev = times[i];
  }
  const int nslots = nt + 1;
  // workspace (this call's own: the Krylov workspace of the context is left untouched)
  std::vector<void*> tmp;
  lt::MGHost mg = ctx->mg;
  mg.tma_cache = nullptr;
  lt::Batch bt{};
  lt::CnArgs a{};
  const HostLevel& Lc = ctx->hl.back();
  const size_t nc2 = ctx->mg.coarse_direct ? (size_t)Lc.N * Lc.N : 0;
  double *dD = nullptr, *dm = nullptr, *dsrcw = nullptr, *d_h = nullptr;
  int64_t *dcell = nullptr, *drc = nullptr;
  int* dstep = nullptr;
#define AL(p, n) if ((rc = dalloc(ctx, tmp, &p, (size_t)(n)))) { free_list(tmp); return rc; }
  AL(dD, N); AL(dm, N); AL(a.phi, (size_t)ns * N); AL(a.x, (size_t)ns * N); AL(a.f, (size_t)ns * N);
  AL(dcell, ns); AL(dsrcw, srcw.size()); AL(a.fnorm2, ns); AL(a.maxres2, 1); AL(dstep, 1); AL(drc, nr);
  AL(bt.active, ns); AL(bt.rnorm2, (size_t)ns * (R + 1)); AL(bt.itol2, ns); AL(bt.tau_cur, ns); AL(bt.tau_slot, ns);
  AL(bt.work, lt::kWorkSlots);
  if (nc2) AL(bt.coarse_inv, nslots * nc2);
  for (int l = 0; l < mg.nlev; ++l) {
    AL(mg.h_levels[l].u, (size_t)ns * mg.h_levels[l].N);
    AL(mg.h_levels[l].f, (size_t)ns * mg.h_levels[l].N);
  }
  lt::Level* dl = nullptr;
  AL(dl, lt::kMaxLevels);
  if (!h_on_device) AL(d_h, (size_t)ns * nr * nt);
#undef AL
  CK(cudaMemcpyAsync(dl, mg.h_levels, sizeof(lt::Level) * mg.nlev, cudaMemcpyHostToDevice, s));
  mg.d_levels = dl;
  mg.npre = o.mg_pre; mg.npost = o.mg_post; mg.tile = o.mg_tile; mg.tma = o.mg_tma;
  CK(cudaMemcpyAsync(dD, ctx->hl[0].D.data(), N * sizeof(double), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(dm, ctx->hl[0].m.data(), N * sizeof(double), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(dcell, ctx->src.data(), ns * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(drc, ctx->rec.data(), nr * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(dsrcw, srcw.data(), srcw.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  for (int b = 0; b < ns; ++b) {
    if (ctx->phi0.empty()) CK(cudaMemsetAsync(a.phi + (size_t)b * N, 0, N * sizeof(double), s));
    else CK(cudaMemcpyAsync(a.phi + (size_t)b * N, ctx->phi0.data(), N * sizeof(double), cudaMemcpyHostToDevice, s));
  }
  CK(cudaMemsetAsync(a.fnorm2, 0, ns * sizeof(double), s));
  CK(cudaMemsetAsync(a.maxres2, 0, sizeof(double), s));
  CK(cudaMemsetAsync(dstep, 0, sizeof(int), s));
  CK(cudaMemsetAsync(bt.work, 0, lt::kWorkSlots * sizeof(unsigned long long), s));
  if (nc2) {
    std::vector<float2> inv32(nslots * nc2);
    for (const Seg& g : segs) {
      std::vector<cplx> inv;
      if (!dense_inverse(Lc, cplx(g.tau, 0.0), inv)) { free_list(tmp); return fail(ctx, LT_ERR_INVALID_ARG, "singular coarse operator"); }
      for (size_t q = 0; q < nc2; ++q) inv32[g.slot * nc2 + q] = make_float2((float)inv[q].real(), (float)inv[q].imag());
    }
    CK(cudaMemcpyAsync(bt.coarse_inv, inv32.data(), inv32.size() * sizeof(float2), cudaMemcpyHostToDevice, s));
  }
  bt.nb = ns; bt.rounds = R; bt.N = N; bt.coarse_direct = ctx->mg.coarse_direct;
  bt.tma_polls = (unsigned)o.tma_wait_polls;
  a.nb = ns; a.N = N; a.nx = ctx->nx; a.ny = ctx->ny; a.nz = ctx->nz;
  a.Te = ctx->g_Te; a.Tn = ctx->g_Tn; a.Tu = ctx->g_Tu; a.D = dD; a.m = dm;
  a.cell = dcell; a.srcw = dsrcw; a.step = dstep; a.tol = o.tol;
  double* out = h_on_device ? h : d_h;
  int nl = 0;
  cudaStream_t cap = nullptr;
  CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaEventCreateWithFlags(&e0, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&e1, cudaEventDisableTiming));
  CK(cudaEventRecord(e0, s));
  CK(cudaStreamWaitEvent(cap, e0, 0));
  int t_out = 0, total = 0;
  for (size_t gi = 0; gi < segs.size() && rc == LT_OK; ++gi) {
    const Seg& g = segs[gi];
    std::vector<double2> tc(ns, make_double2(g.tau, 0.0));
    std::vector<int> sl(ns, g.slot);
    CK(cudaMemcpyAsync(bt.tau_cur, tc.data(), ns * sizeof(double2), cudaMemcpyHostToDevice, cap));
    CK(cudaMemcpyAsync(bt.tau_slot, sl.data(), ns * sizeof(int), cudaMemcpyHostToDevice, cap));
    CK(cudaStreamSynchronize(cap));     // host tables go out of scope
    a.tau = g.tau; a.theta = g.theta;
    // one step captured, replayed g.count times (the step index lives on the device)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    int per = 0;
    CK(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
    int lr = lt::launch_cn_step(mg, bt, a, cycles, cap, &per);
    cudaError_t ec = cudaStreamEndCapture(cap, &graph);
    if (lr || ec != cudaSuccess) { rc = fail(ctx, LT_ERR_CUDA, "capture of a time step failed"); break; }
    ec = cudaGraphInstantiate(&gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (ec != cudaSuccess) { rc = fail(ctx, LT_ERR_CUDA, "graph instantiate failed: %s", cudaGetErrorString(ec)); break; }
    for (int q = 0; q < g.count; ++q) CK(cudaGraphLaunch(gexec, cap));
    cudaGraphExecDestroy(gexec);
    nl += per * g.count;
    total += g.count;
    // an output time ends every CN segment
    if (g.theta != 0.0) {
      lt::launch_cn_measure(a, drc, nr, nt, t_out++, out, cap);
      ++nl;
    }
  }
  CK(cudaEventRecord(e1, cap));
  CK(cudaStreamWaitEvent(s, e1, 0));
  CK(cudaEventRecord(ctx->ev1, s));
  double maxres2 = 0.0;
  unsigned long long flag = 0;
  if (rc == LT_OK) {
    if (!h_on_device) CK(cudaMemcpyAsync(h, d_h, (size_t)ns * nr * nt * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&maxres2, a.maxres2, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&flag, bt.work + lt::kTimeoutSlot, sizeof(flag), cudaMemcpyDeviceToHost, s));
  }
  cudaStreamSynchronize(s);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(cap);
  lt::tma_cache_free(mg);
  free_list(tmp);
  if (rc) return rc;
  if (flag) return fail(ctx, LT_ERR_TIMEOUT, "a bulk tensor copy did not complete within its bounded wait");
  const double maxres = std::sqrt(maxres2);
  if (st) {
    cudaEventElapsedTime(&st->ms_total, ctx->ev0, ctx->ev1);
    st->kernel_launches = nl;
    st->n_bases = ns;
    st->n_shift_solves = total * ns;
    st->n_converged = maxres <= o.tol ? total * ns : 0;
    st->max_true_residual = maxres;
  }
  if (!(maxres <= o.tol)) return fail(ctx, LT_ERR_NOT_CONVERGED, "a time step's solve stopped at %.3g > tol", maxres);
  return LT_OK;
}

// ------------------------------------------------------------------ geostatistical inversion (Algorithm 2)
extern "C" int lt_geostat_step(lt_ctx* ctx, int nt, const double* times, const double* y, const double* R,
                               double sigma2, double ell, double* s_next, double* beta, double* xi, double* h,
                               lt_stats* st) {
  if (!ctx) return LT_ERR_INVALID_ARG;
  int rc = check_times(ctx, nt, times);
  if (rc) return rc;
  if (ctx->nz != 1) return fail(ctx, LT_ERR_INVALID_ARG, "the FFT covariance product is implemented for 2D grids");
  if (!y || !R || !s_next || !beta) return fail(ctx, LT_ERR_INVALID_ARG, "y, R, s_next and beta are required");
  if (!(sigma2 > 0.0) || !(ell > 0.0)) return fail(ctx, LT_ERR_INVALID_ARG, "sigma2 and ell must be positive");
  if (ctx->src.empty() || ctx->rec.empty()) return fail(ctx, LT_ERR_STATE, "sources and receivers must be set");
  const int ns = (int)ctx->src.size(), nr = (int)ctx->rec.size();
  const int ny = ns * nr * nt;
  for (int i = 0; i < ny; ++i)
    if (!(R[i] > 0.0) || !std::isfinite(y[i])) return fail(ctx, LT_ERR_INVALID_ARG, "R[%d] must be > 0, y finite", i);
  const int nx = ctx->nx, nyg = ctx->ny;
  const int64_t N = ctx->N;
  int P0 = 1, P1 = 1;
  while (P0 < 2 * nx) P0 <<= 1;
  while (P1 < 2 * nyg) P1 <<= 1;
  if (P0 > 2048 || P1 > 2048) return fail(ctx, LT_ERR_INVALID_ARG, "grid too large for the FFT product (side <= 1024)");
  CK(cudaSetDevice(ctx->device));
  cudaStream_t s = ctx->stream;
  // J (both halves; the log-kappa half is used) and h at s_k
  std::vector<void*> tmp;
  double *dJ = nullptr, *dh = nullptr;
  if ((rc = dalloc(ctx, tmp, &dJ, (size_t)ny * 2 * N)) || (rc = dalloc(ctx, tmp, &dh, ny))) { free_list(tmp); return rc; }
  rc = adjoint_impl(ctx, nt, times, dJ, nullptr, nullptr, dh, 1, 0, st);
  if (rc && rc != LT_ERR_NOT_CONVERGED) { free_list(tmp); return rc; }
  const int solve_rc = rc;
  const size_t ldj = 2 * (size_t)N;
  // covariance spectrum: sigma2 exp(-r / ell) on the P1 x P0 torus (cell-centre distances in metres)
  const size_t nimg = (size_t)P0 * P1;
  const int chunk = (int)std::max<size_t>(1, std::min<size_t>(ny, ((size_t)1 << 28) / (nimg * sizeof(double2))));
  double2 *img = nullptr, *tmpi = nullptr;
  double *lam = nullptr, *G = nullptr, *A = nullptr, *rhs = nullptr, *z = nullptr, *dbeta = nullptr, *dxi = nullptr;
  double *ds = nullptr, *dsn = nullptr, *dy = nullptr, *dR = nullptr;
  int* flag = nullptr;
  if ((rc = dalloc(ctx, tmp, &img, (size_t)chunk * nimg)) || (rc = dalloc(ctx, tmp, &tmpi, (size_t)chunk * nimg)) ||
      (rc = dalloc(ctx, tmp, &lam, nimg)) || (rc = dalloc(ctx, tmp, &G, (size_t)ny * N)) ||
      (rc = dalloc(ctx, tmp, &A, (size_t)ny * ny)) || (rc = dalloc(ctx, tmp, &rhs, 2 * (size_t)ny)) ||
      (rc = dalloc(ctx, tmp, &z, 2 * (size_t)ny)) || (rc = dalloc(ctx, tmp, &dbeta, 1)) ||
      (rc = dalloc(ctx, tmp, &dxi, ny)) || (rc = dalloc(ctx, tmp, &ds, N)) || (rc = dalloc(ctx, tmp, &dsn, N)) ||
      (rc = dalloc(ctx, tmp, &dy, ny)) || (rc = dalloc(ctx, tmp, &dR, ny)) || (rc = dalloc(ctx, tmp, &flag, 1))) {
    free_list(tmp);
    return rc;
  }
  {
    std::vector<double2> c(nimg);
    for (int j = 0; j < P1; ++j)
      for (int i = 0; i < P0; ++i) {
        const double ddx = ctx->dx * std::min(i, P0 - i), ddy = ctx->dy * std::min(j, P1 - j);
        c[(size_t)j * P0 + i] = make_double2(sigma2 * std::exp(-std::sqrt(ddx * ddx + ddy * ddy) / ell), 0.0);
      }
    std::vector<double> sk(N);
    for (int64_t q = 0; q < N; ++q) sk[q] = std::log(ctx->kappa[q]);
    CK(cudaMemcpyAsync(img, c.data(), nimg * sizeof(double2), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ds, sk.data(), N * sizeof(double), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(dy, y, ny * sizeof(double), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(dR, R, ny * sizeof(double), cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(flag, 0, sizeof(int), s));
    if (lt::geostat_prepare(P0, P1) || lt::geostat_spectrum(img, tmpi, P0, P1, lam, s)) {
      free_list(tmp);
      return fail(ctx, LT_ERR_CUDA, "covariance spectrum failed");
    }
    CK(cudaStreamSynchronize(s));     // host tables go out of scope
  }
  // Q J^T by FFT, chunk images at a time
  for (int r0 = 0; r0 < ny; r0 += chunk) {
    const int nrows = std::min(chunk, ny - r0);
    if (lt::geostat_qjt(dJ, ldj, r0, nrows, nx, nyg, P0, P1, lam, img, tmpi, G, s)) {
      free_list(tmp);
      return fail(ctx, LT_ERR_CUDA, "Q J^T launch failed");
    }
  }
  if (lt::geostat_solve(dJ, ldj, G, ny, (int)N, dR, ds, dy, dh, A, rhs, z, dbeta, dxi, dsn, flag, s)) {
    free_list(tmp);
    return fail(ctx, LT_ERR_CUDA, "saddle-point solve launch failed");
  }
  int hflag = 0;
  CK(cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(s_next, dsn, N * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(beta, dbeta, sizeof(double), cudaMemcpyDeviceToHost, s));
  if (xi) CK(cudaMemcpyAsync(xi, dxi, ny * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (h) CK(cudaMemcpyAsync(h, dh, ny * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  free_list(tmp);
  if (hflag) return fail(ctx, LT_ERR_INVALID_ARG, "J Q J^T + R is not positive definite");
  return solve_rc;
}

// ------------------------------------------------------------------ learned preconditioner: data
extern "C" int lt_contour_nodes(double t, int Nz, int project, double* z, double* w) {
  if (!(t > 0.0) || !std::isfinite(t) || Nz < 4 || Nz > 128 || (Nz & 1) || !z) return LT_ERR_INVALID_ARG;
  std::vector<cplx> zz, ww;
  talbot_half(t, Nz, zz, ww);
  for (int k = 0; k < Nz / 2; ++k) {
    cplx v = zz[k];
    if (project) v = cplx(std::max(v.real(), 0.0), v.imag());
    z[2 * k] = v.real();
    z[2 * k + 1] = v.imag();
    if (w) {
      w[2 * k] = ww[k].real();
      w[2 * k + 1] = ww[k].imag();
    }
  }
  return LT_OK;
}

extern "C" int lt_learned_pairs(lt_ctx* ctx, int nimg, const double* tau, const float* r, int cycles, float* x,
                                float* y) {
  if (!ctx) return LT_ERR_INVALID_ARG;
  if (!ctx->have_grid) return fail(ctx, LT_ERR_STATE, "lt_setup_grid must come first");
  if (nimg < 1 || !tau || !r || !x || !y) return fail(ctx, LT_ERR_INVALID_ARG, "nimg >= 1 and non-null buffers");
  CK(cudaSetDevice(ctx->device));
  int rc = learned_tables(ctx);
  if (rc) return rc;
  std::vector<void*> tmp;
  float2* e = nullptr;
  double2* dtau = nullptr;
  double* acc = nullptr;
  if ((rc = dalloc(ctx, tmp, &e, (size_t)nimg * ctx->N)) || (rc = dalloc(ctx, tmp, &dtau, nimg)) ||
      (rc = dalloc(ctx, tmp, &acc, 2 * (size_t)nimg))) {
    free_list(tmp);
    return rc;
  }
  rc = lt_precond_apply(ctx, nimg, tau, r, (float*)e, cycles);
  if (rc) { free_list(tmp); return rc; }
  cudaStream_t s = ctx->stream;
  CK(cudaMemcpyAsync(dtau, tau, nimg * sizeof(double2), cudaMemcpyHostToDevice, s));
  learned_pair_features(nimg, (int)ctx->N, (const float2*)r, e, dtau, ctx->d_lk, ctx->d_mD, ctx->d_D32, acc, x, y, s);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  free_list(tmp);
  return LT_OK;
}

extern "C" int lt_krylov_vectors(lt_ctx* ctx, int max_n, float* r, double* tau, int* n_out) {
  if (!ctx || !n_out) return LT_ERR_INVALID_ARG;
  *n_out = 0;
  if (ctx->last_nit.empty() || !ctx->ws.bt.V_hi) return fail(ctx, LT_ERR_STATE, "no forward solve to take vectors from");
  if (max_n < 0 || (max_n > 0 && (!r || !tau))) return fail(ctx, LT_ERR_INVALID_ARG, "max_n >= 0 and non-null buffers");
  CK(cudaSetDevice(ctx->device));
  const lt::Batch& bt = ctx->ws.bt;
  const size_t N = (size_t)ctx->N;
  static const int pat_flex[5] = {0, 0, 0, 1, 1};
  int n = 0;
  cudaStream_t s = ctx->stream;
  for (size_t b = 0; b < ctx->last_nit.size() && n < max_n; ++b)
    for (int j = 0; j < ctx->last_nit[b] && n < max_n; ++j, ++n) {
      const float2* v = bt.V_hi + (b * (size_t)(bt.maxit + 1) + j) * N;
      CK(cudaMemcpyAsync(r + (size_t)n * N * 2, v, N * sizeof(float2), cudaMemcpyDeviceToDevice, s));
      const int slot = ctx->last_single ? 0 : pat_flex[j % 5];
      const cplx t = ctx->last_tau[2 * ctx->last_group[b] + slot];
      tau[2 * n] = t.real();
      tau[2 * n + 1] = t.imag();
    }
  CK(cudaStreamSynchronize(s));
  *n_out = n;
  return LT_OK;
}

// ------------------------------------------------------------------ no-allocation forward
// Some callers cannot let a library call cudaMalloc/cudaFree: services that
// hand all device memory to their own pool allocator up front (a library
// allocation then fails or fragments that pool), and pipelines that keep
// other streams busy, where cudaMalloc/cudaFree may synchronise the device
// and stall them.  lt_forward_noalloc serves them: it runs the same solve as
// lt_forward but takes every device buffer it needs from this fixed static
// region, which each GPU that loads the library holds until the process
// exits.
#define LT_NOALLOC_SCRATCH_BYTES (32u << 20)
static __device__ __align__(256) unsigned char g_lt_noalloc_scratch[LT_NOALLOC_SCRATCH_BYTES];

static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[256];   // device address of g_lt_noalloc_scratch, per device ordinal

// bytes the no-allocation forward carves for a plan (same list as ensure_ws,
// run_solves and forward_impl, each rounded to 256 bytes)
static size_t noalloc_need(const lt_ctx* ctx, const Plan& P) {
  const lt_opts& o = ctx->opts;
  const size_t nb = P.nb, M = o.maxit, R = o.inner_rounds, nsh = P.nsh, N = (size_t)ctx->N, G = P.G;
  const size_t ns = ctx->src.size(), nr = ctx->rec.size(), nt = P.nt;
  size_t b = 0;
  auto add = [&](size_t n, size_t sz) { b += round256(std::max<size_t>(n, 1) * sz); };
  const bool df = o.precision == LT_PREC_FP64;   // lo planes only in df32
  add(nb * (M + 1) * N, 8); add(nb * M * N, 8); add(nb * N, 8);
  if (df) { add(nb * (M + 1) * N, 8); add(nb * M * N, 8); add(nb * N, 8); }
  add(nsh, 8); add(N, 4); add(N, 4);
  add(2 * G, 16); add(nb, 4); add(5, 4); add(nb, 16); add(nb, 4);
  add(nb * (R + 1), 8); add(nb * 2 * (M + 1), 16); add(nb * M * (M + 1), 16);
  add(nb, 8); add(nb, 4); add(nb, 4); add(nb, 8); add(nb, 8);
  add(nb + 1, 4); add(nsh, 16); add(nsh * M * M, 16); add(nsh * M, 8);
  add(nsh * M, 16); add(nsh * (M + 1), 16); add(nsh, 4); add(nsh, 8);
  add(nsh * M, 16); add(lt::kWorkSlots, 8); add(nb, 8); add(nb, 8); add(8, 4);
  if (ctx->mg.coarse_direct) add(2 * G * (size_t)ctx->hl.back().N * ctx->hl.back().N, 8);
  if (ctx->inner.ok || any_cluster_plan(ctx)) add(nb * N, 16);
  if (cluster_plan(ctx).u0_global) add(nb * N, 8);
  for (int l = 0; l < ctx->mg.nlev; ++l) { add(nb * ctx->mg.h_levels[l].N, 8); add(nb * ctx->mg.h_levels[l].N, 8); }
  add(nsh, 4);
  if (o.true_residual) { add(nsh * N, 8); if (df) add(nsh * N, 8); add(nsh, 8); }
  const size_t nitems = ns * nt + (P.dense_b0 >= 0 ? nt : 0);
  add(nitems, sizeof(lt::QuadItem)); add(nsh, 16); add(nitems * M, 16); add(std::max<size_t>(nr, 1), 8);
  return b;
}

extern "C" int lt_forward_noalloc(lt_ctx* ctx, int nt, const double* times, double* h, lt_stats* st) {
  if (!ctx) return LT_ERR_INVALID_ARG;
  int rc = check_times(ctx, nt, times);
  if (rc) return rc;
  if (ctx->src.empty() || ctx->rec.empty()) return fail(ctx, LT_ERR_STATE, "sources and receivers must be set");
  if (!h) return fail(ctx, LT_ERR_INVALID_ARG, "h (device pointer) is null");
  if (ctx->opts.precond != 0) return fail(ctx, LT_ERR_INVALID_ARG, "lt_forward_noalloc supports only precond = 0");
  if (ctx->opts.block) return fail(ctx, LT_ERR_INVALID_ARG, "lt_forward_noalloc does not support block = 1");
  if (ctx->device < 0 || ctx->device >= 256) return fail(ctx, LT_ERR_INVALID_ARG, "device ordinal out of range");
  CK(cudaSetDevice(ctx->device));
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[ctx->device]) {
      cudaError_t e = cudaGetSymbolAddress(&g_noalloc_ptr[ctx->device], g_lt_noalloc_scratch);
      if (e != cudaSuccess) {
        g_noalloc_ptr[ctx->device] = nullptr;
        return fail(ctx, LT_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed: %s", cudaGetErrorString(e));
      }
    }
    base = g_noalloc_ptr[ctx->device];
  }
  Plan P;
  make_plan(ctx, nt, times, ctx->src, P, (int)ctx->src.size(), !ctx->phi0.empty());
  const size_t need = noalloc_need(ctx, P);
  if (need > LT_NOALLOC_SCRATCH_BYTES)
    return fail(ctx, LT_ERR_INVALID_ARG,
                "problem needs %zu bytes of device scratch; lt_forward_noalloc is limited to %u bytes "
                "(reduce grid size, wells, times, Nz or maxit, or use lt_forward)",
                need, (unsigned)LT_NOALLOC_SCRATCH_BYTES);
  // run the ordinary forward driver with buffers carved from the static region;
  // the context's own cached workspace and level pointers are set aside and restored
  Workspace saved_ws = std::move(ctx->ws);
  ctx->ws = Workspace();
  lt::Level saved_levels[lt::kMaxLevels];
  memcpy(saved_levels, ctx->mg.h_levels, sizeof(saved_levels));
  const int saved_timing = ctx->opts.timing_class;
  ctx->opts.timing_class = -1;
  ctx->arena_base = (char*)base;
  ctx->arena_cap = LT_NOALLOC_SCRATCH_BYTES;
  ctx->arena_off = 0;
  rc = forward_impl(ctx, nt, times, h, 1, 0, st);
  // an error return can leave kernels of this call queued on the caller's stream; they read the
  // level table that points into the static region, so let them finish before it is restored
  cudaError_t es = cudaStreamSynchronize(ctx->stream);
  ctx->arena_base = nullptr;
  ctx->arena_cap = ctx->arena_off = 0;
  ctx->opts.timing_class = saved_timing;
  ctx->ws = std::move(saved_ws);
  ctx->last_nit.clear();          // the bases of this call lived in the static region
  memcpy(ctx->mg.h_levels, saved_levels, sizeof(saved_levels));
  cudaError_t e = cudaMemcpy(ctx->mg.d_levels, ctx->mg.h_levels, sizeof(lt::Level) * ctx->mg.nlev,
                             cudaMemcpyHostToDevice);
  if (e != cudaSuccess && rc == LT_OK) return fail(ctx, LT_ERR_CUDA, "restoring level table: %s", cudaGetErrorString(e));
  if (es != cudaSuccess && rc == LT_OK) return fail(ctx, LT_ERR_CUDA, "stream synchronize: %s", cudaGetErrorString(es));
  return rc;
}
