// inner.cu -- the preconditioner solve (K + tau_j M) u_j = v_j of one Krylov
// basis (Sec. 3: the shift-and-invert step of Algorithm 1), all refinement
// rounds and V-cycles, inside one thread-block cluster.
//
// The arithmetic is that of the batched launches in krylov.cu and mg.cu:
// rounds of  r = v_j - (K + tau M) u_j  in df32, float32 V-cycles on A d = r
// (red-black Gauss-Seidel, sum restriction, bilinear prolongation, dense
// inverse or sweeps at the coarsest level), u_j += d in df32, until
// ||r||^2 <= itol2.  What changes is where the data lives:
//   * the cs CTAs of a cluster (8, or 16 with half-height strips) split every multigrid level above
//     kCoarseCells cells into cs strips of whole rows; each CTA keeps the
//     iterate and right-hand side of its strips in shared memory for the
//     whole solve and reads the row just outside a strip from the
//     neighbouring CTA's shared memory (distributed shared memory);
//   * the levels of at most kCoarseCells cells live in rank 0, which runs
//     their sweeps; the dense inverse of the coarsest level is applied by all
//     ranks, a slice of its rows each;
//   * a cluster barrier follows every red or black half-sweep, so every
//     half-sweep sees the other colour exactly as the global sweep does;
//   * the squared residual norm of each round is summed over the cluster in
//     rank order, so every CTA takes the same branch;
//   * the V-cycles of a round stop once the fine residual the restriction
//     computes anyway is below the round's goal (at most `cycles`);
//   * per-cell records and strip arrays are kept in red-black order, so a
//     half-sweep reads contiguous runs (global loads and shared-memory banks).
// One launch replaces the (rounds x (cycles x V-cycle launches + 2)) launches
// of the batched path.
#include <cooperative_groups.h>

#include "df32.cuh"
#include "exact.cuh"
#include "lt_internal.h"
#include "lt_kernels.h"
#include "mg_dev.cuh"

namespace cg = cooperative_groups;

namespace lt {

constexpr int kIT = 512;                      // most threads per CTA (the launch bound)
constexpr size_t kInnerSmemMax = 220 * 1024;  // dynamic shared memory per CTA
constexpr int kL0Batch = 1;                   // finest-level cells per thread whose loads are issued together

// Division by a runtime divisor d >= 1 of a numerator below 2^31 as a multiply-high and a shift
// (Granlund and Montgomery, "Division by invariant integers using multiplication", 1994):
// l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1, q / d = (umulhi(q, m) + q) >> l.
struct FastDiv {
  uint32_t m;
  int s;
};
static FastDiv make_fastdiv(uint32_t d) {
  int l = 0;
  while ((1u << l) < d) ++l;
  const uint64_t m = ((uint64_t(1) << 32) * ((uint64_t(1) << l) - d)) / d + 1;
  return FastDiv{(uint32_t)m, l};
}
__device__ __forceinline__ int fdiv(int q, FastDiv f) {
  const uint32_t t = __umulhi((uint32_t)q, f.m);
  return (int)((t + (uint32_t)q) >> f.s);
}

// Byte offsets of one level's arrays in dynamic shared memory.  The finest
// level keeps only its iterate there; its coefficients come from global
// memory as two 16-byte loads per cell (the four face transmissibilities,
// shared by all bases, and per basis the inverse complex diagonal with the
// right-hand side), batched.  Every coarser level also keeps its right-hand
// side, east/north face transmissibilities and the inverse of its complex
// diagonal, staged once per launch.
struct LevOff { int u, f, te, tn, di; };

struct InnerArgs {
  Batch bt;
  FineExact fe;
  const Level* levels;          // device copy of the level descriptors
  const float4* p4;             // [N] finest level: (Te east, Te west, Tn north, Tn south), red-black order
  float4* q4;                   // [nb][N] finest level: (1 / (D + tau m), right-hand side) per basis, same order
  int nlev, ld;                 // levels [0, ld) in strips, [ld, nlev) in rank 0
  int cs;                       // CTAs per cluster (row strips per strip level)
  float2* u0g;                  // [nb][N] finest-level iterates in strip blocks, or null (shared memory)
  int npre, npost, dmask, coarse_direct, rounds, cycles;
  LevOff off[kMaxLevels];
  int off_rhs;                  // byte offset of rank 0's coarsest right-hand side copy
  FastDiv dnx[kMaxLevels];      // divisions by the level's row length
  FastDiv dhx[kMaxLevels];      // ... and by half of it (cells of one colour per row)
};

// Strip levels keep their shared-memory arrays in red-black order too: colour c = (x + y) & 1, then
// the strip's rows, then x / 2 ([2][h][nx/2]; strips start on even rows, so the colour of local row
// ly is (x + ly) & 1).  A half-sweep's own cells and each of its four neighbour streams are then
// contiguous across a warp (no shared-memory bank conflicts).  For a cell of colour c in local row
// ly at position k (x = 2k + p, p = (c + ly) & 1) the neighbours have colour 1 - c and positions
// k + p (east), k - 1 + p (west), k (north, south).

// The finest level's rows [y0, y0 + h) of this CTA.
struct L0V {
  int nx, ny, h, y0, hx, plane;  // hx = nx / 2, plane = h hx (cells of one colour in the strip)
  int gl;                        // 1: the iterates are strip blocks of a global array (rows of the neighbour
                                 //    ranks are read past L1, from L2), 0: shared memory
  const float4* __restrict__ P;  // faces (red-black order over the whole level)
  const float4* Q;               // inverse diagonal and right-hand side (same order; rewritten every round)
  float2* u;                     // [2][h][hx], shared memory or global
  const float2* u_dn;            // iterate of rank - 1 (its last row lies just below y0), or null
  const float2* u_up;            // iterate of rank + 1 (its first row lies just above y0 + h - 1), or null
};

// A strip level below the finest, staged in shared memory in red-black order.
struct RBV {
  int nx, ny, h, y0, hx, plane;
  float2* u;                     // [2][h][hx]
  float2* f;                     // [2][h][hx]
  float* te;                     // [2][h][hx]     east face of the cell
  float* ts;                     // [2][h+1][hx]   south face of the cell in local row r (r = h: the row above)
  float2* di;                    // [2][h][hx]     1 / (D + tau m)
  const float2* u_dn;
  const float2* u_up;
};

// A whole coarse level held by rank 0, staged in shared memory in natural order (y0 = 0, h = ny; the
// neighbour pointers stay null, as no row lies outside the level).
struct SV {
  int nx, ny, h, y0;
  float2* u;                     // [h][nx]
  float2* f;                     // [h][nx]
  float* te;                     // [h][nx]    face (x, y)-(x+1, y)
  float* tn;                     // [h+1][nx]  row r: face (x, y0+r-1)-(x, y0+r)
  float2* di;                    // [h][nx]    1 / (D + tau m)
  const float2* u_dn;
  const float2* u_up;
};

// Read access to the iterate of the next coarser level, for the prolongation.
struct CoarseView {
  int nx, ny;
  int full;                      // 1: the whole level in one array (rank 0's, natural order), 0: red-black strips
  int hc, yc0, hxc, planec;      // own strip rows, half row length and cells per colour when !full
  const float2* loc;
  const float2* dn;
  const float2* up;
};

__device__ __forceinline__ void axpy_c(float2& r, float t, float2 v) { r.x += t * v.x; r.y += t * v.y; }

// ---------------------------------------------------------------- finest level (global coefficients)
// The finest level's per-cell records are stored in red-black order: all cells of colour 0,
// then all of colour 1, each colour row by row, so that the cells one half-sweep visits are
// contiguous (cell (x, y) of an nx-wide level at  ((x + y) & 1) * N/2 + y * nx/2 + x/2).
__device__ __forceinline__ int rb_index(int x, int y, int nx, int nhalf) {
  return ((x + y) & 1) * nhalf + y * (nx >> 1) + (x >> 1);
}

// loads of one cell of the finest level: the four faces, inverse diagonal and right-hand side
struct L0Cell { float4 t; float4 q; };

__device__ __forceinline__ L0Cell l0_load(const L0V& S, int r) {
  L0Cell v;
  v.t = S.P[r];
  v.q = S.Q[r];
  return v;
}

// neighbour iterates (red-black strip order) of the colour-c cell at local row ly, position k (zero where
// the cell has no neighbour); u, u_dn, u_up: this strip's and the neighbour ranks' arrays
__device__ __forceinline__ void rb_gather(const float2* u, const float2* u_dn, const float2* u_up, int nx, int ny,
                                          int h, int y0, int hx, int plane, int c, int ly, int k, float2* nb) {
  const float2 z = make_float2(0.f, 0.f);
  const int p = (c + ly) & 1, x = 2 * k + p, y = y0 + ly;
  const int ob = (c ^ 1) * plane, row = ob + ly * hx;
  nb[0] = x + 1 < nx ? u[row + k + p] : z;
  nb[1] = x > 0 ? u[row + k - 1 + p] : z;
  nb[2] = y + 1 < ny ? (ly + 1 < h ? u[row + hx + k] : u_up[ob + k]) : z;
  nb[3] = y > 0 ? (ly > 0 ? u[row - hx + k] : u_dn[ob + (h - 1) * hx + k]) : z;
}
__device__ __forceinline__ void l0_gather(const L0V& S, int c, int ly, int k, float2* nb) {
  if (!S.gl) {
    rb_gather(S.u, S.u_dn, S.u_up, S.nx, S.ny, S.h, S.y0, S.hx, S.plane, c, ly, k, nb);
    return;
  }
  // global strip blocks: a neighbour rank's rows were written by another SM, so they come from L2
  const float2 z = make_float2(0.f, 0.f);
  const int p = (c + ly) & 1, x = 2 * k + p, y = S.y0 + ly;
  const int ob = (c ^ 1) * S.plane, row = ob + ly * S.hx;
  nb[0] = x + 1 < S.nx ? S.u[row + k + p] : z;
  nb[1] = x > 0 ? S.u[row + k - 1 + p] : z;
  nb[2] = y + 1 < S.ny ? (ly + 1 < S.h ? S.u[row + S.hx + k] : __ldcg(&S.u_up[ob + k])) : z;
  nb[3] = y > 0 ? (ly > 0 ? S.u[row - S.hx + k] : __ldcg(&S.u_dn[ob + (S.h - 1) * S.hx + k])) : z;
}

__device__ __forceinline__ float2 nb_dot(float4 t, const float2* nb) {
  return make_float2(t.x * nb[0].x + t.y * nb[1].x + t.z * nb[2].x + t.w * nb[3].x,
                     t.x * nb[0].y + t.y * nb[1].y + t.z * nb[2].y + t.w * nb[3].y);
}

// one red (color 0) or black (color 1) half-sweep over the strip's cells of that colour
__device__ __forceinline__ void l0_half_sweep(const L0V& S, FastDiv dhx, int color) {
  const int hx = S.nx >> 1, n = S.h * hx;
  for (int q0 = threadIdx.x; q0 < n; q0 += kL0Batch * (int)blockDim.x) {
    L0Cell cq[kL0Batch];
#pragma unroll
    for (int k = 0; k < kL0Batch; ++k) {
      const int q = q0 + k * (int)blockDim.x;
      if (q < n) {
        cq[k] = l0_load(S, color * (S.ny * hx) + S.y0 * hx + q);   // red-black order: contiguous in q
      }
    }
#pragma unroll
    for (int k = 0; k < kL0Batch; ++k) {
      const int q = q0 + k * (int)blockDim.x;
      if (q < n) {
        const int ly = fdiv(q, dhx);
        float2 nb[4];
        l0_gather(S, color, ly, q - ly * hx, nb);
        float2 r = nb_dot(cq[k].t, nb);
        r.x += cq[k].q.z; r.y += cq[k].q.w;
        S.u[color * S.plane + q] = cmul(r, make_float2(cq[k].q.x, cq[k].q.y));
      }
    }
  }
}

// Where the restriction writes coarse cell (I, row J of the strip): the next strip level's red-black
// arrays (fc_planec > 0: cells per colour of its strip, half row length fc_hx), or rank 0's whole
// level in natural order (fc_planec = 0: row J + rowoff, ncx columns).
__device__ __forceinline__ int coarse_slot(int I, int lJ, int ncx, int rowoff, int fc_hx, int fc_planec) {
  return fc_planec > 0 ? ((I + lJ) & 1) * fc_planec + lJ * fc_hx + (I >> 1) : (lJ + rowoff) * ncx + I;
}

// Residual summed over the 2x2 children into the coarse right-hand side; returns this thread's sum of
// |r|^2 over the fine cells (the V-cycle's convergence monitor).  After a red-black sweep ending with
// the black half-sweep every black cell satisfies its equation, so its residual is zero up to rounding
// and only the two red children are evaluated; red_only = false evaluates all four.  The children of
// coarse cell I all sit at position k = I of their colour and row (strips start on even rows).
// Which fine cells the restriction evaluates (the others have a zero residual, or all four when
// nothing is known): kRestrictAll; kRestrictRed after a sweep ending with a black half-sweep;
// kRestrictBlack after one ending with a red half-sweep; kRestrictZeroU when the iterate is zero,
// so the residual is the right-hand side itself (no neighbours read).
constexpr int kRestrictAll = 0, kRestrictRed = 1, kRestrictBlack = 2, kRestrictZeroU = 3;

__device__ __forceinline__ float l0_restrict(const L0V& S, float2* fc, int ncx, FastDiv dncx, int rowoff, int fc_hx,
                                             int fc_planec, int mode) {
  const int nch = S.h >> 1, n = nch * ncx;
  float rr = 0.f;
  if (mode == kRestrictZeroU) {
    for (int q = threadIdx.x; q < n; q += (int)blockDim.x) {
      const int lJ = fdiv(q, dncx), I = q - lJ * ncx;
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int ch = 0; ch < 4; ++ch) {
        const int c = ch >> 1, ly = 2 * lJ + (ch & 1);
        const float4 qq = S.Q[c * (S.ny * S.hx) + (S.y0 + ly) * S.hx + I];
        acc.x += qq.z;
        acc.y += qq.w;
        rr += qq.z * qq.z + qq.w * qq.w;
      }
      fc[coarse_slot(I, lJ, ncx, rowoff, fc_hx, fc_planec)] = acc;
    }
    return rr;
  }
  const int nchild = mode == kRestrictAll ? 4 : 2;
  const int c1 = mode == kRestrictBlack ? 1 : 0;   // colour of the two children when only two are evaluated
  for (int q = threadIdx.x; q < n; q += (int)blockDim.x) {
    const int lJ = fdiv(q, dncx), I = q - lJ * ncx;
    float2 acc = make_float2(0.f, 0.f);
    for (int ch = 0; ch < nchild; ++ch) {
      const int c = nchild == 4 ? ch >> 1 : c1, ly = 2 * lJ + (ch & 1);
      const L0Cell cq = l0_load(S, c * (S.ny * S.hx) + (S.y0 + ly) * S.hx + I);
      float2 nb[4];
      l0_gather(S, c, ly, I, nb);
      const float2 s = nb_dot(cq.t, nb);
      const float2 a = cmul(cinv(make_float2(cq.q.x, cq.q.y)), S.u[c * S.plane + ly * S.hx + I]);
      const float rx = cq.q.z - a.x + s.x, ry = cq.q.w - a.y + s.y;
      acc.x += rx;
      acc.y += ry;
      rr += rx * rx + ry * ry;
    }
    fc[coarse_slot(I, lJ, ncx, rowoff, fc_hx, fc_planec)] = acc;
  }
  return rr;
}

// ---------------------------------------------------------------- staged strip levels (red-black)
__device__ __forceinline__ void rbv_cell(const RBV& S, int c, int ly, int k, float4& t, float2* nb) {
  const int p = (c + ly) & 1, x = 2 * k + p, y = S.y0 + ly;
  const int o = c ^ 1;
  t.x = x + 1 < S.nx ? S.te[c * S.plane + ly * S.hx + k] : 0.f;
  t.y = x > 0 ? S.te[o * S.plane + ly * S.hx + k - 1 + p] : 0.f;
  const int tplane = (S.h + 1) * S.hx;
  t.z = y + 1 < S.ny ? S.ts[o * tplane + (ly + 1) * S.hx + k] : 0.f;
  t.w = y > 0 ? S.ts[c * tplane + ly * S.hx + k] : 0.f;
  rb_gather(S.u, S.u_dn, S.u_up, S.nx, S.ny, S.h, S.y0, S.hx, S.plane, c, ly, k, nb);
}

__device__ __forceinline__ void rbv_half_sweep(const RBV& S, FastDiv dhx, int color) {
  const int n = S.plane;
  for (int q = threadIdx.x; q < n; q += (int)blockDim.x) {
    const int ly = fdiv(q, dhx), k = q - ly * S.hx;
    float4 t;
    float2 nb[4];
    rbv_cell(S, color, ly, k, t, nb);
    float2 r = nb_dot(t, nb);
    const int own = color * S.plane + q;
    const float2 fv = S.f[own];
    r.x += fv.x; r.y += fv.y;
    S.u[own] = cmul(r, S.di[own]);
  }
}

__device__ __forceinline__ void rbv_restrict(const RBV& S, float2* fc, int ncx, FastDiv dncx, int rowoff, int fc_hx,
                                             int fc_planec, int mode) {
  const int nch = S.h >> 1, n = nch * ncx;
  if (mode == kRestrictZeroU) {
    for (int q = threadIdx.x; q < n; q += (int)blockDim.x) {
      const int lJ = fdiv(q, dncx), I = q - lJ * ncx;
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int ch = 0; ch < 4; ++ch) {
        const float2 fv = S.f[(ch >> 1) * S.plane + (2 * lJ + (ch & 1)) * S.hx + I];
        acc.x += fv.x;
        acc.y += fv.y;
      }
      fc[coarse_slot(I, lJ, ncx, rowoff, fc_hx, fc_planec)] = acc;
    }
    return;
  }
  const int nchild = mode == kRestrictAll ? 4 : 2;
  const int c1 = mode == kRestrictBlack ? 1 : 0;
  for (int q = threadIdx.x; q < n; q += (int)blockDim.x) {
    const int lJ = fdiv(q, dncx), I = q - lJ * ncx;
    float2 acc = make_float2(0.f, 0.f);
    for (int ch = 0; ch < nchild; ++ch) {
      const int c = nchild == 4 ? ch >> 1 : c1, ly = 2 * lJ + (ch & 1);
      float4 t;
      float2 nb[4];
      rbv_cell(S, c, ly, I, t, nb);
      const float2 s = nb_dot(t, nb);
      const int own = c * S.plane + ly * S.hx + I;
      const float2 a = cmul(cinv(S.di[own]), S.u[own]);
      const float2 fv = S.f[own];
      acc.x += fv.x - a.x + s.x;
      acc.y += fv.y - a.y + s.y;
    }
    fc[coarse_slot(I, lJ, ncx, rowoff, fc_hx, fc_planec)] = acc;
  }
}

// ---------------------------------------------------------------- staged levels (shared memory)
// neighbour iterates and faces of a staged cell
__device__ __forceinline__ void sv_gather(const SV& S, int x, int y, int ly, int li, float4& t, float2* nb) {
  const float2 z = make_float2(0.f, 0.f);
  t.x = x + 1 < S.nx ? S.te[li] : 0.f;
  t.y = x > 0 ? S.te[li - 1] : 0.f;
  t.z = y + 1 < S.ny ? S.tn[li + S.nx] : 0.f;
  t.w = y > 0 ? S.tn[li] : 0.f;
  nb[0] = x + 1 < S.nx ? S.u[li + 1] : z;
  nb[1] = x > 0 ? S.u[li - 1] : z;
  nb[2] = y + 1 < S.ny ? (ly + 1 < S.h ? S.u[li + S.nx] : S.u_up[x]) : z;
  nb[3] = y > 0 ? (ly > 0 ? S.u[li - S.nx] : S.u_dn[(S.h - 1) * S.nx + x]) : z;
}

// red-black half-sweep of a natural-order level with an even number of columns: thread q takes the q-th
// cell of the colour
__device__ __forceinline__ void sv_half_sweep_even(const SV& S, FastDiv dhx, int color) {
  const int hx = S.nx >> 1, n = S.h * hx;
  for (int q = threadIdx.x; q < n; q += (int)blockDim.x) {
    const int ly = fdiv(q, dhx), y = S.y0 + ly, x = 2 * (q - ly * hx) + ((color + y) & 1);
    const int li = ly * S.nx + x;
    float4 t;
    float2 nb[4];
    sv_gather(S, x, y, ly, li, t, nb);
    float2 r = nb_dot(t, nb);
    const float2 fv = S.f[li];
    r.x += fv.x; r.y += fv.y;
    S.u[li] = cmul(r, S.di[li]);
  }
}

// red-black half-sweep of a whole coarse level (any shape) held by this CTA
__device__ __forceinline__ void sv_half_sweep_full(const SV& S, FastDiv dnx, int color) {
  const int n = S.h * S.nx;
  for (int q = threadIdx.x; q < n; q += (int)blockDim.x) {
    const int ly = fdiv(q, dnx), x = q - ly * S.nx;
    if (((x + S.y0 + ly) & 1) != color) continue;
    const int y = S.y0 + ly, li = q;
    float4 t;
    float2 nb[4];
    sv_gather(S, x, y, ly, li, t, nb);
    float2 r = nb_dot(t, nb);
    const float2 fv = S.f[li];
    r.x += fv.x; r.y += fv.y;
    S.u[li] = cmul(r, S.di[li]);
  }
}

// residual of a coarse level (rank 0, natural order) summed over rx x ry children into the next level's
// right-hand side fc (coarse row J at row J - row0); uc non-null: also clear the next level's iterate;
// red_only (2x2 coarsening, sweep ended black): only the red children, see l0_restrict
__device__ __forceinline__ void sv_restrict(const SV& S, int rx, int ry, float2* fc, float2* uc, int ncx,
                                            FastDiv dncx, int row0, int mode) {
  const int nch = S.h / ry, n = nch * ncx;
  const bool red_only = mode == kRestrictRed;
  for (int q = threadIdx.x; q < n; q += (int)blockDim.x) {
    const int lJ = fdiv(q, dncx), I = q - lJ * ncx;
    float2 acc = make_float2(0.f, 0.f);
    for (int dj = 0; dj < ry; ++dj)
      for (int di = 0; di < rx; ++di) {
        if (mode == kRestrictZeroU) {   // zero iterate: the residual is the right-hand side
          const float2 fv = S.f[(lJ * ry + dj) * S.nx + I * rx + di];
          acc.x += fv.x;
          acc.y += fv.y;
          continue;
        }
        if (red_only && di != dj) continue;
        const int x = I * rx + di, ly = lJ * ry + dj, y = S.y0 + ly, li = ly * S.nx + x;
        float4 t;
        float2 nb[4];
        sv_gather(S, x, y, ly, li, t, nb);
        const float2 s = nb_dot(t, nb);
        const float2 a = cmul(cinv(S.di[li]), S.u[li]);
        const float2 fv = S.f[li];
        acc.x += fv.x - a.x + s.x;
        acc.y += fv.y - a.y + s.y;
      }
    const int C = (S.y0 / ry + lJ - row0) * ncx + I;
    fc[C] = acc;
    if (uc) uc[C] = make_float2(0.f, 0.f);
  }
}

__device__ __forceinline__ float2 cv_get(const CoarseView& V, int I, int J) {
  if (V.full) return V.loc[J * V.nx + I];
  const int lJ = J - V.yc0, slot = ((I + J) & 1) * V.planec + (I >> 1);
  if (lJ < 0) return V.dn[slot + (V.hc - 1) * V.hxc];
  if (lJ >= V.hc) return V.up[slot];
  return V.loc[slot + lJ * V.hxc];
}

// u += bilinear interpolation of the coarse correction (weights 3/4 and 1/4 per axis) on rows
// [y0, y0 + h), one thread per 2x2 block of fine cells: the block's four cells interpolate from the
// same 3x3 coarse neighbourhood, read once.  Across a domain face the coarse neighbour is the cell
// itself, negated for a Dirichlet face (odd reflection) and kept for a Neumann face (even).
// rb: the fine level's arrays are in red-black strip order (strip levels), else natural (rank 0's levels)
__device__ __forceinline__ void strip_prolong(float2* u, int nx, FastDiv dhx, int h, int y0, const CoarseView& V,
                                              int dmask, bool rb) {
  const int ncx = nx >> 1, n = (h >> 1) * ncx;
  const float sxl = (dmask & 1) ? -1.f : 1.f, sxh = (dmask & 2) ? -1.f : 1.f;
  const float syl = (dmask & 4) ? -1.f : 1.f, syh = (dmask & 8) ? -1.f : 1.f;
  for (int q = threadIdx.x; q < n; q += (int)blockDim.x) {
    const int lJ = fdiv(q, dhx), I = q - lJ * ncx, J = (y0 >> 1) + lJ;
    float2 c[3][3];
#pragma unroll
    for (int dy = 0; dy < 3; ++dy) {
      int Jq = J + dy - 1;
      float sy = 1.f;
      if (Jq < 0) { Jq = J; sy = syl; }
      else if (Jq >= V.ny) { Jq = J; sy = syh; }
#pragma unroll
      for (int dx = 0; dx < 3; ++dx) {
        int Iq = I + dx - 1;
        float sx = 1.f;
        if (Iq < 0) { Iq = I; sx = sxl; }
        else if (Iq >= V.nx) { Iq = I; sx = sxh; }
        const float2 v = cv_get(V, Iq, Jq);
        c[dy][dx] = make_float2(sx * sy * v.x, sx * sy * v.y);
      }
    }
#pragma unroll
    for (int bb = 0; bb < 2; ++bb)
#pragma unroll
      for (int aa = 0; aa < 2; ++aa) {
        // along each axis: the own coarse cell (index 1) with 3/4, the nearer neighbour (0 or 2) with 1/4
        const int ny_ = bb ? 2 : 0, nx_ = aa ? 2 : 0;
        const float2 e = make_float2(
            0.5625f * c[1][1].x + 0.1875f * (c[1][nx_].x + c[ny_][1].x) + 0.0625f * c[ny_][nx_].x,
            0.5625f * c[1][1].y + 0.1875f * (c[1][nx_].y + c[ny_][1].y) + 0.0625f * c[ny_][nx_].y);
        float2& v = rb ? u[((aa + bb) & 1) * (h * ncx) + (2 * lJ + bb) * ncx + I] : u[(2 * lJ + bb) * nx + 2 * I + aa];
        v.x += e.x;
        v.y += e.y;
      }
  }
}

// sum of v over the CTA's threads into *dst (thread 0's view after the call)
__device__ __forceinline__ void block_sum(float v, float* red, double* dst) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) *dst = (double)v;
  }
}

// sum of v over the cluster's threads; identical on every CTA (ranks added in order)
__device__ __forceinline__ double cluster_sum(cg::cluster_group& cl, int cs, float v, float* red, double* part,
                                              int slot, double* bcast) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) part[slot] = (double)v;
  }
  cl.sync();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int q = 0; q < cs; ++q) s += *cl.map_shared_rank(&part[slot], q);
    *bcast = s;
  }
  __syncthreads();
  return *bcast;
}

__global__ void __launch_bounds__(kIT, 1) k_inner_cluster(const __grid_constant__ InnerArgs a) {
  extern __shared__ float4 dsm4[];
  char* smb = reinterpret_cast<char*>(dsm4);
  __shared__ Level sL[kMaxLevels];
  __shared__ float red[32];
  __shared__ double part[2];
  __shared__ double bcast;
  __shared__ double vpart[2];           // per-cycle fine residual norm^2 of this CTA's rows
  __shared__ int vstop;                 // 1: this V-cycle ends the round
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int cs = a.cs;                  // CTAs per cluster (8 or 16)
  const int nthr = (int)blockDim.x;     // threads per CTA
  const int b = blockIdx.x / cs;
  const Batch& bt = a.bt;
  if (!bt.active[b]) return;            // the same answer on every CTA of the cluster
  const int tid = threadIdx.x;
  if (tid < a.nlev) sL[tid] = a.levels[tid];
  __syncthreads();
  const int j = *bt.jdev;
  const double2 td = bt.tau_cur[b];
  const float2 tau = make_float2((float)td.x, (float)td.y);
  const df taur = df_from_double(td.x), taui = df_from_double(td.y);
  const int R = a.rounds, R1 = R + 1;
  const double itol2 = bt.itol2[b];

  // views of the levels: strips [1, ld) in red-black order (rows of this rank), whole coarse levels
  // [ld, nlev) in natural order (rank 0)
  auto rbview = [&](int l) {
    const Level& L = sL[l];
    const LevOff& o = a.off[l];
    RBV S;
    S.nx = L.nx; S.ny = L.ny; S.h = L.ny / cs; S.y0 = rank * S.h; S.hx = L.nx >> 1; S.plane = S.h * S.hx;
    S.u = reinterpret_cast<float2*>(smb + o.u);
    S.f = reinterpret_cast<float2*>(smb + o.f);
    S.te = reinterpret_cast<float*>(smb + o.te);
    S.ts = reinterpret_cast<float*>(smb + o.tn);
    S.di = reinterpret_cast<float2*>(smb + o.di);
    S.u_dn = rank > 0 ? cl.map_shared_rank(S.u, rank - 1) : nullptr;
    S.u_up = rank + 1 < cs ? cl.map_shared_rank(S.u, rank + 1) : nullptr;
    return S;
  };
  auto sview = [&](int l) {
    const Level& L = sL[l];
    const LevOff& o = a.off[l];
    SV S;
    S.nx = L.nx; S.ny = L.ny; S.h = L.ny; S.y0 = 0;
    S.u = reinterpret_cast<float2*>(smb + o.u);
    S.f = reinterpret_cast<float2*>(smb + o.f);
    S.te = reinterpret_cast<float*>(smb + o.te);
    S.tn = reinterpret_cast<float*>(smb + o.tn);
    S.di = reinterpret_cast<float2*>(smb + o.di);
    S.u_dn = nullptr;
    S.u_up = nullptr;
    return S;
  };
  auto cview = [&](int l) {   // view of level l + 1 from level l
    const Level& Lc = sL[l + 1];
    CoarseView V;
    V.nx = Lc.nx; V.ny = Lc.ny;
    float2* uc = reinterpret_cast<float2*>(smb + a.off[l + 1].u);
    if (l + 1 == a.ld) {
      V.full = 1; V.hc = Lc.ny; V.yc0 = 0; V.hxc = 0; V.planec = 0;
      V.loc = cl.map_shared_rank(uc, 0);
      V.dn = nullptr; V.up = nullptr;
    } else {
      V.full = 0; V.hc = Lc.ny / cs; V.yc0 = rank * V.hc; V.hxc = Lc.nx >> 1; V.planec = V.hc * V.hxc;
      V.loc = uc;
      V.dn = rank > 0 ? cl.map_shared_rank(uc, rank - 1) : nullptr;
      V.up = rank + 1 < cs ? cl.map_shared_rank(uc, rank + 1) : nullptr;
    }
    return V;
  };

  // stage the coefficients of the strip levels >= 1 (own rows, red-black order) and, in rank 0, of the
  // coarse levels (natural order); clear every coarse iterate (each V-cycle clears them again after use)
  for (int l = 1; l < a.ld; ++l) {
    const Level& L = sL[l];
    const RBV S = rbview(l);
    const int tplane = (S.h + 1) * S.hx;
    for (int q = tid; q < S.h * S.nx; q += nthr) {
      const int ly = q / S.nx, x = q - ly * S.nx, c = (S.y0 + ly) * S.nx + x;
      const int rbi = ((x + ly) & 1) * S.plane + ly * S.hx + (x >> 1);
      S.te[rbi] = L.Te[c];
      const float mm = L.m[c];
      S.di[rbi] = cinv(make_float2(L.D[c] + tau.x * mm, tau.y * mm));
      S.u[rbi] = make_float2(0.f, 0.f);
    }
    for (int q = tid; q < (S.h + 1) * S.nx; q += nthr) {   // south faces of local rows 0 .. h
      const int r = q / S.nx, x = q - r * S.nx, y = S.y0 + r;
      S.ts[((x + r) & 1) * tplane + r * S.hx + (x >> 1)] = (y >= 1 && y - 1 < S.ny) ? L.Tn[(y - 1) * S.nx + x] : 0.f;
    }
  }
  if (rank == 0)
    for (int l = a.ld; l < a.nlev; ++l) {
      const Level& L = sL[l];
      const SV S = sview(l);
      const int n = S.h * S.nx;
      for (int q = tid; q < n; q += nthr) {
        S.te[q] = L.Te[q];
        S.tn[S.nx + q] = L.Tn[q];
        const float mm = L.m[q];
        S.di[q] = cinv(make_float2(L.D[q] + tau.x * mm, tau.y * mm));
        S.u[q] = make_float2(0.f, 0.f);
      }
      for (int x = tid; x < S.nx; x += nthr) S.tn[x] = 0.f;
    }
  L0V S0;
  float4* q0 = a.q4 + (size_t)b * bt.N;
  {
    const Level& L = sL[0];
    S0.nx = L.nx; S0.ny = L.ny; S0.h = L.ny / cs; S0.y0 = rank * S0.h;
    S0.hx = L.nx >> 1; S0.plane = S0.h * S0.hx;
    S0.P = a.p4;
    S0.Q = q0;
    S0.gl = a.u0g != nullptr;
    if (S0.gl) {
      // this rank's block of the basis's array; the neighbour ranks' blocks lie just before and after
      S0.u = a.u0g + (size_t)b * bt.N + (size_t)rank * S0.h * S0.nx;
      S0.u_dn = rank > 0 ? S0.u - S0.h * S0.nx : nullptr;
      S0.u_up = rank + 1 < cs ? S0.u + S0.h * S0.nx : nullptr;
    } else {
      S0.u = reinterpret_cast<float2*>(smb + a.off[0].u);
      S0.u_dn = rank > 0 ? cl.map_shared_rank(S0.u, rank - 1) : nullptr;
      S0.u_up = rank + 1 < cs ? cl.map_shared_rank(S0.u, rank + 1) : nullptr;
    }
    // inverse diagonal of this basis's shift on this CTA's rows (right-hand sides follow every round)
    for (int q = tid; q < S0.h * S0.nx; q += nthr) {
      const int c = S0.y0 * S0.nx + q;
      const float mm = L.m[c];
      const float2 di = cinv(make_float2(L.D[c] + tau.x * mm, tau.y * mm));
      q0[rb_index(c % S0.nx, c / S0.nx, S0.nx, (int)(bt.N >> 1))] = make_float4(di.x, di.y, 0.f, 0.f);
    }
  }
  __syncthreads();
  cl.sync();   // every CTA of the cluster is running and initialised before any remote access

  const int c0 = S0.y0 * S0.nx, n0 = S0.h * S0.nx;
  const size_t vb = ((size_t)b * (bt.maxit + 1) + j) * bt.N;
  const size_t ub = ((size_t)b * bt.maxit + j) * bt.N;
  int slot = 0;
  unsigned long long n_res = 0, n_cyc = 0;   // rank 0, thread 0: work counters, added once at the end
  for (int r = 0; r <= R; ++r) {
    // df32 residual of the current u_j on this CTA's rows; it is the next round's right-hand side
    // (two cells per pass, both evaluated before either is stored, so their loads overlap)
    float acc = 0.f;
    for (int q0i = tid; q0i < n0; q0i += 2 * nthr) {
      cdf rr[2];
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const int q = q0i + k * nthr;
        if (q < n0) {
          const int c = c0 + q;
          rr[k] = load_cdf(bt.V_hi, bt.V_lo, vb + c);
          if (r > 0) rr[k] = cdf_sub(rr[k], apply_exact(a.fe, bt.U_hi + ub, lo_at(bt.U_lo, ub), c, taur, taui));
        }
      }
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const int q = q0i + k * nthr;
        if (q < n0) {
          if (r < R) {
            const int ly = fdiv(q, a.dnx[0]), x = q - ly * S0.nx;
            reinterpret_cast<float2*>(q0 + rb_index(x, S0.y0 + ly, S0.nx, (int)(bt.N >> 1)))[1] =
                make_float2(rr[k].re.hi, rr[k].im.hi);
            S0.u[q] = make_float2(0.f, 0.f);
          }
          acc += rr[k].re.hi * rr[k].re.hi + rr[k].im.hi * rr[k].im.hi;
        }
      }
    }
    const double rn2 = cluster_sum(cl, cs, acc, red, part, slot, &bcast);
    slot ^= 1;
    const bool done = (r == R) || (rn2 <= itol2);
    if (rank == 0 && tid == 0) {
      bt.rnorm2[b * R1 + r] = rn2;
      if (r < R && done) bt.rnorm2[b * R1 + R] = rn2;   // u_j is final: its residual is this one
      n_res += (unsigned long long)bt.N;
    }
    if (done) {
      if (r == 0)   // v_j itself is below the tolerance: u_j = 0
        for (int q = tid; q < n0; q += nthr) {
          bt.U_hi[ub + c0 + q] = make_float2(0.f, 0.f);
          if (bt.U_lo) bt.U_lo[ub + c0 + q] = make_float2(0.f, 0.f);
        }
      break;
    }
    // V-cycles until the fine residual after pre-smoothing is below the round's goal: the inner
    // tolerance, or the float32 floor (1e-11 of the round's right-hand side, squared norms), at most a.cycles
    const double goal2 = fmax(itol2, 1e-11 * rn2);
    for (int cy = 0; cy < a.cycles; ++cy) {
      // ---- down: pre-smoothing, residual, restriction on the strip levels
      for (int l = 0; l < a.ld; ++l) {
        const bool last = (l + 1 == a.ld);
        float2* fc = reinterpret_cast<float2*>(smb + a.off[l + 1].f);
        if (last) fc = cl.map_shared_rank(fc, 0);
        const int ncx = sL[l + 1].nx;
        if (l == 0) {
          for (int h = 0; h < 2 * a.npre; ++h) {
            l0_half_sweep(S0, a.dhx[0], h & 1);
            cl.sync();
          }
          const int fhx = last ? 0 : sL[1].nx >> 1, fplane = last ? 0 : (sL[1].ny / cs) * fhx;
          // after pre-smoothing (ending black) only the red children carry a residual; without it, the
          // first cycle of a round starts from u = 0 and every later one follows post-smoothing that
          // ended with a red half-sweep
          const int mode = a.npre > 0 ? kRestrictRed : cy == 0 ? kRestrictZeroU
                         : a.npost > 0 ? kRestrictBlack : kRestrictAll;
          const float rr = l0_restrict(S0, fc, ncx, a.dnx[1], S0.y0 / 2, fhx, fplane, mode);
          block_sum(rr, red, &vpart[cy & 1]);
        } else {
          const RBV S = rbview(l);
          for (int h = 0; h < 2 * a.npre; ++h) {
            rbv_half_sweep(S, a.dhx[l], h & 1);
            cl.sync();
          }
          const int fhx = last ? 0 : sL[l + 1].nx >> 1, fplane = last ? 0 : (sL[l + 1].ny / cs) * fhx;
          // the coarser strip levels start every cycle from u = 0 (cleared after the last prolongation)
          rbv_restrict(S, fc, ncx, a.dnx[l + 1], S.y0 / 2, fhx, fplane, a.npre > 0 ? kRestrictRed : kRestrictZeroU);
        }
        __syncthreads();   // the next level's sweeps read right-hand sides written by other threads
      }
      cl.sync();   // rank 0 holds the whole restricted residual of level ld
      if (tid == 0) {
        double s2 = 0.0;
        for (int q = 0; q < cs; ++q) s2 += *cl.map_shared_rank(&vpart[cy & 1], q);
        vstop = s2 <= goal2;
        n_cyc += (unsigned long long)bt.N;
      }
      // ---- coarse levels in rank 0
      // (levels coarsened 2x2 use the colour-compact sweep, red-only restriction and block prolongation)
      if (rank == 0)
        for (int l = a.ld; l < a.nlev - 1; ++l) {
          const SV S = sview(l);
          const bool q22 = sL[l].rx == 2 && sL[l].ry == 2;
          for (int h = 0; h < 2 * a.npre; ++h) {
            if (q22) sv_half_sweep_even(S, a.dhx[l], h & 1);
            else sv_half_sweep_full(S, a.dnx[l], h & 1);
            __syncthreads();
          }
          const Level& Lc = sL[l + 1];
          sv_restrict(S, sL[l].rx, sL[l].ry, reinterpret_cast<float2*>(smb + a.off[l + 1].f),
                      reinterpret_cast<float2*>(smb + a.off[l + 1].u), Lc.nx, a.dnx[l + 1], 0,
                      a.npre == 0 ? kRestrictZeroU : q22 ? kRestrictRed : kRestrictAll);
          __syncthreads();
        }
      if (a.coarse_direct) {
        // u_c = A_c^{-1} f_c; every rank takes a slice of the rows of the dense inverse
        cl.sync();
        const int lc = a.nlev - 1, N = sL[lc].N;
        const float2* fr = cl.map_shared_rank(reinterpret_cast<float2*>(smb + a.off[lc].f), 0);
        float2* ur = cl.map_shared_rank(reinterpret_cast<float2*>(smb + a.off[lc].u), 0);
        float2* rhs = reinterpret_cast<float2*>(smb + a.off_rhs);
        for (int i = tid; i < N; i += nthr) rhs[i] = fr[i];
        __syncthreads();
        const float2* A = bt.coarse_inv + (size_t)bt.tau_slot[b] * N * N;
        const int warp = tid >> 5, lane = tid & 31;
        for (int row = rank * (nthr / 32) + warp; row < N; row += cs * (nthr / 32)) {
          const float2* Ar = A + (size_t)row * N;
          float sx = 0.f, sy = 0.f;
          for (int c = lane; c < N; c += 32) {
            const float2 av = Ar[c], x = rhs[c];
            sx += av.x * x.x - av.y * x.y;
            sy += av.x * x.y + av.y * x.x;
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            sx += __shfl_xor_sync(0xffffffffu, sx, o);
            sy += __shfl_xor_sync(0xffffffffu, sy, o);
          }
          if (lane == 0) ur[row] = make_float2(sx, sy);
        }
        cl.sync();
      } else if (rank == 0) {
        const SV S = sview(a.nlev - 1);
        for (int h = 0; h < 2 * kCoarseSweeps; ++h) {
          sv_half_sweep_full(S, a.dnx[a.nlev - 1], h & 1);
          __syncthreads();
        }
      }
      if (rank == 0)
        for (int l = a.nlev - 2; l >= a.ld; --l) {
          const SV S = sview(l);
          const bool q22 = sL[l].rx == 2 && sL[l].ry == 2;
          const float2* uc = reinterpret_cast<const float2*>(smb + a.off[l + 1].u);
          if (q22) {
            CoarseView V;
            V.nx = sL[l + 1].nx; V.ny = sL[l + 1].ny;
            V.full = 1; V.hc = V.ny; V.yc0 = 0; V.hxc = 0; V.planec = 0;
            V.loc = uc; V.dn = nullptr; V.up = nullptr;
            strip_prolong(S.u, S.nx, a.dhx[l], S.h, 0, V, a.dmask, false);
          } else {
            for (int c = tid; c < sL[l].N; c += nthr) prolong_cell(sL[l], sL[l + 1], S.u, uc, c, a.dmask);
          }
          __syncthreads();
          for (int h = 0; h < 2 * a.npost; ++h) {
            if (q22) sv_half_sweep_even(S, a.dhx[l], (h + 1) & 1);
            else sv_half_sweep_full(S, a.dnx[l], (h + 1) & 1);
            __syncthreads();
          }
        }
      cl.sync();   // rank 0's level ld holds the coarse correction
      // ---- up: prolongation, correction, post-smoothing on the strip levels
      for (int l = a.ld - 1; l >= 0; --l) {
        const CoarseView V = cview(l);
        if (l == 0) strip_prolong(S0.u, S0.nx, a.dhx[0], S0.h, S0.y0, V, a.dmask, true);
        else {
          const RBV S = rbview(l);
          strip_prolong(S.u, S.nx, a.dhx[l], S.h, S.y0, V, a.dmask, true);
        }
        cl.sync();
        // every rank has read the coarse iterate: clear it for the next cycle
        if (l + 1 < a.ld) {
          const RBV C = rbview(l + 1);
          for (int q = tid; q < C.h * C.nx; q += nthr) C.u[q] = make_float2(0.f, 0.f);
        } else if (rank == 0) {
          const SV C = sview(l + 1);
          for (int q = tid; q < C.h * C.nx; q += nthr) C.u[q] = make_float2(0.f, 0.f);
        }
        for (int h = 0; h < 2 * a.npost; ++h) {
          if (l == 0) l0_half_sweep(S0, a.dhx[0], (h + 1) & 1);
          else rbv_half_sweep(rbview(l), a.dhx[l], (h + 1) & 1);
          cl.sync();
        }
      }
      if (vstop) break;   // the same on every CTA: all read the same partial sums in the same order
    }
    // u_j += d (df32) on this CTA's rows; the next residual reads the neighbours' rows
    for (int q = tid; q < n0; q += nthr) {
      const size_t ui = ub + c0 + q;
      const int ly = fdiv(q, a.dnx[0]), x = q - ly * S0.nx;
      const float2 d = S0.u[((x + ly) & 1) * S0.plane + ly * S0.hx + (x >> 1)];
      if (r == 0) {
        bt.U_hi[ui] = d;
        if (bt.U_lo) bt.U_lo[ui] = make_float2(0.f, 0.f);
      } else {
        cdf u = load_cdf(bt.U_hi, bt.U_lo, ui);
        u.re = df_add_f(u.re, d.x);
        u.im = df_add_f(u.im, d.y);
        store_cdf(bt.U_hi, bt.U_lo, ui, u);
      }
    }
    cl.sync();
  }
  if (rank == 0 && tid == 0) {
    atomicAdd(&bt.work[KC_EXACT_RES], n_res);
    atomicAdd(&bt.work[KC_INNER], n_cyc);
  }
  cl.sync();   // no CTA leaves while another may still read its shared memory
}

static size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

int inner_cluster_plan(const MGHost& mg, InnerPlan& p, int cs, int threads, int u0_global) {
  p.ok = 0;
  p.cs = cs;
  p.threads = threads;
  p.u0_global = u0_global;
  // levels [ld, nlev) live whole in rank 0 (their arrays are reserved in every CTA): those of at most
  // kCoarseCells cells; in the two-CTAs-per-SM forms (16-CTA clusters, or the finest iterate in global
  // memory) the levels of more than 256 cells among them are split into strips too where they split
  // evenly
  auto splits = [&](int l) {
    if (l + 1 >= mg.nlev) return false;
    const Level& L = mg.h_levels[l];
    const Level& Lc = mg.h_levels[l + 1];
    return L.rx == 2 && L.ry == 2 && L.rz == 1 && L.nx % 2 == 0 && L.ny % (2 * cs) == 0 && Lc.nx * 2 == L.nx &&
           Lc.ny * 2 == L.ny;
  };
  int ld = mg.lc;
  if (cs > 8 || u0_global)
    while (ld < mg.nlev && mg.h_levels[ld].N > 256 && splits(ld)) ++ld;
  if (ld < 1 || ld >= mg.nlev) return 0;
  for (int l = 0; l < mg.nlev; ++l)
    if (mg.h_levels[l].nz != 1) return 0;
  for (int l = 0; l < ld; ++l) {
    const Level& L = mg.h_levels[l];
    const Level& Lc = mg.h_levels[l + 1];
    if (L.rx != 2 || L.ry != 2 || L.rz != 1) return 0;
    if (L.nx % 2 != 0 || L.ny % (2 * cs) != 0) return 0;
    if (Lc.nx * 2 != L.nx || Lc.ny * 2 != L.ny) return 0;
  }
  size_t cur = 0;
  auto take = [&](size_t bytes) { const size_t o = cur; cur = align16(cur + bytes); return (int)o; };
  for (int l = 0; l < mg.nlev; ++l) {
    const Level& L = mg.h_levels[l];
    const size_t h = l < ld ? (size_t)L.ny / cs : (size_t)L.ny;
    const size_t n = h * L.nx;
    p.off_u[l] = take(l == 0 && u0_global ? 0 : n * sizeof(float2));
    if (l == 0) {
      p.off_f[l] = p.off_te[l] = p.off_tn[l] = p.off_di[l] = 0;
      continue;
    }
    p.off_f[l] = take(n * sizeof(float2));
    p.off_te[l] = take(n * sizeof(float));
    p.off_tn[l] = take((h + 1) * L.nx * sizeof(float));
    p.off_di[l] = take(n * sizeof(float2));
  }
  p.off_rhs = take(mg.coarse_direct ? (size_t)mg.h_levels[mg.nlev - 1].N * sizeof(float2) : 0);
  p.smem = cur;
  if (p.smem > kInnerSmemMax) return 0;
  // the attribute belongs to the kernel, not to this grid: always the ceiling, so that contexts with
  // different grids can launch it in any order
  if (cudaFuncSetAttribute(k_inner_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kInnerSmemMax) !=
      cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (cs > 8 && cudaFuncSetAttribute(k_inner_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  // the cluster must fit on the device (cs CTAs with this much shared memory each)
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cs);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = p.smem;
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeClusterDimension;
  attr.val.clusterDim.x = cs; attr.val.clusterDim.y = 1; attr.val.clusterDim.z = 1;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  int nclusters = 0;
  if (cudaOccupancyMaxActiveClusters(&nclusters, k_inner_cluster, &cfg) != cudaSuccess || nclusters < 1) {
    cudaGetLastError();
    return 0;
  }
  p.ld = ld;
  p.max_clusters = nclusters;
  p.ok = 1;
  return 1;
}

int launch_inner_cluster(const MGHost& mg, const InnerPlan& p, const Batch& bt, const FineExact& fe, float4* q4,
                         float2* u0, int cycles, cudaStream_t st, Prof* pf) {
  InnerArgs a;
  a.bt = bt;
  a.fe = fe;
  a.levels = mg.d_levels;
  a.p4 = p.p4;
  a.q4 = q4;
  a.nlev = mg.nlev;
  a.ld = p.ld;
  a.npre = mg.npre;
  a.npost = mg.npost;
  a.dmask = mg.dmask;
  a.coarse_direct = mg.coarse_direct;
  a.rounds = bt.rounds;
  a.cycles = cycles;
  for (int l = 0; l < kMaxLevels; ++l)
    a.off[l] = LevOff{p.off_u[l], p.off_f[l], p.off_te[l], p.off_tn[l], p.off_di[l]};
  a.off_rhs = p.off_rhs;
  for (int l = 0; l < kMaxLevels; ++l) {
    const int nx = l < mg.nlev ? mg.h_levels[l].nx : 2;
    a.dnx[l] = make_fastdiv((uint32_t)nx);
    a.dhx[l] = make_fastdiv((uint32_t)(nx / 2 > 0 ? nx / 2 : 1));
  }
  a.cs = p.cs;
  a.u0g = p.u0_global ? u0 : nullptr;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(bt.nb * p.cs));
  cfg.blockDim = dim3((unsigned)p.threads);
  cfg.dynamicSmemBytes = p.smem;
  cfg.stream = st;
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeClusterDimension;
  attr.val.clusterDim.x = p.cs; attr.val.clusterDim.y = 1; attr.val.clusterDim.z = 1;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  prof_begin(pf, KC_INNER, st);
  const cudaError_t e = cudaLaunchKernelEx(&cfg, k_inner_cluster, a);
  prof_end(pf, KC_INNER, st);
  return (e == cudaSuccess && cudaGetLastError() == cudaSuccess) ? 0 : -3;
}

}  // namespace lt
