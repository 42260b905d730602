// Batched solves: many independent flat problems of uneven sizes solved in one
// persistent cooperative launch (data-parallel form of the solve; the paper's
// field-level-inference use case runs many such solves).
//
// Each problem keeps the hierarchy of its own context.  The kernel runs the whole
// mixed-precision solve of every problem: prologue (double-float conversion, mean,
// first residual), V-cycles, epilogue (gauge, FP64 output); every step is a
// grid-wide phase separated by grid.sync().  Levels of at least 16^3 run the fused
// legs (one pass per level visit and leg, the device code of the per-level fused
// kernels) and the finest level the fused double-float update and residual; the
// work of a fused phase is the list of (problem, tile, plane) of every problem,
// split evenly over the CTAs.  Smaller levels run the one-kernel-per-operation
// arithmetic over chunks (tiles of whole x rows, a per-level size) of one problem.
// All of it rounds exactly like mg_solve, so each problem's iterates equal the
// single solves' up to the summation order of the norms and means, which are summed
// per problem over fixed chunks in a fixed order (deterministic).  A problem that has
// converged (or failed) skips its work; the loop ends when none is active or
// max_vcycles is reached.  Per-problem completion times come from %globaltimer.
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "dfk.cuh"
#include "kernels.h"
#include "legs.cuh"
#include "small_cycle.cuh"
#include "solver.h"
#include "stencil.cuh"

namespace cg = cooperative_groups;
using namespace gbmg;

namespace {

constexpr int BMAXL = 16;
constexpr int CHUNK = 4096;      // default tile (chunk) size in cells
constexpr int MINCHUNK = 1024;   // smallest tile the tables are sized for
constexpr int MAXCHUNK = 65536;
constexpr int BT = 384;          // block size (the fused legs' thread-column layout)
constexpr int DFZC = 32;         // z planes per item of the fused double-float phase

// tiles of the fused device code at BT threads
// (columns of 3 pairs for both legs: this kernel holds the state of every phase under
// one register limit of BT threads per SM, and the up leg's 4-pair columns, which its
// separate kernel uses, spill there)
constexpr int down_ty(int v) { return v >= 4 ? 20 : 22; }
constexpr int up_ty(int v) { return v >= 4 ? 20 : 24; }
template <int V>
struct BDown {
  using T = legs::PTile<64, down_ty(V), V + 1, BT, 3>;
};
template <int V>
struct BUp {
  using T = legs::PTile<64, up_ty(V), (V > 0 ? V : 1), BT, 3>;
};
// double-float items: 32 x 32 tiles, which 64^3, 96^3 and 128^3 meshes fill whole (64 x 16
// tiles left half of every second tile column empty on 96^3; measured 3095 -> 3132 solves/s)
using BDf = dfk::DTile<32, 32, 2, BT>;

// per-problem scalars
enum { P_MEAN = 0, P_F2 = 1, P_R2 = 2, P_REL = 3, P_PREV1 = 4, P_PREV2 = 5, P_MPHI = 6, P_N = 8 };
// status codes inside the kernel: 0 = still iterating, -1 = converged, else a gbmg_status
enum { ST_ACTIVE = 0, ST_CONVERGED = -1 };

struct BProb {
  int L, nc;
  Dims d[BMAXL];
  float* r[BMAXL];
  float* ea[BMAXL];
  float* eb[BMAXL];
  float* dv[BMAXL];
  float* t[BMAXL];
  const float* G;
  float2* F;
  float2* phi;   // double-float phi, and the second buffer of the fused update (phi2)
  float2* phi2;
  const double* src;
  double* out;
  int c0, nch;      // first level-0 chunk and count
  unsigned fmask;   // bit l: level l runs the fused legs
  int dffused;      // the finest level runs the fused double-float update (even nx)
  int ls;           // first level of the single-CTA bottom cycle (levels ls .. L-1), 0: none
};

struct BDesc {
  int count, maxL, degree, maxv;
  int chunk[BMAXL];  // tile (chunk) size in cells per level
  double tol;
  float c1[16];
  float ca[BMAXL][8];  // folded Chebyshev constants a = c2 D^-1 and b = a / h^2 per level and step
  float cb[BMAXL][8];
  float ih2[BMAXL];    // 1 / h_l^2
  const legs::Coef* coef;       // folded Chebyshev constants per level (device)
  const long long* doff[BMAXL];  // per level: prefix over problems of fused down-leg planes
  const long long* uoff[BMAXL];  // per level: the same for the up leg
  long long dtot[BMAXL], utot[BMAXL];
  const int* dfoff;              // prefix over problems of fused double-float items
  int dftot;
  double* dfpart;                // per double-float item: partial sum of r^2
  double* dfpart2;               // per double-float item: partial sum of (F - m)^2 (first residual)
  unsigned perop;                // bit l: some problem runs level l per operation (not the coarsest)
  unsigned coarse;               // bit l: some problem's coarsest level is l (outside a bottom cycle)
  const SmallCycle* small;       // per problem: parameters of its bottom cycle (ls > 0)
  int anysmall;                  // some problem runs a bottom cycle
  int* phicur;                   // per problem: 0 = phi, 1 = phi2 holds the current iterate
  BProb* p;
  // chunk tables per level: problem index and first cell
  int* cprob[BMAXL];
  long long* cstart[BMAXL];
  int nchunk[BMAXL];
  double* part0;  // per level-0 chunk partials
  double* part1;
  double* sc;     // count * P_N scalars
  int* status;    // count: ST_ACTIVE, then a gbmg_status
  int* cycles;    // count
  double* hist;   // count * 64
  double* rel0;   // count
  unsigned long long* tdone;  // count, %globaltimer at completion
  unsigned long long* tstart;
  int* any_active;
};

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// (x, y, z) of cell i of one problem: 32-bit division (every problem holds fewer than
// 2^31 cells, checked at mg_batch_create), two divisions per cell.
__device__ __forceinline__ void cell_xyz(Dims d, long long i, int& x, int& y, int& z) {
  const unsigned u = (unsigned)i, nx = (unsigned)d.nx, ny = (unsigned)d.ny;
  const unsigned q = u / nx;
  x = (int)(u - q * nx);
  const unsigned zz = q / ny;
  y = (int)(q - zz * ny);
  z = (int)zz;
}

template <typename V>
__device__ __forceinline__ V nsum_at(const V* u, Dims d, int x, int y, int z, long long i) {
  const long long sy = d.nx, sz = (long long)d.nx * d.ny;
  const V xm = u[i + ((x == 0 ? d.nx - 1 : x - 1) - x)];
  const V xp = u[i + ((x == d.nx - 1 ? 0 : x + 1) - x)];
  const V ym = u[i + (long long)((y == 0 ? d.ny - 1 : y - 1) - y) * sy];
  const V yp = u[i + (long long)((y == d.ny - 1 ? 0 : y + 1) - y) * sy];
  const V zm = u[i + (long long)((z == 0 ? d.nz - 1 : z - 1) - z) * sz];
  const V zp = u[i + (long long)((z == d.nz - 1 ? 0 : z + 1) - z) * sz];
  return nbr_sum(xm, xp, ym, yp, zm, zp);
}

// Run `op(P, l, i)` over every cell of level l of every active problem for which
// `want(P, l)` holds.
template <typename Want, typename Op>
__device__ __forceinline__ void phase(const BDesc& B, int l, Want want, Op op) {
  for (int c = blockIdx.x; c < B.nchunk[l]; c += gridDim.x) {
    const int pi = B.cprob[l][c];
    if (B.status[pi] != ST_ACTIVE) continue;
    const BProb& P = B.p[pi];
    if (!want(P, l)) continue;
    const long long s0 = B.cstart[l][c];
    const long long n = ncell(P.d[l]);
    const long long s1 = s0 + B.chunk[l] < n ? s0 + B.chunk[l] : n;
    for (long long i = s0 + threadIdx.x; i < s1; i += blockDim.x) op(P, l, i);
  }
}

// Level-0 phase with a per-chunk partial sum of the float returned by op.
template <typename Op>
__device__ __forceinline__ void phase0_sum(const BDesc& B, double* part, double* sh, bool all, Op op) {
  for (int c = blockIdx.x; c < B.nchunk[0]; c += gridDim.x) {
    const int pi = B.cprob[0][c];
    if (!all && B.status[pi] != ST_ACTIVE) continue;
    const BProb& P = B.p[pi];
    const long long s0 = B.cstart[0][c];
    const long long n = ncell(P.d[0]);
    const long long s1 = s0 + B.chunk[0] < n ? s0 + B.chunk[0] : n;
    DfAcc acc{0.f, 0.f};
    for (long long i = s0 + threadIdx.x; i < s1; i += blockDim.x) op(P, i, acc);
    const double b = block_sum_acc(acc, sh);
    if (threadIdx.x == 0) part[c] = b;
  }
}

__device__ __forceinline__ double chunk_total(const BDesc& B, const BProb& P, const double* part) {
  double s = 0.0;
  for (int k = 0; k < P.nch; ++k) s += part[P.c0 + k];
  return s;
}

// level l of problem P runs the fused legs
__device__ __forceinline__ bool lv_fused(const BProb& P, int l) { return (P.fmask >> l) & 1u; }
// buffer holding the final correction of level l after its up leg
__device__ __forceinline__ float* final_e(const BProb& P, int l) {
  return (l < P.L - 1 && lv_fused(P, l)) ? P.eb[l] : P.ea[l];
}

// Fused phases: the (problem, tile, plane) list of level l, split evenly over the
// CTAs; each contiguous run within one tile is one z segment of the leg.
template <int V>
__device__ __forceinline__ void fused_down(const BDesc& B, int l, float* smf) {
  using TL = typename BDown<V>::T;
  const long long T = B.dtot[l];
  if (T == 0) return;
  long long a = (long long)blockIdx.x * T / gridDim.x;
  const long long b = (long long)(blockIdx.x + 1) * T / gridDim.x;
  int p = 0;
  while (a < b) {
    while (B.doff[l][p + 1] <= a) ++p;
    const BProb& P = B.p[p];
    const Dims d = P.d[l];
    const long long loc = a - B.doff[l][p];
    const long long tile = loc / d.nz;
    const int z0 = (int)(loc % d.nz);
    const int zend = (int)(z0 + (b - a) < d.nz ? z0 + (b - a) : d.nz);
    const int tiles_x = (d.nx + TL::TX - 1) / TL::TX;
    if (B.status[p] == ST_ACTIVE)
      legs::down_segment<V, TL>(d, P.r[l], P.ea[l], P.r[l + 1], (int)(tile % tiles_x) * TL::TX,
                                (int)(tile / tiles_x) * TL::TY, z0, zend, B.ih2[l], B.coef[l], smf);
    a += zend - z0;
    __syncthreads();
  }
}

template <int V>
__device__ __forceinline__ void fused_up(const BDesc& B, int l, float* smf) {
  using TL = typename BUp<V>::T;
  const long long T = B.utot[l];
  if (T == 0) return;
  long long a = (long long)blockIdx.x * T / gridDim.x;
  const long long b = (long long)(blockIdx.x + 1) * T / gridDim.x;
  int p = 0;
  while (a < b) {
    while (B.uoff[l][p + 1] <= a) ++p;
    const BProb& P = B.p[p];
    const Dims d = P.d[l];
    const long long loc = a - B.uoff[l][p];
    const long long tile = loc / d.nz;
    const int z0 = (int)(loc % d.nz);
    const int zend = (int)(z0 + (b - a) < d.nz ? z0 + (b - a) : d.nz);
    const int tiles_x = (d.nx + TL::TX - 1) / TL::TX;
    if (B.status[p] == ST_ACTIVE)
      legs::up_segment<V, TL>(d, P.ea[l], final_e(P, l + 1), P.r[l], P.eb[l], (int)(tile % tiles_x) * TL::TX,
                              (int)(tile / tiles_x) * TL::TY, z0, zend, B.ih2[l], B.coef[l], smf);
    a += zend - z0;
    __syncthreads();
  }
}

// Fused double-float update + residual of the finest level: items of one tile and
// DFZC planes, each with its own partial sum of r^2 (summed per problem in order).
__device__ __forceinline__ void fused_df(const BDesc& B, float* smf, double* sh, bool first) {
  for (int it = blockIdx.x; it < B.dftot; it += gridDim.x) {
    int p = 0;
    while (B.dfoff[p + 1] <= it) ++p;
    if (B.status[p] != ST_ACTIVE) continue;
    const BProb& P = B.p[p];
    const Dims d = P.d[0];
    const int loc = it - B.dfoff[p];
    const int tiles_x = (d.nx + BDf::TX - 1) / BDf::TX, nzc = (d.nz + DFZC - 1) / DFZC;
    const int tile = loc / nzc, zc = loc % nzc;
    const int cur = B.phicur[p];
    const float2 m1 = f64_to_df(B.sc[p * P_N + P_MEAN]);
    float r2 = 0.f, f2 = 0.f;
    PAcc ps{bcast(0.f), bcast(0.f)};
    // first: the residual of the initial iterate (no update, phi not written)
    dfk::df_segment<BDf>(d, cur ? P.phi2 : P.phi, first ? nullptr : final_e(P, 0), P.F,
                         DF2{bcast(m1.x), bcast(m1.y)}, first ? nullptr : (cur ? P.phi : P.phi2), P.r[0],
                         (tile % tiles_x) * BDf::TX, (tile / tiles_x) * BDf::TY, zc * DFZC,
                         min(zc * DFZC + DFZC, d.nz), smf, r2, ps, f2);
    const double s = block_sum_f(r2, sh);
    if (threadIdx.x == 0) B.dfpart[it] = s;
    if (first) {
      const double sf = block_sum_f(f2, sh);
      if (threadIdx.x == 0) B.dfpart2[it] = sf;
    }
  }
}

// V = 1..4: the Chebyshev degree, fused legs on levels of at least 16^3; V = 0: any
// degree (B.degree), one kernel per operation everywhere.
template <int V>
__global__ void __launch_bounds__(BT, 1) k_batched_solve(BDesc B) {
  cg::grid_group grid = cg::this_grid();
  extern __shared__ __align__(16) float smf[];
  __shared__ double sh[32];
  const int Vd = V > 0 ? V : B.degree;
  const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
  if (lead) *B.tstart = globaltimer();
  // ---- prologue: double-float copies and the mean of F
  phase0_sum(B, B.part0, sh, true, [&](const BProb& P, long long i, DfAcc& acc) {
    const float2 f = f64_to_df(P.src[i]);
    P.F[i] = f;
    P.phi[i] = f64_to_df(P.out[i]);
    acc.add(f.x);
    acc.c += f.y;
  });
  for (int pi = blockIdx.x * blockDim.x + threadIdx.x; pi < B.count; pi += gridDim.x * blockDim.x) B.phicur[pi] = 0;
  grid.sync();
  for (int pi = blockIdx.x * blockDim.x + threadIdx.x; pi < B.count; pi += gridDim.x * blockDim.x) {
    const BProb& P = B.p[pi];
    B.sc[pi * P_N + P_MEAN] = chunk_total(B, P, B.part0) / (double)ncell(P.d[0]);
  }
  grid.sync();
  // residual of the current iterate (per operation, problems selected by `sel`) and,
  // on the first call, ||F - mean||^2
  auto df_residual_phase = [&](bool with_f2, bool fused_too) {
    for (int c = blockIdx.x; c < B.nchunk[0]; c += gridDim.x) {
      const int pi = B.cprob[0][c];
      if (B.status[pi] != ST_ACTIVE) continue;
      const BProb& P = B.p[pi];
      if (!fused_too && V > 0 && P.dffused) continue;
      const Dims d = P.d[0];
      const float2 m = f64_to_df(B.sc[pi * P_N + P_MEAN]);
      const long long s0 = B.cstart[0][c];
      const long long n = ncell(d);
      const long long s1 = s0 + B.chunk[0] < n ? s0 + B.chunk[0] : n;
      float r2 = 0.f, f2 = 0.f;
      for (long long i = s0 + threadIdx.x; i < s1; i += blockDim.x) {
        int x, y, z;
        cell_xyz(d, i, x, y, z);
        const long long sy = d.nx, sz = (long long)d.nx * d.ny;
        const float2* u = P.phi;
        const float2 f = P.F[i];
        const float rv = df_resid(u[i], u[i + ((x == 0 ? d.nx - 1 : x - 1) - x)], u[i + ((x == d.nx - 1 ? 0 : x + 1) - x)],
                                  u[i + (long long)((y == 0 ? d.ny - 1 : y - 1) - y) * sy],
                                  u[i + (long long)((y == d.ny - 1 ? 0 : y + 1) - y) * sy],
                                  u[i + (long long)((z == 0 ? d.nz - 1 : z - 1) - z) * sz],
                                  u[i + (long long)((z == d.nz - 1 ? 0 : z + 1) - z) * sz], f, m);
        P.r[0][i] = rv;
        r2 += rv * rv;
        const float fv = __fadd_rn(__fsub_rn(f.x, m.x), __fsub_rn(f.y, m.y));
        f2 += fv * fv;
      }
      const double br = block_sum_f(r2, sh);
      if (threadIdx.x == 0) B.part0[c] = br;
      if (with_f2) {
        const double bf = block_sum_f(f2, sh);
        if (threadIdx.x == 0) B.part1[c] = bf;
      }
    }
  };
  // relative residual of every active problem, history and status
  auto finalize = [&](bool first) {
    for (int pi = blockIdx.x * blockDim.x + threadIdx.x; pi < B.count; pi += gridDim.x * blockDim.x) {
      if (B.status[pi] != ST_ACTIVE) continue;
      const BProb& P = B.p[pi];
      double* s = B.sc + pi * P_N;
      const bool fz = V > 0 && P.dffused;
      if (first) {
        if (fz) {
          double f2 = 0.0;
          for (int k = B.dfoff[pi]; k < B.dfoff[pi + 1]; ++k) f2 += B.dfpart2[k];
          s[P_F2] = f2;
        } else {
          s[P_F2] = chunk_total(B, P, B.part1);
        }
      }
      double r2;
      if (fz) {
        r2 = 0.0;
        for (int k = B.dfoff[pi]; k < B.dfoff[pi + 1]; ++k) r2 += B.dfpart[k];
        if (!first) B.phicur[pi] ^= 1;  // the fused update wrote the other buffer
      } else {
        r2 = chunk_total(B, P, B.part0);
      }
      const double rel = s[P_F2] > 0.0 ? sqrt(r2 / s[P_F2]) : sqrt(r2);
      int cyc = B.cycles[pi];
      if (first) {
        B.rel0[pi] = rel;
        s[P_PREV1] = s[P_PREV2] = -1.0;
      } else {
        if (cyc < 64) B.hist[pi * 64 + cyc] = rel;
        cyc += 1;
        B.cycles[pi] = cyc;
      }
      s[P_REL] = rel;
      int st = ST_ACTIVE;
      if (!isfinite(rel)) st = GBMG_ERR_NONFINITE;
      else if (rel <= B.tol) st = ST_CONVERGED;
      else if (!first && s[P_PREV2] > 0.0 && rel > 10.0 * s[P_PREV2]) st = GBMG_ERR_DIVERGED;
      else if (cyc >= B.maxv) st = GBMG_ERR_NOT_CONVERGED;
      s[P_PREV2] = s[P_PREV1];
      s[P_PREV1] = rel;
      if (st != ST_ACTIVE) {
        B.status[pi] = st;  // ST_CONVERGED is reported as GBMG_OK by the host
        B.tdone[pi] = globaltimer();
      }
    }
  };
  if constexpr (V > 0) fused_df(B, smf, sh, true);
  df_residual_phase(true, V == 0);
  grid.sync();
  finalize(true);
  grid.sync();
  // ---- V-cycles
  for (int cycle = 0; cycle < B.maxv; ++cycle) {
    if (lead) {
      int a = 0;
      for (int pi = 0; pi < B.count; ++pi) a += B.status[pi] == ST_ACTIVE;
      *B.any_active = a;
    }
    grid.sync();
    if (*((volatile int*)B.any_active) == 0) break;
    // down: levels 0 .. maxL-2, then the coarsest solves
    for (int l = 0; l + 1 < B.maxL; ++l) {
      // per-operation levels (smaller than 16^3, or every level for V = 0)
      auto smoothed = [&](const BProb& P, int lv) {
        return lv < P.L - 1 && !(V > 0 && lv_fused(P, lv)) && !(P.ls > 0 && lv >= P.ls);
      };
      if constexpr (V > 0) fused_down<V>(B, l, smf);
      const bool perop = V == 0 || (B.perop >> l & 1u);
      bool cur_a = true;  // current e in ea
      for (int k = 0; perop && k < Vd; ++k) {
        const bool from_zero = k == 0;
        const float c1 = B.c1[k];
        const float a = B.ca[l][k], b = B.cb[l][k];
        phase(B, l, smoothed, [&](const BProb& P, int lv, long long i) {
          const Dims d = P.d[lv];
          const float* e = cur_a ? P.ea[lv] : P.eb[lv];
          float* eo = cur_a ? P.eb[lv] : P.ea[lv];
          float c = 0.f, s = 0.f;
          if (!from_zero) {
            int x, y, z;
            cell_xyz(d, i, x, y, z);
            c = e[i];
            s = nsum_at(e, d, x, y, z, i);
          }
          float dd = from_zero ? 0.f : P.dv[lv][i];
          eo[i] = cheb_step(c, P.r[lv][i], s, c, dd, a, b, c1);
          P.dv[lv][i] = dd;
        });
        cur_a = !cur_a;
        grid.sync();
      }
      // residual, then full weighting to the next level
      const float ih2 = B.ih2[l];
      if (perop) {
      phase(B, l, smoothed, [&](const BProb& P, int lv, long long i) {
        const Dims d = P.d[lv];
        const float* e = cur_a ? P.ea[lv] : P.eb[lv];
        int x, y, z;
        cell_xyz(d, i, x, y, z);
        P.t[lv][i] = resid_from_sum(P.r[lv][i], nsum_at(e, d, x, y, z, i), e[i], ih2);
      });
      grid.sync();
      phase(B, l + 1, [&](const BProb& P, int lv) { return smoothed(P, lv - 1); },
            [&](const BProb& P, int lv, long long I) {
              const Dims df = P.d[lv - 1], dc = P.d[lv];
              int X, Y, Z;
              cell_xyz(dc, I, X, Y, Z);
              const float* f = P.t[lv - 1];
              int xs[3], ys[3], zs[3];
#pragma unroll
              for (int k = 0; k < 3; ++k) {
                xs[k] = wrapi(2 * X + k - 1, df.nx);
                ys[k] = wrapi(2 * Y + k - 1, df.ny);
                zs[k] = wrapi(2 * Z + k - 1, df.nz);
              }
              float yv[3];
#pragma unroll
              for (int a = 0; a < 3; ++a) {
                float zv[3];
#pragma unroll
                for (int b = 0; b < 3; ++b)
                  zv[b] = fw3(f[lin(df, xs[a], ys[b], zs[0])], f[lin(df, xs[a], ys[b], zs[1])],
                              f[lin(df, xs[a], ys[b], zs[2])]);
                yv[a] = fw3(zv[0], zv[1], zv[2]);
              }
              P.r[lv][I] = fw3(yv[0], yv[1], yv[2]);
            });
      }
      // (a level without fused or per-operation work, below every problem's bottom-cycle
      // start, has nothing to publish)
      if ((V > 0 && B.dtot[l] > 0) || perop) grid.sync();
      // coarsest solves of the problems whose hierarchy ends at level l + 1
      if (B.coarse >> (l + 1) & 1u) {
        const int warps = blockDim.x / 32, lane = threadIdx.x & 31;
        for (int pi = blockIdx.x; pi < B.count; pi += gridDim.x) {
          const BProb& P = B.p[pi];
          if (B.status[pi] != ST_ACTIVE || P.L - 1 != l + 1 || P.ls > 0) continue;
          const float* r = P.r[l + 1];
          float* e = P.ea[l + 1];
          for (int row = threadIdx.x / 32; row < P.nc; row += warps) {
            float acc = 0.f;
            for (int j = lane; j < P.nc; j += 32) acc = t_fma(P.G[(long long)row * P.nc + j], r[j], acc);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc = t_add(acc, __shfl_xor_sync(0xffffffffu, acc, o));
            if (lane == 0) e[row] = acc;
          }
        }
        grid.sync();
      }
    }
    // bottom cycles: the levels of each problem that fit in shared memory, one CTA per
    // problem (its correction at level ls lands in ea, where final_e reads it)
    if (V > 0 && B.anysmall) {
      for (int pi = blockIdx.x; pi < B.count; pi += gridDim.x) {
        const BProb& P = B.p[pi];
        if (B.status[pi] != ST_ACTIVE || P.ls == 0) continue;
        smallc::block_vcycle(B.small[pi], P.r[P.ls], P.ea[P.ls], smf);
        __syncthreads();
      }
      grid.sync();
    }
    // up: levels maxL-2 .. 0.  Per operation: pre-smoothing from zero leaves e in eb
    // when V is odd and in ea when V is even; V more steps then always end in ea,
    // which is where the coarser level's correction is read from and where the
    // coarsest solve writes.  Fused levels end in eb (final_e).
    for (int l = B.maxL - 2; l >= 0; --l) {
      auto smoothed = [&](const BProb& P, int lv) {
        return lv < P.L - 1 && !(V > 0 && lv_fused(P, lv)) && !(P.ls > 0 && lv >= P.ls);
      };
      if constexpr (V > 0) fused_up<V>(B, l, smf);
      const bool perop = V == 0 || (B.perop >> l & 1u);
      bool cur_a = (Vd % 2) == 0;
      if (perop)
        phase(B, l, smoothed, [&](const BProb& P, int lv, long long i) {
          const Dims d = P.d[lv];
          int x, y, z;
          cell_xyz(d, i, x, y, z);
          float* e = cur_a ? P.ea[lv] : P.eb[lv];
          e[i] = t_add(e[i], prolong_value(final_e(P, lv + 1), P.d[lv + 1], x, y, z));
        });
      if ((V > 0 && B.utot[l] > 0) || perop) grid.sync();
      for (int k = 0; perop && k < Vd; ++k) {
        const float c1 = B.c1[k];
        const float a = B.ca[l][k], b = B.cb[l][k];
        phase(B, l, smoothed, [&](const BProb& P, int lv, long long i) {
          const Dims d = P.d[lv];
          const float* e = cur_a ? P.ea[lv] : P.eb[lv];
          float* eo = cur_a ? P.eb[lv] : P.ea[lv];
          int x, y, z;
          cell_xyz(d, i, x, y, z);
          const float c = e[i];
          float dd = k == 0 ? 0.f : P.dv[lv][i];
          eo[i] = cheb_step(c, P.r[lv][i], nsum_at(e, d, x, y, z, i), c, dd, a, b, c1);
          P.dv[lv][i] = dd;
        });
        cur_a = !cur_a;
        grid.sync();
      }
    }
    // phi += e, next residual, convergence
    if constexpr (V > 0) fused_df(B, smf, sh, false);
    phase(B, 0, [&](const BProb& P, int) { return !(V > 0 && P.dffused); },
          [&](const BProb& P, int, long long i) { P.phi[i] = df_add_f(P.phi[i], final_e(P, 0)[i]); });
    grid.sync();
    df_residual_phase(false, false);
    grid.sync();
    finalize(false);
    grid.sync();
  }
  // problems still active after max_vcycles
  for (int pi = blockIdx.x * blockDim.x + threadIdx.x; pi < B.count; pi += gridDim.x * blockDim.x) {
    if (B.status[pi] == ST_ACTIVE) {
      B.status[pi] = GBMG_ERR_NOT_CONVERGED;
      B.tdone[pi] = globaltimer();
    }
  }
  grid.sync();
  // ---- epilogue: gauge and FP64 output for every problem
  phase0_sum(B, B.part0, sh, true, [&](const BProb& P, long long i, DfAcc& acc) {
    const float2 v = (B.phicur[&P - B.p] ? P.phi2 : P.phi)[i];
    acc.add(v.x);
    acc.c += v.y;
  });
  grid.sync();
  for (int pi = blockIdx.x * blockDim.x + threadIdx.x; pi < B.count; pi += gridDim.x * blockDim.x) {
    const BProb& P = B.p[pi];
    B.sc[pi * P_N + P_MPHI] = chunk_total(B, P, B.part0) / (double)ncell(P.d[0]);
  }
  grid.sync();
  for (int c = blockIdx.x; c < B.nchunk[0]; c += gridDim.x) {
    const int pi = B.cprob[0][c];
    const BProb& P = B.p[pi];
    const float2* ph = B.phicur[pi] ? P.phi2 : P.phi;
    float2 ms = f64_to_df(B.sc[pi * P_N + P_MPHI]);
    ms.x = -ms.x;
    ms.y = -ms.y;
    const long long s0 = B.cstart[0][c];
    const long long n = ncell(P.d[0]);
    const long long s1 = s0 + B.chunk[0] < n ? s0 + B.chunk[0] : n;
    for (long long i = s0 + threadIdx.x; i < s1; i += blockDim.x) P.out[i] = df_to_f64(df_add(ph[i], ms));
  }
}

}  // namespace

struct gbmg_batch {
  std::vector<gbmg_ctx*> ctx;
  int count = 0, maxL = 0, blocks = 0;
  cudaStream_t stream = nullptr;
  int device = 0;
  char* mem = nullptr;  // device memory of the descriptor tables and results
  BDesc desc{};
  int cap[BMAXL] = {};     // chunk-table capacity per level (tiles of MINCHUNK cells)
  BProb* hprob = nullptr;  // pinned host copy of the problem table
  int* hstatus = nullptr;  // pinned host results
  int* hcycles = nullptr;
  double* hhist = nullptr;
  double* hrel0 = nullptr;
  double* hsc = nullptr;
  unsigned long long* htime = nullptr;
  unsigned long long* htstart = nullptr;
  size_t res_bytes = 0;
  // CUDA graph of one solve (copy-in, resets, the cooperative launch, copy-out),
  // captured on a private stream and replayed while its key is unchanged
  bool use_graph = false;
  cudaStream_t gstream = nullptr;
  cudaEvent_t gev[2] = {nullptr, nullptr};
  cudaGraphExec_t gexec = nullptr;
  unsigned version = 0, g_version = ~0u;
  double g_tol = -1.0;
  int g_maxv = -1, g_blocks = -1;
  // kernel for the batch's degree and its dynamic shared memory; device memory of the
  // second phi buffers and the fused-phase tables
  const void* kern = nullptr;
  size_t smem = 0;
  char* mem2 = nullptr;
  ~gbmg_batch() {
    if (gexec) cudaGraphExecDestroy(gexec);
    if (mem2) cudaFree(mem2);
    if (gstream) cudaStreamDestroy(gstream);
    for (auto ev : gev)
      if (ev) cudaEventDestroy(ev);
    if (mem) cudaFree(mem);
    if (hprob) cudaFreeHost(hprob);
    if (hstatus) cudaFreeHost(hstatus);
  }
};

namespace {

long long ceil_div(long long a, long long b) { return (a + b - 1) / b; }

// Chunk tables of every level for the current tile sizes desc.chunk[], uploaded
// synchronously after the batch's stream has drained.
gbmg_status build_tables(gbmg_batch* b) {
  BDesc& D = b->desc;
  TRY(cudaStreamSynchronize(b->stream));
  for (int l = 0; l < b->maxL; ++l) {
    std::vector<int> cprob;
    std::vector<long long> cstart;
    for (int i = 0; i < b->count; ++i) {
      const gbmg_ctx* c = b->ctx[i];
      if (l >= c->L) continue;
      const long long n = ncell(c->lv[l].d);
      if (l == 0) b->hprob[i].c0 = (int)cprob.size();
      for (long long s = 0; s < n; s += D.chunk[l]) {
        cprob.push_back(i);
        cstart.push_back(s);
      }
      if (l == 0) b->hprob[i].nch = (int)cprob.size() - b->hprob[i].c0;
    }
    if ((long long)cprob.size() > b->cap[l]) return fail(GBMG_ERR_INVALID_ARG, "batch: tile table overflow");
    TRY(cudaMemcpy(D.cprob[l], cprob.data(), sizeof(int) * cprob.size(), cudaMemcpyHostToDevice));
    TRY(cudaMemcpy(D.cstart[l], cstart.data(), sizeof(long long) * cstart.size(), cudaMemcpyHostToDevice));
    D.nchunk[l] = (int)cprob.size();
  }
  b->version += 1;
  return GBMG_OK;
}

// dynamic shared memory of the fused phases at degree V
template <int V>
size_t batch_smem() {
  size_t s = 0;
  if constexpr (V > 0) {
    using TD = typename BDown<V>::T;
    using TU = typename BUp<V>::T;
    s = std::max(s, (size_t)(V + 1) * 2 * TD::PLANE * sizeof(float));
    s = std::max(s, ((size_t)V * 2 * TU::PLANE + 3 * legs::PCoarse<TU>::CN) * sizeof(float));
    s = std::max(s, (size_t)3 * BDf::PLANE * sizeof(float));
  }
  return s;
}

void pick_kernel(int degree, const void*& k, size_t& smem) {
  switch (degree) {
    case 1: k = (const void*)k_batched_solve<1>; smem = batch_smem<1>(); return;
    case 2: k = (const void*)k_batched_solve<2>; smem = batch_smem<2>(); return;
    case 3: k = (const void*)k_batched_solve<3>; smem = batch_smem<3>(); return;
    case 4: k = (const void*)k_batched_solve<4>; smem = batch_smem<4>(); return;
    default: k = (const void*)k_batched_solve<0>; smem = 0; return;
  }
}

gbmg_status max_blocks(const gbmg_batch* b, int& blocks) {
  int per_sm = 0, sms = 0;
  TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, b->kern, BT, b->smem));
  TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device));
  if (per_sm < 1) return fail(GBMG_ERR_CUDA, "batch: kernel does not fit on an SM");
  blocks = per_sm * sms;
  return GBMG_OK;
}

}  // namespace

extern "C" gbmg_status mg_batch_create(gbmg_batch** out, gbmg_ctx* const* ctxs, int count, void* cuda_stream) {
  g_last_error.clear();
  if (!out || !ctxs || count < 1) return fail(GBMG_ERR_INVALID_ARG, "mg_batch_create: bad argument");
  for (int i = 0; i < count; ++i) {
    const gbmg_ctx* c = ctxs[i];
    if (!c) return fail(GBMG_ERR_INVALID_ARG, "mg_batch_create: NULL context");
    if (c->o.op != GBMG_OP_FLAT7 || c->o.prec != GBMG_MIXED || c->o.smoother != GBMG_SMOOTH_CHEBYSHEV || c->o.fused)
      return fail(GBMG_ERR_INVALID_ARG,
                  "mg_batch_create: contexts must be flat, mixed precision, Chebyshev, fused = 0");
    if (c->L > BMAXL || c->L < 2) return fail(GBMG_ERR_INVALID_ARG, "mg_batch_create: each problem needs 2 to 16 levels");
    if (ncell(c->lv[0].d) >= (1ll << 31)) return fail(GBMG_ERR_INVALID_ARG, "mg_batch_create: a problem has 2^31 cells or more");
    if (c->o.degree > 8) return fail(GBMG_ERR_INVALID_ARG, "mg_batch_create: Chebyshev degree above 8");
    if (c->o.coarse_store) return fail(GBMG_ERR_INVALID_ARG, "mg_batch_create: coarse_store is for single solves");
    if (c->o.degree != ctxs[0]->o.degree || c->o.alpha != ctxs[0]->o.alpha)
      return fail(GBMG_ERR_INVALID_ARG, "mg_batch_create: all contexts need the same smoother");
    if (c->device != ctxs[0]->device) return fail(GBMG_ERR_INVALID_ARG, "mg_batch_create: contexts on different devices");
  }
  DeviceGuard g(ctxs[0]->device);
  auto* b = new (std::nothrow) gbmg_batch();
  if (!b) return fail(GBMG_ERR_OOM, "mg_batch_create: host allocation");
  b->ctx.assign(ctxs, ctxs + count);
  b->count = count;
  b->stream = (cudaStream_t)cuda_stream;
  b->device = ctxs[0]->device;
  int maxL = 0;
  for (auto* c : b->ctx) maxL = std::max(maxL, c->L);
  b->maxL = maxL;
  for (int l = 0; l < maxL; ++l) {
    long long cap = 0;
    for (auto* c : b->ctx)
      if (l < c->L) cap += ceil_div(ncell(c->lv[l].d), MINCHUNK);
    b->cap[l] = (int)cap;
  }
  // device layout
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += (bytes + 255) & ~(size_t)255;
    return o;
  };
  const size_t oP = take(sizeof(BProb) * count);
  std::vector<size_t> ocp(maxL), ocs(maxL);
  for (int l = 0; l < maxL; ++l) {
    ocp[l] = take(sizeof(int) * b->cap[l]);
    ocs[l] = take(sizeof(long long) * b->cap[l]);
  }
  const size_t n0 = (size_t)b->cap[0];
  const size_t oP0 = take(sizeof(double) * n0), oP1 = take(sizeof(double) * n0);
  const size_t oSc = take(sizeof(double) * P_N * count);
  // results block (copied back together): status, cycles, hist, rel0, times
  const size_t oRes = off;
  const size_t oSt = take(sizeof(int) * count), oCy = take(sizeof(int) * count);
  const size_t oHi = take(sizeof(double) * 64 * count), oR0 = take(sizeof(double) * count);
  const size_t oTd = take(sizeof(unsigned long long) * count), oTs = take(sizeof(unsigned long long));
  const size_t resEnd = off;
  const size_t oAny = take(sizeof(int));
  cudaError_t e = cudaMalloc((void**)&b->mem, off);
  if (e != cudaSuccess) {
    delete b;
    return cuda_fail(e, "mg_batch_create: device allocation");
  }
  b->res_bytes = resEnd - oRes;
  e = cudaMallocHost((void**)&b->hprob, sizeof(BProb) * count);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&b->hstatus, b->res_bytes + 8 * P_N * count);
  if (e != cudaSuccess) {
    delete b;
    return cuda_fail(e, "mg_batch_create: pinned allocation");
  }
  char* base = (char*)b->hstatus;
  b->hcycles = (int*)(base + (oCy - oRes));
  b->hhist = (double*)(base + (oHi - oRes));
  b->hrel0 = (double*)(base + (oR0 - oRes));
  b->htime = (unsigned long long*)(base + (oTd - oRes));
  b->htstart = (unsigned long long*)(base + (oTs - oRes));
  b->hsc = (double*)(base + b->res_bytes);
  char* m = b->mem;
  BDesc& D = b->desc;
  D.count = count;
  D.maxL = maxL;
  D.degree = ctxs[0]->o.degree;
  for (int k = 0; k < D.degree && k < 16; ++k) D.c1[k] = (float)ctxs[0]->cc1[k];
  for (int l = 0; l < maxL; ++l) {
    const double h = (double)(1 << l);
    D.ih2[l] = (float)(1.0 / (h * h));
    for (int k = 0; k < D.degree && k < 8; ++k) {
      double a, b;
      cheb_constants(ctxs[0]->cc2[k], h, a, b);
      D.ca[l][k] = (float)a;
      D.cb[l][k] = (float)b;
    }
  }
  D.p = (BProb*)(m + oP);
  for (int l = 0; l < maxL; ++l) {
    D.cprob[l] = (int*)(m + ocp[l]);
    D.cstart[l] = (long long*)(m + ocs[l]);
    D.chunk[l] = CHUNK;
  }
  D.part0 = (double*)(m + oP0);
  D.part1 = (double*)(m + oP1);
  D.sc = (double*)(m + oSc);
  D.status = (int*)(m + oSt);
  D.cycles = (int*)(m + oCy);
  D.hist = (double*)(m + oHi);
  D.rel0 = (double*)(m + oR0);
  D.tdone = (unsigned long long*)(m + oTd);
  D.tstart = (unsigned long long*)(m + oTs);
  D.any_active = (int*)(m + oAny);
  for (int i = 0; i < count; ++i) {
    const gbmg_ctx* c = b->ctx[i];
    BProb& P = b->hprob[i];
    std::memset(&P, 0, sizeof(P));
    P.L = c->L;
    P.nc = c->nc;
    for (int l = 0; l < c->L; ++l) {
      P.d[l] = c->lv[l].d;
      P.r[l] = (float*)c->lv[l].r;
      P.ea[l] = (float*)c->lv[l].e;
      P.eb[l] = (float*)c->lv[l].e2;
      P.dv[l] = (float*)c->lv[l].dv;
      P.t[l] = (float*)c->lv[l].t;
    }
    P.G = c->G32;
    P.F = c->F_df;
    P.phi = c->phi_df;
  }
  // fused phases: levels of at least 16^3 (not the coarsest) for degrees 1..4, the
  // finest level's double-float update for even nx; plane lists per level, items of
  // the double-float phase, second phi buffers, per-level Chebyshev constants
  const int V = (D.degree >= 1 && D.degree <= 4) ? D.degree : 0;
  pick_kernel(D.degree, b->kern, b->smem);
  std::vector<long long> doff((size_t)maxL * (count + 1), 0), uoff((size_t)maxL * (count + 1), 0);
  std::vector<int> dfoff(count + 1, 0);
  long long phi2_cells = 0;
  // bottom cycles: from the first level below the finest whose sub-hierarchy fits in
  // shared memory (fused degrees only); those levels leave the fused and per-operation
  // phases
  std::vector<SmallCycle> small(count);
  for (int i = 0; i < count; ++i) {
    const gbmg_ctx* c = b->ctx[i];
    BProb& P = b->hprob[i];
    for (int l = 1; V > 0 && l + 1 < c->L; ++l)
      if (small_cycle_params(c, l, &small[i])) {
        P.ls = l;
        D.anysmall = 1;
        b->smem = std::max(b->smem, small_cycle_smem(small[i]));
        break;
      }
    const int top = P.ls > 0 ? P.ls : c->L - 1;  // levels below top are fused or per operation
    for (int l = 0; V > 0 && l < top; ++l) {
      const Dims d = c->lv[l].d;
      if (d.nx >= 16 && d.ny >= 16 && d.nz >= 16) P.fmask |= 1u << l;
    }
    P.dffused = V > 0 && c->lv[0].d.nx % 2 == 0;
    if (P.dffused) phi2_cells += ncell(c->lv[0].d);
    for (int l = 0; l < top; ++l)
      if (!(P.fmask >> l & 1u)) D.perop |= 1u << l;
    if (P.ls == 0) D.coarse |= 1u << (c->L - 1);
  }
  for (int l = 0; l < maxL; ++l)
    for (int i = 0; i < count; ++i) {
      const gbmg_ctx* c = b->ctx[i];
      long long dn = 0, un = 0;
      if (b->hprob[i].fmask >> l & 1u) {
        const Dims d = c->lv[l].d;
        dn = (long long)ceil_div(d.nx, 64) * ceil_div(d.ny, down_ty(V)) * d.nz;
        un = (long long)ceil_div(d.nx, 64) * ceil_div(d.ny, up_ty(V)) * d.nz;
      }
      doff[(size_t)l * (count + 1) + i + 1] = doff[(size_t)l * (count + 1) + i] + dn;
      uoff[(size_t)l * (count + 1) + i + 1] = uoff[(size_t)l * (count + 1) + i] + un;
    }
  for (int i = 0; i < count; ++i) {
    const Dims d = b->ctx[i]->lv[0].d;
    const int items = b->hprob[i].dffused ? (int)(ceil_div(d.nx, BDf::TX) * ceil_div(d.ny, BDf::TY) * ceil_div(d.nz, DFZC)) : 0;
    dfoff[i + 1] = dfoff[i] + items;
  }
  std::vector<legs::Coef> coef(maxL);
  for (int l = 0; l < maxL; ++l) {
    std::memset(&coef[l], 0, sizeof(legs::Coef));
    for (int k = 0; k < D.degree && k < 16; ++k) {
      double a, bb;
      cheb_constants(ctxs[0]->cc2[k], (double)(1 << l), a, bb);
      coef[l].c1[k] = (float)ctxs[0]->cc1[k];
      coef[l].a[k] = (float)a;
      coef[l].b[k] = (float)bb;
    }
  }
  {
    size_t off2 = 0;
    auto take2 = [&](size_t bytes) {
      const size_t o = off2;
      off2 += (bytes + 255) & ~(size_t)255;
      return o;
    };
    const size_t oPhi2 = take2(sizeof(float2) * (size_t)std::max(phi2_cells, 1ll));
    const size_t oDoff = take2(sizeof(long long) * doff.size()), oUoff = take2(sizeof(long long) * uoff.size());
    const size_t oDf = take2(sizeof(int) * dfoff.size());
    const size_t oDfp = take2(sizeof(double) * (size_t)std::max(dfoff[count], 1));
    const size_t oDfp2 = take2(sizeof(double) * (size_t)std::max(dfoff[count], 1));
    const size_t oCur = take2(sizeof(int) * count), oCoef = take2(sizeof(legs::Coef) * maxL);
    const size_t oSmall = take2(sizeof(SmallCycle) * count);
    e = cudaMalloc((void**)&b->mem2, off2);
    if (e == cudaSuccess) e = cudaMemcpy(b->mem2 + oDoff, doff.data(), sizeof(long long) * doff.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->mem2 + oUoff, uoff.data(), sizeof(long long) * uoff.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->mem2 + oDf, dfoff.data(), sizeof(int) * dfoff.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->mem2 + oCoef, coef.data(), sizeof(legs::Coef) * maxL, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->mem2 + oSmall, small.data(), sizeof(SmallCycle) * count, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      delete b;
      return cuda_fail(e, "mg_batch_create: fused-phase tables");
    }
    long long acc = 0;
    for (int i = 0; i < count; ++i)
      if (b->hprob[i].dffused) {
        b->hprob[i].phi2 = reinterpret_cast<float2*>(b->mem2 + oPhi2) + acc;
        acc += ncell(b->ctx[i]->lv[0].d);
      }
    for (int l = 0; l < maxL; ++l) {
      D.doff[l] = reinterpret_cast<const long long*>(b->mem2 + oDoff) + (size_t)l * (count + 1);
      D.uoff[l] = reinterpret_cast<const long long*>(b->mem2 + oUoff) + (size_t)l * (count + 1);
      D.dtot[l] = doff[(size_t)l * (count + 1) + count];
      D.utot[l] = uoff[(size_t)l * (count + 1) + count];
    }
    D.dfoff = reinterpret_cast<const int*>(b->mem2 + oDf);
    D.dftot = dfoff[count];
    D.dfpart = reinterpret_cast<double*>(b->mem2 + oDfp);
    D.dfpart2 = reinterpret_cast<double*>(b->mem2 + oDfp2);
    D.phicur = reinterpret_cast<int*>(b->mem2 + oCur);
    D.coef = reinterpret_cast<const legs::Coef*>(b->mem2 + oCoef);
    D.small = reinterpret_cast<const SmallCycle*>(b->mem2 + oSmall);
  }
  if (b->smem > 0) {
    e = cudaFuncSetAttribute(b->kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem);
    if (e != cudaSuccess) {
      delete b;
      return cuda_fail(e, "mg_batch_create: shared-memory attribute");
    }
  }
  gbmg_status st = build_tables(b);
  // persistent grid: every block resident at once (cooperative launch)
  if (st == GBMG_OK) st = max_blocks(b, b->blocks);
  if (st != GBMG_OK) {
    delete b;
    return st;
  }
  *out = b;
  return GBMG_OK;
}

extern "C" void mg_batch_destroy(gbmg_batch* b) { delete b; }

extern "C" gbmg_status mg_batch_set_blocks(gbmg_batch* b, int blocks) {
  if (!b || blocks < 1) return fail(GBMG_ERR_INVALID_ARG, "mg_batch_set_blocks: bad argument");
  DeviceGuard g(b->device);
  int most = 0;
  TRYS(max_blocks(b, most));
  if (blocks > most) return fail(GBMG_ERR_INVALID_ARG, "mg_batch_set_blocks: more blocks than can be resident");
  b->blocks = blocks;
  return GBMG_OK;
}

extern "C" gbmg_status mg_batch_use_graph(gbmg_batch* b, int on) {
  if (!b) return fail(GBMG_ERR_INVALID_ARG, "mg_batch_use_graph: NULL batch");
  b->use_graph = on != 0;
  return GBMG_OK;
}

extern "C" gbmg_status mg_batch_set_tiles(gbmg_batch* b, const int* tile_cells, int nlevels) {
  if (!b || !tile_cells || nlevels < 1) return fail(GBMG_ERR_INVALID_ARG, "mg_batch_set_tiles: bad argument");
  for (int l = 0; l < nlevels && l < b->maxL; ++l)
    if (tile_cells[l] < MINCHUNK || tile_cells[l] > MAXCHUNK || tile_cells[l] % 256 != 0)
      return fail(GBMG_ERR_INVALID_ARG, "mg_batch_set_tiles: tile sizes must be multiples of 256 in [1024, 65536]");
  DeviceGuard g(b->device);
  for (int l = 0; l < nlevels && l < b->maxL; ++l) b->desc.chunk[l] = tile_cells[l];
  return build_tables(b);
}

extern "C" gbmg_status mg_batch_get_tiles(const gbmg_batch* b, int* tile_cells, int nlevels) {
  if (!b || !tile_cells) return fail(GBMG_ERR_INVALID_ARG, "mg_batch_get_tiles: bad argument");
  for (int l = 0; l < nlevels; ++l) tile_cells[l] = l < b->maxL ? b->desc.chunk[l] : 0;
  return GBMG_OK;
}

extern "C" int mg_batch_num_levels(const gbmg_batch* b) { return b ? b->maxL : 0; }

extern "C" gbmg_status mg_batch_solve(gbmg_batch* b, const double* const* src_dev, double* const* phi_dev, double tol,
                                      int max_vcycles, gbmg_stats* stats, double* times_ms) {
  g_last_error.clear();
  if (!b || !src_dev || !phi_dev) return fail(GBMG_ERR_INVALID_ARG, "mg_batch_solve: NULL argument");
  if (!(tol >= 0.0)) return fail(GBMG_ERR_INVALID_ARG, "mg_batch_solve: tol must be >= 0");
  DeviceGuard g(b->device);
  for (int i = 0; i < b->count; ++i) {
    if (!src_dev[i] || !phi_dev[i]) return fail(GBMG_ERR_INVALID_ARG, "mg_batch_solve: NULL field");
    b->hprob[i].src = src_dev[i];
    b->hprob[i].out = phi_dev[i];
  }
  BDesc D = b->desc;
  D.tol = tol;
  D.maxv = max_vcycles < 0 ? 0 : max_vcycles;
  // the whole solve as one stream-ordered sequence
  auto enqueue = [&](cudaStream_t st) -> gbmg_status {
    TRY(cudaMemcpyAsync(D.p, b->hprob, sizeof(BProb) * b->count, cudaMemcpyHostToDevice, st));
    TRY(cudaMemsetAsync(D.status, 0, sizeof(int) * b->count, st));
    TRY(cudaMemsetAsync(D.cycles, 0, sizeof(int) * b->count, st));
    void* args[] = {&D};
    TRY(cudaLaunchCooperativeKernel(b->kern, dim3(b->blocks), dim3(BT), args, b->smem, st));
    TRY(cudaMemcpyAsync(b->hstatus, D.status, b->res_bytes, cudaMemcpyDeviceToHost, st));
    TRY(cudaMemcpyAsync(b->hsc, D.sc, sizeof(double) * P_N * b->count, cudaMemcpyDeviceToHost, st));
    return GBMG_OK;
  };
  if (!b->use_graph) {
    TRYS(enqueue(b->stream));
  } else {
    if (!b->gstream) {
      TRY(cudaStreamCreateWithFlags(&b->gstream, cudaStreamNonBlocking));
      TRY(cudaEventCreateWithFlags(&b->gev[0], cudaEventDisableTiming));
      TRY(cudaEventCreateWithFlags(&b->gev[1], cudaEventDisableTiming));
    }
    if (!b->gexec || b->g_version != b->version || b->g_tol != tol || b->g_maxv != D.maxv ||
        b->g_blocks != b->blocks) {
      if (b->gexec) {
        cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
      }
      cudaGraph_t graph = nullptr;
      TRY(cudaStreamBeginCapture(b->gstream, cudaStreamCaptureModeThreadLocal));
      const gbmg_status cs = enqueue(b->gstream);
      const cudaError_t ce = cudaStreamEndCapture(b->gstream, &graph);
      if (cs != GBMG_OK) {
        if (graph) cudaGraphDestroy(graph);
        return cs;
      }
      TRY(ce);
      const cudaError_t ie = cudaGraphInstantiate(&b->gexec, graph, 0);
      cudaGraphDestroy(graph);
      TRY(ie);
      b->g_version = b->version;
      b->g_tol = tol;
      b->g_maxv = D.maxv;
      b->g_blocks = b->blocks;
    }
    // order the graph after earlier work on the caller's stream and before later work
    TRY(cudaEventRecord(b->gev[0], b->stream));
    TRY(cudaStreamWaitEvent(b->gstream, b->gev[0], 0));
    TRY(cudaGraphLaunch(b->gexec, b->gstream));
    TRY(cudaEventRecord(b->gev[1], b->gstream));
    TRY(cudaStreamWaitEvent(b->stream, b->gev[1], 0));
  }
  note_launch();
  TRY(cudaStreamSynchronize(b->stream));
  gbmg_status worst = GBMG_OK;
  const unsigned long long t0 = *b->htstart;
  for (int i = 0; i < b->count; ++i) {
    const int s = b->hstatus[i];
    const gbmg_status st = s == ST_CONVERGED ? GBMG_OK : (gbmg_status)s;
    if (st != GBMG_OK && worst == GBMG_OK) worst = st;
    if (stats) {
      gbmg_stats& S = stats[i];
      std::memset(&S, 0, sizeof(S));
      S.cycles = b->hcycles[i];
      S.status = st;
      S.rel_res0 = b->hrel0[i];
      S.rel_res = b->hsc[i * P_N + P_REL];
      for (int k = 0; k < S.cycles && k < 64; ++k) S.res_hist[k] = b->hhist[i * 64 + k];
    }
    if (times_ms) times_ms[i] = (double)(b->htime[i] - t0) * 1e-6;
  }
  return worst;
}

namespace {

// One timed trial from the saved initial guesses.
gbmg_status trial(gbmg_batch* b, const double* const* src, double* const* phi, double* const* save, double tol,
                  int maxv, cudaEvent_t e0, cudaEvent_t e1, float& ms) {
  for (int i = 0; i < b->count; ++i)
    TRY(cudaMemcpyAsync(phi[i], save[i], sizeof(double) * ncell(b->ctx[i]->lv[0].d), cudaMemcpyDeviceToDevice,
                        b->stream));
  TRY(cudaEventRecord(e0, b->stream));
  const gbmg_status s = mg_batch_solve(b, src, phi, tol, maxv, nullptr, nullptr);
  if (s == GBMG_ERR_CUDA || s == GBMG_ERR_INVALID_ARG || s == GBMG_ERR_OOM) return s;
  TRY(cudaEventRecord(e1, b->stream));
  TRY(cudaEventSynchronize(e1));
  TRY(cudaEventElapsedTime(&ms, e0, e1));
  return GBMG_OK;
}

}  // namespace

extern "C" gbmg_status mg_batch_autotune(gbmg_batch* b, const double* const* src_dev, double* const* phi_dev,
                                         double tol, int max_vcycles, int* blocks_out, int* tiles_out) {
  if (!b || !src_dev || !phi_dev) return fail(GBMG_ERR_INVALID_ARG, "mg_batch_autotune: NULL argument");
  DeviceGuard g(b->device);
  int most = 0, sms = 0;
  TRYS(max_blocks(b, most));
  TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device));
  // every trial starts from the caller's initial guesses
  std::vector<double*> save(b->count, nullptr);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  gbmg_status st = GBMG_OK;
  auto run = [&]() -> gbmg_status {
    for (int i = 0; i < b->count; ++i) {
      const size_t bytes = sizeof(double) * ncell(b->ctx[i]->lv[0].d);
      TRY(cudaMalloc((void**)&save[i], bytes));
      TRY(cudaMemcpyAsync(save[i], phi_dev[i], bytes, cudaMemcpyDeviceToDevice, b->stream));
    }
    TRY(cudaEventCreate(&e0));
    TRY(cudaEventCreate(&e1));
    float ms = 0.f, best_ms = -1.f;
    // grid size: 1 .. (resident blocks per SM) times the SM count
    int best = b->blocks;
    for (int blocks = sms; blocks <= most; blocks += sms) {
      b->blocks = blocks;
      TRYS(trial(b, src_dev, phi_dev, save.data(), tol, max_vcycles, e0, e1, ms));
      if (best_ms < 0.f || ms < best_ms) best_ms = ms, best = blocks;
    }
    b->blocks = best;
    // tile size per level, one level at a time (coordinate descent from the current sizes)
    for (int l = 0; l < b->maxL; ++l) {
      long long biggest = 0;
      for (auto* c : b->ctx)
        if (l < c->L) biggest = std::max(biggest, ncell(c->lv[l].d));
      int keep = b->desc.chunk[l];
      for (int cand = MINCHUNK; cand <= MAXCHUNK; cand *= 2) {
        if (cand == keep || (cand > biggest && cand / 2 >= biggest)) continue;
        b->desc.chunk[l] = cand;
        TRYS(build_tables(b));
        TRYS(trial(b, src_dev, phi_dev, save.data(), tol, max_vcycles, e0, e1, ms));
        if (ms < best_ms) best_ms = ms, keep = cand;
      }
      b->desc.chunk[l] = keep;
      TRYS(build_tables(b));
    }
    // leave the caller's phi holding the solution from the initial guesses
    TRYS(trial(b, src_dev, phi_dev, save.data(), tol, max_vcycles, e0, e1, ms));
    return GBMG_OK;
  };
  st = run();
  cudaStreamSynchronize(b->stream);
  for (double* p : save)
    if (p) cudaFree(p);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st != GBMG_OK) return st;
  if (blocks_out) *blocks_out = b->blocks;
  if (tiles_out)
    for (int l = 0; l < b->maxL; ++l) tiles_out[l] = b->desc.chunk[l];
  return GBMG_OK;
}
