// Temporally blocked FP32 level kernels (the single-GPU form of the paper's
// communication-avoiding whole-level fusion, Sec. 3.4 implementation list): one
// HBM pass per level visit instead of one per operation.
//
//   k_down_fused : Chebyshev pre-smoothing from e = 0 (degree V), residual and
//                  full-weighting restriction.  Reads r, writes e and R(r - A e).
//   k_up_fused   : trilinear prolongation + correction and Chebyshev
//                  post-smoothing.  Reads e, e_c, r; writes the new e.
//   k_df_update_residual : finest level, phi' = phi + e in double-float and the
//                  next defect-correction residual r' = F - m - A phi'.
//
// Blocking scheme.  A CTA owns an output tile of TX x TY cells in (x, y) and a
// chunk of z planes; it computes on the tile plus a halo of H cells, so that the
// stages, each of which needs its input on one more ring of cells, still produce
// valid values on the tile.  The CTA streams through z: in each iteration it
// loads one input plane and every stage advances one plane, stage s working one
// plane behind stage s-1.  The current plane of each stage's input sits in a
// padded, double-buffered shared-memory plane (x/y neighbours); the two older
// planes of the z direction stay in registers.  One barrier per iteration.
// Cells outside the valid region of a stage hold garbage that never reaches an
// output.  Arithmetic is the same per-cell code as the one-kernel-per-operation
// path, so results are bit-identical to it.
#include <cstdio>

#include "kernels.h"
#include "stencil.cuh"

namespace gbmg {

namespace {

__device__ __forceinline__ int wrapmod(int i, int n) {
  const int r = i % n;
  return r < 0 ? r + n : r;
}

template <int TX, int TY, int H, int NT>
struct Tile {
  static constexpr int WX = TX + 2 * H;
  static constexpr int WY = TY + 2 * H;
  static constexpr int NPOS = WX * WY;
  static constexpr int K = (NPOS + NT - 1) / NT;  // positions per thread
  static constexpr int PAD = WX + 1;              // padding so p +- 1, p +- WX stay in bounds
  // every thread slot (valid or not) owns a plane entry, so no slot needs a guard
  static constexpr int PLANE = K * NT + 2 * PAD;
};

// Per-thread position bookkeeping: plane offset of each owned position in the
// (wrapped) global mesh, and bit masks of valid / in-tile positions.
template <int TX, int TY, int H, int NT>
struct Positions {
  using TL = Tile<TX, TY, H, NT>;
  int goff[TL::K];
  unsigned vmask = 0, tmask = 0;
  __device__ __forceinline__ void init(Dims d, int x0, int y0) {
#pragma unroll
    for (int k = 0; k < TL::K; ++k) {
      const int p = threadIdx.x + k * NT;
      goff[k] = 0;
      if (p < TL::NPOS) {
        const int px = p % TL::WX, py = p / TL::WX;
        const int ux = x0 - H + px, uy = y0 - H + py;
        goff[k] = wrapmod(ux, d.nx) + wrapmod(uy, d.ny) * d.nx;
        vmask |= 1u << k;
        if (px >= H && px < H + TX && py >= H && py < H + TY && ux < d.nx && uy < d.ny) tmask |= 1u << k;
      }
    }
  }
};

// Folded Chebyshev constants of one level: c1 and a = c2 D^-1, b = a / h^2 per step.
struct Coef {
  float c1[16];
  float a[16];
  float b[16];
};

// ------------------------------------------------------------------ down leg

template <int V, int TX, int TY, int NT>
__device__ __forceinline__ void down_segment(Dims d, const float* __restrict__ r, float* __restrict__ e_out,
                                             float* __restrict__ rc, int x0, int y0, int z0, int zend,
                                             float inv_h2, const Coef& cf, float* sm) {
  constexpr int H = V + 1;
  using TL = Tile<TX, TY, H, NT>;
  constexpr int WX = TL::WX, K = TL::K, PLANE = TL::PLANE, PAD = TL::PAD;
  constexpr int NCO = (TX / 2) * (TY / 2);  // coarse outputs per tile plane
  // plane(s, b): s = 0..V-1 holds e_{s+1}, s = V holds the z-weighted residual
  auto plane = [&](int s, int b) -> float* { return sm + (s * 2 + b) * PLANE + PAD; };

  const int tid = threadIdx.x;
  const long long pst = (long long)d.nx * d.ny;
  Positions<TX, TY, H, NT> P;
  P.init(d, x0, y0);
  const Dims dc{d.nx / 2, d.ny / 2, d.nz / 2};

  float rq[V + 1][K];              // rq[j][k] = r at plane t - j
  float wp[V + 2][K], wc[V + 2][K];  // stage s input window: planes p-1, p
  float dh[V + 1][K];              // d_{s-1} at stage s's plane
  float rsp[K], rsc[K];            // residual window
  float rnext[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
#pragma unroll
    for (int j = 0; j <= V; ++j) rq[j][k] = 0.f, dh[j][k] = 0.f;
#pragma unroll
    for (int s = 0; s < V + 2; ++s) wp[s][k] = 0.f, wc[s][k] = 0.f;
    rsp[k] = rsc[k] = 0.f;
  }
  // last iteration: the coarse plane c = zend - 1 (a segment may end on an odd plane)
  // is written at t = c + V + 2
  const int tb = z0 - H, te = zend + V + 1;
  {
    const long long base = (long long)wrapmod(tb, d.nz) * pst;
#pragma unroll
    for (int k = 0; k < K; ++k) rnext[k] = __ldg(r + base + P.goff[k]);
  }
  for (int t = tb; t <= te; ++t) {
    const int cur = (t - tb) & 1, prv = cur ^ 1;
#pragma unroll
    for (int k = 0; k < K; ++k) {
#pragma unroll
      for (int j = V; j > 0; --j) rq[j][k] = rq[j - 1][k];
      rq[0][k] = rnext[k];
    }
    if (t < te) {
      const long long base = (long long)wrapmod(t + 1, d.nz) * pst;
#pragma unroll
      for (int k = 0; k < K; ++k) rnext[k] = __ldg(r + base + P.goff[k]);
    }
    float en[V + 1][K], dn[V + 1][K];
    // stage 1 (pointwise, e starts at zero): e_1 = d_1 = c2_0 D^-1 r
#pragma unroll
    for (int k = 0; k < K; ++k) {
      float dd = 0.f;
      en[1][k] = cheb_step(0.f, rq[0][k], 0.f, 0.f, dd, cf.a[0], cf.b[0], cf.c1[0]);
      dn[1][k] = dd;
      plane(0, cur)[tid + k * NT] = en[1][k];
    }
    // stages 2..V: Chebyshev steps with the stencil on e_{s-1}
#pragma unroll
    for (int s = 2; s <= V; ++s) {
      const float* src = plane(s - 2, prv);
      float* dst = plane(s - 1, cur);
      const int zp = t - s + 1;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const int p = tid + k * NT;
        const float c = wc[s][k];
        const float sn = nbr_sum(src[p - 1], src[p + 1], src[p - WX], src[p + WX], wp[s][k], en[s - 1][k]);
        float dd = dh[s][k];
        en[s][k] = cheb_step(c, rq[s - 1][k], sn, c, dd, cf.a[s - 1], cf.b[s - 1], cf.c1[s - 1]);
        dn[s][k] = dd;
        dst[p] = en[s][k];
        if (s == V && (P.tmask >> k & 1u) && zp >= z0 && zp < zend) e_out[(long long)zp * pst + P.goff[k]] = en[s][k];
      }
    }
    if (V == 1) {
      const int zp = t;
#pragma unroll
      for (int k = 0; k < K; ++k)
        if ((P.tmask >> k & 1u) && zp >= z0 && zp < zend) e_out[(long long)zp * pst + P.goff[k]] = en[1][k];
    }
    // residual stage at plane t - V, then z weights of the restriction at c = t - V - 1
    {
      const float* src = plane(V - 1, prv);
      float* zsd = plane(V, cur);
      const int c = t - V - 1;
      const bool cz = ((c & 1) == 0) && c >= z0 && c < zend;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const int p = tid + k * NT;
        const float rn = resid_from_sum(rq[V][k],
                                        nbr_sum(src[p - 1], src[p + 1], src[p - WX], src[p + WX], wp[V + 1][k], en[V][k]),
                                        wc[V + 1][k], inv_h2);
        if (cz) zsd[p] = fw3(rsp[k], rsc[k], rn);
        rsp[k] = rsc[k];
        rsc[k] = rn;
      }
    }
    // coarse output from the z-weighted plane of the previous iteration
    {
      const int c = t - V - 2;
      if (((c & 1) == 0) && c >= z0 && c < zend) {
        const float* zs = plane(V, prv);
        for (int q = tid; q < NCO; q += NT) {
          const int ccx = q % (TX / 2), ccy = q / (TX / 2);
          const int cX = x0 / 2 + ccx, cY = y0 / 2 + ccy;
          if (cX < dc.nx && cY < dc.ny) {
            const int cp = (H + 2 * ccy) * WX + H + 2 * ccx;
            float yv[3];
#pragma unroll
            for (int a = -1; a <= 1; ++a) yv[a + 1] = fw3(zs[cp + a - WX], zs[cp + a], zs[cp + a + WX]);
            rc[((long long)(c >> 1) * dc.ny + cY) * dc.nx + cX] = fw3(yv[0], yv[1], yv[2]);
          }
        }
      }
    }
    // advance the z windows
#pragma unroll
    for (int k = 0; k < K; ++k) {
#pragma unroll
      for (int s = 2; s <= V + 1; ++s) {
        wp[s][k] = wc[s][k];
        wc[s][k] = en[s - 1][k];
      }
#pragma unroll
      for (int s = 2; s <= V; ++s) dh[s][k] = dn[s - 1][k];
    }
    __syncthreads();
  }
}

// Persistent schedule: the tiles' planes form one list (tile-major); CTA b takes the
// contiguous range [b T / G, (b+1) T / G) and runs it as one segment per tile touched.
struct Sched {
  int tiles_x;
  long long total;  // tiles * nz
};

template <int V, int TX, int TY, int NT>
__global__ void __maxnreg__(65536 / ((NT + 127) / 128 * 128) / 8 * 8)
k_down_fused(Dims d, const float* __restrict__ r, float* __restrict__ e_out, float* __restrict__ rc, Sched sc,
             float inv_h2, Coef cf) {
  extern __shared__ float sm[];
  long long a = (long long)blockIdx.x * sc.total / gridDim.x;
  const long long b = (long long)(blockIdx.x + 1) * sc.total / gridDim.x;
  while (a < b) {
    const long long tile = a / d.nz;
    const int z0 = (int)(a % d.nz);
    const int zend = (int)(z0 + (b - a) < d.nz ? z0 + (b - a) : d.nz);
    down_segment<V, TX, TY, NT>(d, r, e_out, rc, (int)(tile % sc.tiles_x) * TX, (int)(tile / sc.tiles_x) * TY, z0,
                                zend, inv_h2, cf, sm);
    a += zend - z0;
    __syncthreads();
  }
}

// ------------------------------------------------------------------ up leg

__device__ __forceinline__ int floor_half(int v) { return v >= 0 ? v / 2 : -((1 - v) / 2); }
__device__ __forceinline__ int mod3(int v) {
  const int r = v % 3;
  return r < 0 ? r + 3 : r;
}

// Coarse tile of the up leg: the coarse nodes under a fine region of WX x WY cells
// starting at fine (x0 - H, y0 - H), one node of margin for the +1 neighbour.
template <int TX, int TY, int H>
struct CoarseTile {
  static constexpr int WX = TX + 2 * H, WY = TY + 2 * H;
  static constexpr int CW = (WX + 3) / 2 + 1;
  static constexpr int CH = (WY + 3) / 2 + 1;
  static constexpr int CN = CW * CH;
};

template <int V, int TX, int TY, int NT>
__device__ __forceinline__ void up_segment(Dims d, const float* __restrict__ e_in, const float* __restrict__ ec,
                                           const float* __restrict__ r, float* __restrict__ e_out, int x0, int y0,
                                           int z0, int zend, float inv_h2, const Coef& cf, float* sm) {
  constexpr int H = V;
  using TL = Tile<TX, TY, H, NT>;
  using CT = CoarseTile<TX, TY, H>;
  constexpr int WX = TL::WX, K = TL::K, PLANE = TL::PLANE, PAD = TL::PAD;
  constexpr int CW = CT::CW, CN = CT::CN, CL = (CN + NT - 1) / NT;
  // plane(s, b): e_s for s = 0..V-1 (e_0 = e + P e_c); then three coarse planes
  auto plane = [&](int s, int b) -> float* { return sm + (s * 2 + b) * PLANE + PAD; };
  float* cring = sm + V * 2 * PLANE;

  const int tid = threadIdx.x;
  const long long pst = (long long)d.nx * d.ny;
  const Dims dc{d.nx / 2, d.ny / 2, d.nz / 2};
  const long long cpst = (long long)dc.nx * dc.ny;
  Positions<TX, TY, H, NT> P;
  P.init(d, x0, y0);
  // coarse node under each position (local offset in the coarse tile) and the odd flags
  const int CX0 = floor_half(x0 - H), CY0 = floor_half(y0 - H);
  int co[K];
  unsigned oddx = 0, oddy = 0;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int p = tid + k * NT;
    co[k] = 0;
    if (p < TL::NPOS) {
      const int ux = x0 - H + p % WX, uy = y0 - H + p / WX;
      const int I = floor_half(ux), J = floor_half(uy);
      co[k] = (J - CY0) * CW + (I - CX0);
      oddx |= (unsigned)(ux - 2 * I) << k;
      oddy |= (unsigned)(uy - 2 * J) << k;
    }
  }
  // coarse tile cells this thread loads
  int cgo[CL];
#pragma unroll
  for (int j = 0; j < CL; ++j) {
    const int q = tid + j * NT;
    cgo[j] = -1;
    if (q < CN) cgo[j] = wrapmod(CX0 + q % CW, dc.nx) + wrapmod(CY0 + q / CW, dc.ny) * dc.nx;
  }
  auto load_coarse = [&](int Ku, float (&vals)[CL]) {
    const long long base = (long long)wrapmod(Ku, dc.nz) * cpst;
#pragma unroll
    for (int j = 0; j < CL; ++j) vals[j] = cgo[j] >= 0 ? __ldg(ec + base + cgo[j]) : 0.f;
  };
  auto store_coarse = [&](int Ku, const float (&vals)[CL]) {
    float* dst = cring + mod3(Ku) * CN;
#pragma unroll
    for (int j = 0; j < CL; ++j)
      if (cgo[j] >= 0) dst[tid + j * NT] = vals[j];
  };

  float rq[V + 1][K];
  float wp[V + 1][K], wc[V + 1][K];
  float dh[V + 1][K];
  float rnext[K], enext[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
#pragma unroll
    for (int j = 0; j <= V; ++j) rq[j][k] = 0.f, dh[j][k] = 0.f, wp[j][k] = 0.f, wc[j][k] = 0.f;
  }
  const int tb = z0 - V, te = zend + V - 1;
  auto load = [&](int t) {
    const long long base = (long long)wrapmod(t, d.nz) * pst;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      rnext[k] = __ldg(r + base + P.goff[k]);
      enext[k] = __ldg(e_in + base + P.goff[k]);
    }
  };
  {
    float cv[CL];
    const int K0 = floor_half(tb);
    load_coarse(K0, cv);
    store_coarse(K0, cv);
    load_coarse(K0 + 1, cv);
    store_coarse(K0 + 1, cv);
  }
  load(tb);
  __syncthreads();
  for (int t = tb; t <= te; ++t) {
    const int cur = (t - tb) & 1, prv = cur ^ 1;
    float en[V + 1][K], dn[V + 1][K];
    const int Ku = floor_half(t);
    const bool zodd = (t - 2 * Ku) != 0;
    // next coarse plane (needed from the next even t on), stored at the end of this iteration
    float cv[CL];
    const bool need_c = zodd && t < te;
    if (need_c) load_coarse(Ku + 2, cv);
#pragma unroll
    for (int k = 0; k < K; ++k) {
#pragma unroll
      for (int j = V; j > 0; --j) rq[j][k] = rq[j - 1][k];
      rq[0][k] = rnext[k];
      en[0][k] = enext[k];
    }
    if (t < te) load(t + 1);
    // stage 0: e_0 = e + P e_c (pointwise), P from the coarse planes Ku and Ku + 1
    {
      const float* c0 = cring + mod3(Ku) * CN;
      const float* c1 = cring + mod3(Ku + 1) * CN;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        {
          const bool dx = oddx >> k & 1u, dy = oddy >> k & 1u;
          auto cxv = [&](const float* cp, int off) -> float {
            const float v0 = cp[off];
            return dx ? half_sum(v0, cp[off + 1]) : v0;
          };
          auto cyv = [&](const float* cp) -> float {
            const float v0 = cxv(cp, co[k]);
            return dy ? half_sum(v0, cxv(cp, co[k] + CW)) : v0;
          };
          const float v0 = cyv(c0);
          const float pv = zodd ? half_sum(v0, cyv(c1)) : v0;
          en[0][k] = t_add(en[0][k], pv);
          plane(0, cur)[tid + k * NT] = en[0][k];
        }
      }
    }
    // stages 1..V: Chebyshev post-smoothing steps at plane t - s
#pragma unroll
    for (int s = 1; s <= V; ++s) {
      const float* src = plane(s - 1, prv);
      const int zp = t - s;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const int p = tid + k * NT;
        const float c = wc[s][k];
        const float sn = nbr_sum(src[p - 1], src[p + 1], src[p - WX], src[p + WX], wp[s][k], en[s - 1][k]);
        float dd = s == 1 ? 0.f : dh[s][k];
        en[s][k] = cheb_step(c, rq[s][k], sn, c, dd, cf.a[s - 1], cf.b[s - 1], cf.c1[s - 1]);
        dn[s][k] = dd;
        if (s < V) {
          plane(s, cur)[p] = en[s][k];
        } else if ((P.tmask >> k & 1u) && zp >= z0 && zp < zend) {
          e_out[(long long)zp * pst + P.goff[k]] = en[s][k];
        }
      }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
#pragma unroll
      for (int s = 1; s <= V; ++s) {
        wp[s][k] = wc[s][k];
        wc[s][k] = en[s - 1][k];
      }
#pragma unroll
      for (int s = 2; s <= V; ++s) dh[s][k] = dn[s - 1][k];
    }
    if (need_c) store_coarse(Ku + 2, cv);
    __syncthreads();
  }
}

template <int V, int TX, int TY, int NT>
__global__ void __maxnreg__(65536 / ((NT + 127) / 128 * 128) / 8 * 8)
k_up_fused(Dims d, const float* __restrict__ e_in, const float* __restrict__ ec, const float* __restrict__ r,
           float* __restrict__ e_out, Sched sc, float inv_h2, Coef cf) {
  extern __shared__ float sm[];
  long long a = (long long)blockIdx.x * sc.total / gridDim.x;
  const long long b = (long long)(blockIdx.x + 1) * sc.total / gridDim.x;
  while (a < b) {
    const long long tile = a / d.nz;
    const int z0 = (int)(a % d.nz);
    const int zend = (int)(z0 + (b - a) < d.nz ? z0 + (b - a) : d.nz);
    up_segment<V, TX, TY, NT>(d, e_in, ec, r, e_out, (int)(tile % sc.tiles_x) * TX, (int)(tile / sc.tiles_x) * TY, z0,
                              zend, inv_h2, cf, sm);
    a += zend - z0;
    __syncthreads();
  }
}

// ------------------------------------------------------------------ finest level, double-float

// phi' = phi + e (double-float) on the tile plus a one-cell halo, then
// r' = F - m - A phi' on the tile; block partial sums of r'^2 and of phi'.
// Loads of the next plane are issued before the current plane is processed.
template <int TX, int TY, int NT>
__global__ void __launch_bounds__(NT)
k_df_update_residual(Dims d, const float2* __restrict__ phi_in, const float* __restrict__ e,
                     const float2* __restrict__ F, const double* __restrict__ m_dev, float2* __restrict__ phi_out,
                     float* __restrict__ r_out, double* __restrict__ pr2, double* __restrict__ psum,
                     double* __restrict__ pf2, int zc) {
  constexpr int H = 1;
  using TL = Tile<TX, TY, H, NT>;
  constexpr int WX = TL::WX, K = TL::K, PLANE = TL::PLANE, PAD = TL::PAD;
  __shared__ float2 sp[2][PLANE];
  __shared__ double shr[32];
  const int tid = threadIdx.x;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * zc;
  const int zend = min(z0 + zc, d.nz);
  const long long pst = (long long)d.nx * d.ny;
  Positions<TX, TY, H, NT> P;
  P.init(d, x0, y0);
  const float2 m = f64_to_df(m_dev[0]);
  float2 wp[K], wc[K];
  float2 nphi[K], fq[K];
  float ne[K];
  float r2 = 0.f, f2 = 0.f;
  DfAcc ps{0.f, 0.f};
#pragma unroll
  for (int k = 0; k < K; ++k) wp[k] = wc[k] = fq[k] = make_float2(0.f, 0.f);
#pragma unroll
  for (int k = 0; k < K; ++k) ne[k] = 0.f;
  const int tb = z0 - 1, te = zend;
  auto load = [&](int t) {
    const long long base = (long long)wrapmod(t, d.nz) * pst;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const bool v = P.vmask >> k & 1u;
      nphi[k] = v ? phi_in[base + P.goff[k]] : make_float2(0.f, 0.f);
      if (e) ne[k] = v ? __ldg(e + base + P.goff[k]) : 0.f;
    }
  };
  load(tb);
  for (int t = tb; t <= te; ++t) {
    const int cur = (t - tb) & 1, prv = cur ^ 1;
    const long long base = (long long)wrapmod(t, d.nz) * pst;
    float2 pn[K];
    float2 fcur[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      pn[k] = e ? df_add_f(nphi[k], ne[k]) : nphi[k];
      fcur[k] = fq[k];
    }
    if (t < te) {
      load(t + 1);
      // F of the plane whose residual the next iteration computes (plane t)
      if (t >= z0 && t < zend) {
#pragma unroll
        for (int k = 0; k < K; ++k) fq[k] = (P.tmask >> k & 1u) ? F[base + P.goff[k]] : make_float2(0.f, 0.f);
      }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if (P.vmask >> k & 1u) {
        sp[cur][PAD + tid + k * NT] = pn[k];
        if ((P.tmask >> k & 1u) && t >= z0 && t < zend) {
          if (phi_out) phi_out[base + P.goff[k]] = pn[k];
          ps.add(pn[k].x);
          ps.c += pn[k].y;
        }
      }
    }
    const int zp = t - 1;
    if (zp >= z0 && zp < zend) {
      const float2* src = sp[prv] + PAD;
      const long long pbase = (long long)zp * pst;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        if (P.tmask >> k & 1u) {
          const int p = tid + k * NT;
          const long long gi = pbase + P.goff[k];
          const float rv = df_resid(wc[k], src[p - 1], src[p + 1], src[p - WX], src[p + WX], wp[k], pn[k], fcur[k], m);
          r_out[gi] = rv;
          r2 += rv * rv;
          const float fv = __fadd_rn(__fsub_rn(fcur[k].x, m.x), __fsub_rn(fcur[k].y, m.y));
          f2 += fv * fv;
        }
      }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
      wp[k] = wc[k];
      wc[k] = pn[k];
    }
    __syncthreads();
  }
  const double b2 = block_sum_f(r2, shr);
  const double bs = block_sum_acc(ps, shr);
  const double bf = pf2 ? block_sum_f(f2, shr) : 0.0;
  if (tid == 0) {
    const int bid = block_linear_id();
    pr2[bid] = b2;
    psum[bid] = bs;
    if (pf2) pf2[bid] = bf;
  }
}

// Block sizes are multiples of 128 threads: registers are granted to groups of four
// warps, so e.g. 448 threads at 144 registers would not fit in the 64K register file.
constexpr int DTX = 64, DTY = 32, DNT = 512;   // down-leg tile: 72 x 40 region, 6 slots per thread
constexpr int UTX = 64, UTY = 32, UNT = 384;   // up-leg tile: 70 x 38 region, 7 slots per thread
constexpr int FTX = 64, FTY = 16, FNT = 256;   // double-float update tile

template <int V>
size_t down_smem() {
  return (size_t)(V + 1) * 2 * Tile<DTX, DTY, V + 1, DNT>::PLANE * sizeof(float);
}
template <int V>
size_t up_smem() {
  return ((size_t)V * 2 * Tile<UTX, UTY, V, UNT>::PLANE + 3 * CoarseTile<UTX, UTY, V>::CN) * sizeof(float);
}

Coef make_coef(const double* c1, const double* c2, int v, double h) {
  Coef cf{};
  for (int i = 0; i < v && i < 16; ++i) {
    double a, b;
    cheb_constants(c2[i], h, a, b);
    cf.c1[i] = (float)c1[i];
    cf.a[i] = (float)a;
    cf.b[i] = (float)b;
  }
  return cf;
}

int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1)
      n = 152;
  }
  return n;
}

template <int TX, int TY>
Sched make_sched(Dims d, int& ctas) {
  Sched sc;
  sc.tiles_x = (d.nx + TX - 1) / TX;
  sc.total = (long long)sc.tiles_x * ((d.ny + TY - 1) / TY) * d.nz;
  const long long g = sc.total < sm_count() ? sc.total : sm_count();
  ctas = (int)g;
  return sc;
}

template <int V>
cudaError_t down_v(cudaStream_t st, Dims d, const float* r, float* e, float* rc, float ih2, const Coef& cf) {
  static bool attr = false;
  const size_t sm = down_smem<V>();
  if (!attr) {
    cudaError_t err = cudaFuncSetAttribute(k_down_fused<V, DTX, DTY, DNT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (err != cudaSuccess) return err;
    attr = true;
  }
  int ctas = 0;
  const Sched sc = make_sched<DTX, DTY>(d, ctas);
  k_down_fused<V, DTX, DTY, DNT><<<ctas, DNT, sm, st>>>(d, r, e, rc, sc, ih2, cf);
  note_launch();
  return cudaGetLastError();
}

template <int V>
cudaError_t up_v(cudaStream_t st, Dims d, const float* e_in, const float* ec, const float* r, float* e_out,
                 float ih2, const Coef& cf) {
  static bool attr = false;
  const size_t sm = up_smem<V>();
  if (!attr) {
    cudaError_t err = cudaFuncSetAttribute(k_up_fused<V, UTX, UTY, UNT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (err != cudaSuccess) return err;
    attr = true;
  }
  int ctas = 0;
  const Sched sc = make_sched<UTX, UTY>(d, ctas);
  k_up_fused<V, UTX, UTY, UNT><<<ctas, UNT, sm, st>>>(d, e_in, ec, r, e_out, sc, ih2, cf);
  note_launch();
  return cudaGetLastError();
}

}  // namespace

bool fused_degree_supported(int degree) { return degree >= 1 && degree <= 4; }

cudaError_t launch_down_fused(cudaStream_t st, int degree, Dims d, const float* r, float* e, float* rc, double h,
                              const double* c1, const double* c2) {
  const Coef cf = make_coef(c1, c2, degree, h);
  const float ih2 = (float)(1.0 / (h * h));
  switch (degree) {
    case 1: return down_v<1>(st, d, r, e, rc, ih2, cf);
    case 2: return down_v<2>(st, d, r, e, rc, ih2, cf);
    case 3: return down_v<3>(st, d, r, e, rc, ih2, cf);
    case 4: return down_v<4>(st, d, r, e, rc, ih2, cf);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_up_fused(cudaStream_t st, int degree, Dims d, const float* e_in, const float* ec, const float* r,
                            float* e_out, double h, const double* c1, const double* c2) {
  const Coef cf = make_coef(c1, c2, degree, h);
  const float ih2 = (float)(1.0 / (h * h));
  switch (degree) {
    case 1: return up_v<1>(st, d, e_in, ec, r, e_out, ih2, cf);
    case 2: return up_v<2>(st, d, e_in, ec, r, e_out, ih2, cf);
    case 3: return up_v<3>(st, d, e_in, ec, r, e_out, ih2, cf);
    case 4: return up_v<4>(st, d, e_in, ec, r, e_out, ih2, cf);
  }
  return cudaErrorInvalidValue;
}

// ---- double-float update

// z chunk of the double-float update: at least four waves of three CTAs per SM, so
// that enough loads are in flight; the warm-up costs one plane per chunk.
int df_zchunk(Dims d) {
  const long long tiles = (long long)((d.nx + FTX - 1) / FTX) * ((d.ny + FTY - 1) / FTY);
  int zc = d.nz;
  while (zc > 16 && tiles * ((d.nz + zc - 1) / zc) < 4 * 3 * 152) zc = (zc + 1) / 2;
  return zc;
}

long long df_update_residual_partials(Dims d) {
  const int zc = df_zchunk(d);
  return (long long)((d.nx + FTX - 1) / FTX) * ((d.ny + FTY - 1) / FTY) * ((d.nz + zc - 1) / zc);
}

cudaError_t launch_df_update_residual(cudaStream_t st, Dims d, const float2* phi_in, const float* e, const float2* F,
                                      const double* m_dev, float2* phi_out, float* r_out, double* pr2, double* psum,
                                      double* pf2) {
  const int zc = df_zchunk(d);
  const dim3 grid((d.nx + FTX - 1) / FTX, (d.ny + FTY - 1) / FTY, (d.nz + zc - 1) / zc);
  k_df_update_residual<FTX, FTY, FNT><<<grid, FNT, 0, st>>>(d, phi_in, e, F, m_dev, phi_out, r_out, pr2, psum, pf2, zc);
  note_launch();
  return cudaGetLastError();
}

}  // namespace gbmg
