// Device code of the temporally blocked FP32 level kernels (the fused legs): tile
// geometry, per-thread pair columns and one z segment of the down leg (Chebyshev
// pre-smoothing from zero, residual, full-weighting restriction) and of the up leg
// (trilinear prolongation + correction, Chebyshev post-smoothing).  Used by the
// per-level kernels of legs.cu and by the batched persistent kernel.
#pragma once
#include "kernels.h"
#include "packed.cuh"

namespace gbmg {
namespace legs {

__device__ __forceinline__ int wrapmod(int i, int n) {
  const int r = i % n;
  return r < 0 ? r + n : r;
}
__device__ __forceinline__ int floor_half(int v) { return v >= 0 ? v / 2 : -((1 - v) / 2); }
__device__ __forceinline__ int mod3(int v) {
  const int r = v % 3;
  return r < 0 ? r + 3 : r;
}

// ------------------------------------------------------------------ tile geometry

template <int TX_, int TY_, int H_, int NT_, int R_>
struct PTile {
  static constexpr int TX = TX_, TY = TY_, H = H_, NT = NT_, R = R_;
  static constexpr int HX = (H + 1) / 2 * 2;            // x halo in whole pairs
  static constexpr int WXP = TX / 2 + HX;               // pairs per haloed row
  static constexpr int WS = conflict_free_stride(WXP, R);  // row stride of the planes
  static constexpr int WY = TY + 2 * H;                 // haloed rows
  static constexpr int NCOL = WXP * ((WY + R - 1) / R);  // columns of R pairs
  static constexpr int ROWS = (NT + WXP - 1) / WXP * R;  // plane rows, idle threads included
  static constexpr int PAD = WS + 1;                    // p +- 1, p +- WS stay inside
  static constexpr int HALF = ROWS * WS + 2 * PAD;      // floats of one parity half-plane
  static constexpr int PLANE = 2 * HALF;
  static_assert(TX % 2 == 0 && TY % 2 == 0, "tiles cover whole pairs and coarse cells");
  static_assert(NCOL <= NT, "one column per thread");
};

// The thread's column: plane index of its first pair and the global (z = 0) offset
// of the even cell of each pair; tmask marks pairs inside the output tile.
template <class TL>
struct PPos {
  int px, pyb, p0;
  int goff[TL::R];
  unsigned tmask;
  __device__ __forceinline__ void init(Dims d, int x0, int y0) {
    px = threadIdx.x % TL::WXP;
    pyb = threadIdx.x / TL::WXP;
    p0 = pyb * TL::R * TL::WS + px;
    tmask = 0;
    const int ux = x0 - TL::HX + 2 * px;
    const int gx = wrapmod(ux, d.nx);
#pragma unroll
    for (int j = 0; j < TL::R; ++j) {
      const int py = pyb * TL::R + j, uy = y0 - TL::H + py;
      goff[j] = gx + wrapmod(uy, d.ny) * d.nx;
      const bool in = threadIdx.x < TL::NCOL && px >= TL::HX / 2 && px < TL::HX / 2 + TL::TX / 2 &&
                      py >= TL::H && py < TL::H + TL::TY && ux < d.nx && uy < d.ny;
      if (in) tmask |= 1u << j;
    }
  }
};

// Folded Chebyshev constants of one level: c1 and a = c2 D^-1, b = a / h^2 per step.
struct Coef {
  float c1[16];
  float a[16];
  float b[16];
};

struct Sched {
  int tiles_x;
  long long total;  // tiles * nz
};

__device__ __forceinline__ float2 ld2(const float* p) { return __ldg(reinterpret_cast<const float2*>(p)); }
__device__ __forceinline__ void st2(float* p, float2 v) { *reinterpret_cast<float2*>(p) = v; }

// ------------------------------------------------------------------ down leg

template <int V, class TL>
__device__ __forceinline__ void down_segment(Dims d, const float* __restrict__ r, float* __restrict__ e_out,
                                             float* __restrict__ rc, int x0, int y0, int z0, int zend,
                                             float inv_h2, const Coef& cf, float* sm) {
  constexpr int H = V + 1, R = TL::R, WS = TL::WS, HALF = TL::HALF, PLANE = TL::PLANE, PAD = TL::PAD;
  constexpr int TX = TL::TX, TY = TL::TY, NT = TL::NT;
  static_assert(TL::H == H, "down-leg halo");
  constexpr int NCO = (TX / 2) * (TY / 2);  // coarse outputs per tile plane
  // plane(s, b): even half at the pointer, odd half HALF later; s = 0..V-1 holds
  // e_{s+1}, s = V the z-weighted residual
  auto plane = [&](int s, int b) -> float* { return sm + (s * 2 + b) * PLANE + PAD; };

  const int tid = threadIdx.x;
  const long long pst = (long long)d.nx * d.ny;
  PPos<TL> P;
  P.init(d, x0, y0);
  const Dims dc{d.nx / 2, d.ny / 2, d.nz / 2};
  const float2 Z = bcast(0.f), MIH2 = bcast(-inv_h2);

  float2 rq[V + 1][R];              // rq[i][j] = r at plane t - i
  float2 wp[V + 2][R], wc[V + 2][R];  // stage s input window: planes zp - 1, zp
  float2 dh[V + 1][R];              // d_{s-1} at stage s's plane
  float2 rsp[R], rsc[R];            // residual window
  float2 rnext[R];
#pragma unroll
  for (int j = 0; j < R; ++j) {
#pragma unroll
    for (int i = 0; i <= V; ++i) rq[i][j] = Z, dh[i][j] = Z;
#pragma unroll
    for (int s = 0; s < V + 2; ++s) wp[s][j] = Z, wc[s][j] = Z;
    rsp[j] = rsc[j] = Z;
  }
  // the last coarse plane c = zend - 1 (a segment may end on an odd plane) is
  // written at t = c + V + 2
  const int tb = z0 - H, te = zend + V + 1;
  {
    const float* base = r + (long long)wrapmod(tb, d.nz) * pst;
#pragma unroll
    for (int j = 0; j < R; ++j) rnext[j] = ld2(base + P.goff[j]);
  }
  for (int t = tb; t <= te; ++t) {
    const int cur = (t - tb) & 1, prv = cur ^ 1;
#pragma unroll
    for (int j = 0; j < R; ++j) {
#pragma unroll
      for (int i = V; i > 0; --i) rq[i][j] = rq[i - 1][j];
      rq[0][j] = rnext[j];
    }
    if (t < te) {
      const float* base = r + (long long)wrapmod(t + 1, d.nz) * pst;
#pragma unroll
      for (int j = 0; j < R; ++j) rnext[j] = ld2(base + P.goff[j]);
    }
    float2 en[V + 1][R], dn[V + 1][R];
    // stage 1 (pointwise, e starts at zero): e_1 = d_1 = c2_0 D^-1 r
    {
      float* dE = plane(0, cur);
      const float2 A = bcast(cf.a[0]), MB = bcast(-cf.b[0]), C1 = bcast(cf.c1[0]);
#pragma unroll
      for (int j = 0; j < R; ++j) {
        float2 dd = Z;
        en[1][j] = p_cheb(Z, rq[0][j], Z, Z, dd, A, MB, C1);
        dn[1][j] = dd;
        const int p = P.p0 + j * WS;
        dE[p] = en[1][j].x;
        dE[p + HALF] = en[1][j].y;
      }
    }
    // stages 2..V: Chebyshev steps with the stencil on e_{s-1}
#pragma unroll
    for (int s = 2; s <= V; ++s) {
      const float* sE = plane(s - 2, prv);
      float* dE = plane(s - 1, cur);
      const int zp = t - s + 1;
      const float2 A = bcast(cf.a[s - 1]), MB = bcast(-cf.b[s - 1]), C1 = bcast(cf.c1[s - 1]);
#pragma unroll
      for (int j = 0; j < R; ++j) {
        const int p = P.p0 + j * WS;
        const float2 c = wc[s][j];
        const float2 ym = j > 0 ? wc[s][j - 1] : make_float2(sE[p - WS], sE[p - WS + HALF]);
        const float2 yp = j < R - 1 ? wc[s][j + 1] : make_float2(sE[p + WS], sE[p + WS + HALF]);
        const float2 sn = p_nbr_sum(sE[p - 1 + HALF], sE[p + 1], c, ym, yp, wp[s][j], en[s - 1][j]);
        float2 dd = dh[s][j];
        en[s][j] = p_cheb(c, rq[s - 1][j], sn, c, dd, A, MB, C1);
        dn[s][j] = dd;
        dE[p] = en[s][j].x;
        dE[p + HALF] = en[s][j].y;
        if (s == V && (P.tmask >> j & 1u) && zp >= z0 && zp < zend) st2(e_out + (long long)zp * pst + P.goff[j], en[s][j]);
      }
    }
    if (V == 1) {
      const int zp = t;
#pragma unroll
      for (int j = 0; j < R; ++j)
        if ((P.tmask >> j & 1u) && zp >= z0 && zp < zend) st2(e_out + (long long)zp * pst + P.goff[j], en[1][j]);
    }
    // residual stage at plane t - V, then z weights of the restriction at c = t - V - 1
    {
      const float* sE = plane(V - 1, prv);
      float* zE = plane(V, cur);
      const int c = t - V - 1;
      const bool cz = ((c & 1) == 0) && c >= z0 && c < zend;
#pragma unroll
      for (int j = 0; j < R; ++j) {
        const int p = P.p0 + j * WS;
        const float2 cc = wc[V + 1][j];
        const float2 ym = j > 0 ? wc[V + 1][j - 1] : make_float2(sE[p - WS], sE[p - WS + HALF]);
        const float2 yp = j < R - 1 ? wc[V + 1][j + 1] : make_float2(sE[p + WS], sE[p + WS + HALF]);
        const float2 sn = p_nbr_sum(sE[p - 1 + HALF], sE[p + 1], cc, ym, yp, wp[V + 1][j], en[V][j]);
        const float2 rn = p_resid(rq[V][j], sn, cc, MIH2);
        if (cz) {
          const float2 zw = p_fw3(rsp[j], rsc[j], rn);
          zE[p] = zw.x;
          zE[p + HALF] = zw.y;
        }
        rsp[j] = rsc[j];
        rsc[j] = rn;
      }
    }
    // coarse output from the z-weighted plane of the previous iteration: y weights
    // for the x offsets -1, 0, +1 (odd cell of the pair to the left, even and odd
    // cell of the centre pair), then x weights
    {
      const int c = t - V - 2;
      if (((c & 1) == 0) && c >= z0 && c < zend) {
        const float* zE = plane(V, prv);
        const float* zO = zE + HALF;
        for (int q = tid; q < NCO; q += NT) {
          const int ccx = q % (TX / 2), ccy = q / (TX / 2);
          const int cX = x0 / 2 + ccx, cY = y0 / 2 + ccy;
          if (cX < dc.nx && cY < dc.ny) {
            const int pp = (H + 2 * ccy) * WS + TL::HX / 2 + ccx;
            const float y0v = fw3(zO[pp - 1 - WS], zO[pp - 1], zO[pp - 1 + WS]);
            const float y1v = fw3(zE[pp - WS], zE[pp], zE[pp + WS]);
            const float y2v = fw3(zO[pp - WS], zO[pp], zO[pp + WS]);
            rc[((long long)(c >> 1) * dc.ny + cY) * dc.nx + cX] = fw3(y0v, y1v, y2v);
          }
        }
      }
    }
    // advance the z windows
#pragma unroll
    for (int j = 0; j < R; ++j) {
#pragma unroll
      for (int s = 2; s <= V + 1; ++s) {
        wp[s][j] = wc[s][j];
        wc[s][j] = en[s - 1][j];
      }
#pragma unroll
      for (int s = 2; s <= V; ++s) dh[s][j] = dn[s - 1][j];
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ up leg

// Coarse nodes under the haloed fine region: I in [CX0, CX0 + CW), J in [CY0, CY0 + CH),
// the +1 neighbour included.
// The row stride CW >= WXP + 1 is chosen like the planes' row stride: threads of a
// warp in the next row block read coarse row J + R/2, and the jump must keep the
// warp's 32 loads on distinct banks.
constexpr int coarse_stride(int wxp, int r) {
  for (int cw = wxp + 1; cw < wxp + 33; ++cw)
    if (((r / 2) * cw - wxp) % 32 == 0) return cw;
  return wxp + 1;
}

template <class TL>
struct PCoarse {
  static constexpr int CU = TL::WXP + 1;                  // coarse columns used
  static constexpr int CW = coarse_stride(TL::WXP, TL::R);
  static constexpr int CH = TL::WY / 2 + 2;
  static constexpr int CN = CW * CH;
};

template <int V, class TL>
__device__ __forceinline__ void up_segment(Dims d, const float* __restrict__ e_in, const float* __restrict__ ec,
                                           const float* __restrict__ r, float* __restrict__ e_out, int x0, int y0,
                                           int z0, int zend, float inv_h2, const Coef& cf, float* sm) {
  constexpr int H = V, R = TL::R, WS = TL::WS, HALF = TL::HALF, PLANE = TL::PLANE, PAD = TL::PAD;
  constexpr int NT = TL::NT;
  static_assert(TL::H == H, "up-leg halo");
  using CT = PCoarse<TL>;
  constexpr int CW = CT::CW, CN = CT::CN, CL = (CN + NT - 1) / NT;
  // plane(s, b): e_s for s = 0..V-1 (e_0 = e + P e_c); then three coarse planes
  auto plane = [&](int s, int b) -> float* { return sm + (s * 2 + b) * PLANE + PAD; };
  float* cring = sm + V * 2 * PLANE;

  const int tid = threadIdx.x;
  const long long pst = (long long)d.nx * d.ny;
  const Dims dc{d.nx / 2, d.ny / 2, d.nz / 2};
  const long long cpst = (long long)dc.nx * dc.ny;
  PPos<TL> P;
  P.init(d, x0, y0);
  const float2 Z = bcast(0.f);
  // coarse node under each pair (offset in the coarse tile) and the y parity
  const int CX0 = floor_half(x0 - TL::HX), CY0 = floor_half(y0 - H);
  int co[R];
  unsigned oddy = 0;
#pragma unroll
  for (int j = 0; j < R; ++j) {
    const int py = P.pyb * R + j;
    co[j] = 0;
    if (tid < TL::NCOL && py < TL::WY) {
      const int I = CX0 + P.px, uy = y0 - H + py, J = floor_half(uy);
      co[j] = (J - CY0) * CW + (I - CX0);
      oddy |= (unsigned)(uy - 2 * J) << j;
    }
  }
  // coarse tile cells this thread loads
  int cgo[CL];
#pragma unroll
  for (int i = 0; i < CL; ++i) {
    const int q = tid + i * NT;
    cgo[i] = -1;
    if (q < CN && q % CW < CT::CU) cgo[i] = wrapmod(CX0 + q % CW, dc.nx) + wrapmod(CY0 + q / CW, dc.ny) * dc.nx;
  }
  auto load_coarse = [&](int Ku, float (&vals)[CL]) {
    const float* base = ec + (long long)wrapmod(Ku, dc.nz) * cpst;
#pragma unroll
    for (int i = 0; i < CL; ++i) vals[i] = cgo[i] >= 0 ? __ldg(base + cgo[i]) : 0.f;
  };
  auto store_coarse = [&](int Ku, const float (&vals)[CL]) {
    float* dst = cring + mod3(Ku) * CN;
#pragma unroll
    for (int i = 0; i < CL; ++i)
      if (cgo[i] >= 0) dst[tid + i * NT] = vals[i];
  };

  float2 rq[V + 1][R];
  float2 wp[V + 1][R], wc[V + 1][R];
  float2 dh[V + 1][R];
  float2 rnext[R], enext[R];
#pragma unroll
  for (int j = 0; j < R; ++j) {
#pragma unroll
    for (int i = 0; i <= V; ++i) rq[i][j] = Z, dh[i][j] = Z, wp[i][j] = Z, wc[i][j] = Z;
  }
  const int tb = z0 - V, te = zend + V - 1;
  auto load = [&](int t) {
    const long long base = (long long)wrapmod(t, d.nz) * pst;
#pragma unroll
    for (int j = 0; j < R; ++j) {
      rnext[j] = ld2(r + base + P.goff[j]);
      enext[j] = ld2(e_in + base + P.goff[j]);
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
    float2 en[V + 1][R], dn[V + 1][R];
    const int Ku = floor_half(t);
    const bool zodd = (t - 2 * Ku) != 0;
    // next coarse plane (needed from the next even t on), stored at the end of this iteration
    float cv[CL];
    const bool need_c = zodd && t < te;
    if (need_c) load_coarse(Ku + 2, cv);
#pragma unroll
    for (int j = 0; j < R; ++j) {
#pragma unroll
      for (int i = V; i > 0; --i) rq[i][j] = rq[i - 1][j];
      rq[0][j] = rnext[j];
      en[0][j] = enext[j];
    }
    if (t < te) load(t + 1);
    // stage 0: e_0 = e + P e_c (pointwise): x, then y, then z midpoints
    {
      const float* c0 = cring + mod3(Ku) * CN;
      const float* c1 = cring + mod3(Ku + 1) * CN;
      float* dE = plane(0, cur);
#pragma unroll
      for (int j = 0; j < R; ++j) {
        const bool dy = oddy >> j & 1u;
        auto row = [&](const float* cp, int off) -> float2 {
          const float v0 = cp[off];
          return make_float2(v0, half_sum(v0, cp[off + 1]));
        };
        auto pl = [&](const float* cp) -> float2 {
          const float2 v0 = row(cp, co[j]);
          return dy ? p_half_sum(v0, row(cp, co[j] + CW)) : v0;
        };
        const float2 v0 = pl(c0);
        const float2 pv = zodd ? p_half_sum(v0, pl(c1)) : v0;
        en[0][j] = p_add(en[0][j], pv);
        const int p = P.p0 + j * WS;
        dE[p] = en[0][j].x;
        dE[p + HALF] = en[0][j].y;
      }
    }
    // stages 1..V: Chebyshev post-smoothing steps at plane t - s
#pragma unroll
    for (int s = 1; s <= V; ++s) {
      const float* sE = plane(s - 1, prv);
      const int zp = t - s;
      const float2 A = bcast(cf.a[s - 1]), MB = bcast(-cf.b[s - 1]), C1 = bcast(cf.c1[s - 1]);
#pragma unroll
      for (int j = 0; j < R; ++j) {
        const int p = P.p0 + j * WS;
        const float2 c = wc[s][j];
        const float2 ym = j > 0 ? wc[s][j - 1] : make_float2(sE[p - WS], sE[p - WS + HALF]);
        const float2 yp = j < R - 1 ? wc[s][j + 1] : make_float2(sE[p + WS], sE[p + WS + HALF]);
        const float2 sn = p_nbr_sum(sE[p - 1 + HALF], sE[p + 1], c, ym, yp, wp[s][j], en[s - 1][j]);
        float2 dd = s == 1 ? Z : dh[s][j];
        en[s][j] = p_cheb(c, rq[s][j], sn, c, dd, A, MB, C1);
        dn[s][j] = dd;
        if (s < V) {
          float* dE = plane(s, cur);
          dE[p] = en[s][j].x;
          dE[p + HALF] = en[s][j].y;
        } else if ((P.tmask >> j & 1u) && zp >= z0 && zp < zend) {
          st2(e_out + (long long)zp * pst + P.goff[j], en[s][j]);
        }
      }
    }
#pragma unroll
    for (int j = 0; j < R; ++j) {
#pragma unroll
      for (int s = 1; s <= V; ++s) {
        wp[s][j] = wc[s][j];
        wc[s][j] = en[s - 1][j];
      }
#pragma unroll
      for (int s = 2; s <= V; ++s) dh[s][j] = dn[s - 1][j];
    }
    if (need_c) store_coarse(Ku + 2, cv);
    __syncthreads();
  }
}

}  // namespace legs
}  // namespace gbmg
