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
      // rows beyond the haloed region (the last thread row's overhang, idle threads) read
      // the region's last row again: cache hits instead of DRAM reads of rows no output
      // depends on
      const int ul = y0 - TL::H + (py < TL::WY ? py : TL::WY - 1);
      goff[j] = gx + wrapmod(ul, d.ny) * d.nx;
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

// z phase of a tile's stream.  The (tile, plane) units [u0, u0 + nz) of one tile are
// split among the CTAs of a contiguous-range schedule over `total` units and G CTAs;
// position p of the tile is plane (phase + p) mod nz (the mesh is periodic in z, so a
// tile's stream may start anywhere).  The phase puts plane 0 where the CTA owning the
// tile's middle unit starts (or, if that CTA entered from the previous tile, where the
// next CTA starts): that CTA then streams plane tau at its step tau, like the chosen
// CTAs of the other tiles, so that neighbouring tiles read the halo rows they share at
// about the same time (from L2 for the second reader).  As plane 0 falls on a CTA
// boundary, no CTA's run within the tile crosses the end of the mesh.  The planes and
// the arithmetic of every output are unchanged.
__device__ __forceinline__ int tile_phase(long long u0, int nz, long long total, long long G) {
  const long long bm = ((u0 + nz / 2 + 1) * G - 1) / total;  // owner of unit u0 + nz / 2
  long long sb = bm * total / G;
  if (sb < u0) sb = (bm + 1) * total / G;
  return sb < u0 + nz ? (int)((u0 + nz - sb) % nz) : 0;
}

__device__ __forceinline__ float2 ld2(const float* p) { return __ldg(reinterpret_cast<const float2*>(p)); }
__device__ __forceinline__ void st2(float* p, float2 v) { *reinterpret_cast<float2*>(p) = v; }

// ------------------------------------------------------------------ down leg
//
// Addressing.  Every shared access of a thread is a compile-time offset from one of two
// pointers (its first pair in the current and in the previous buffer of stage plane 0;
// stage plane s sits 2 s PLANE further); global planes are reached through pointers that
// advance by one plane per iteration (wrapped once at the end of the mesh), plus the
// thread's fixed in-plane offsets; the coarse outputs a thread writes are fixed per
// tile and computed once.  Meshes have fewer than 2^31 cells per plane.

template <int V, class TL>
__device__ __forceinline__ void down_segment(Dims d, const float* __restrict__ r, float* __restrict__ e_out,
                                             float* __restrict__ rc, int x0, int y0, int z0, int zend,
                                             float inv_h2, const Coef& cf, float* sm) {
  constexpr int H = V + 1, R = TL::R, WS = TL::WS, HALF = TL::HALF, PLANE = TL::PLANE, PAD = TL::PAD;
  constexpr int TX = TL::TX, TY = TL::TY, NT = TL::NT;
  constexpr int SP = 2 * PLANE;                 // stage plane s, buffer b at (2 s + b) PLANE
  static_assert(TL::H == H, "down-leg halo");
  constexpr int NCO = (TX / 2) * (TY / 2);      // coarse outputs per tile plane
  constexpr int NQ = (NCO + NT - 1) / NT;       // of them per thread

  const int tid = threadIdx.x;
  const int pst = d.nx * d.ny;
  PPos<TL> P;
  P.init(d, x0, y0);
  const int cnx = d.nx >> 1, cny = d.ny >> 1;
  float* const bs = sm + PAD + P.p0;            // the thread's first pair, stage plane 0, buffer 0
  // coarse outputs of the thread: centre in the z-weighted plane and offset in the coarse
  // plane (-1: none)
  int qpp[NQ], qco[NQ];
#pragma unroll
  for (int i = 0; i < NQ; ++i) {
    const int q = tid + i * NT;
    const int ccx = q % (TX / 2), ccy = q / (TX / 2);
    const int cX = (x0 >> 1) + ccx, cY = (y0 >> 1) + ccy;
    qpp[i] = (H + 2 * ccy) * WS + TL::HX / 2 + ccx;
    qco[i] = (q < NCO && cX < cnx && cY < cny) ? cY * cnx + cX : -1;
  }
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
  int zl = wrapmod(tb, d.nz);                   // plane of the latest load of r
  const float* rl = r + (size_t)zl * pst;
#pragma unroll
  for (int j = 0; j < R; ++j) rnext[j] = ld2(rl + P.goff[j]);
  for (int t = tb; t <= te; ++t) {
    const int cur = (t - tb) & 1;
    float* const bc = bs + (cur ? PLANE : 0);
    const float* const bp = bs + (cur ? 0 : PLANE);
#pragma unroll
    for (int j = 0; j < R; ++j) {
#pragma unroll
      for (int i = V; i > 0; --i) rq[i][j] = rq[i - 1][j];
      rq[0][j] = rnext[j];
    }
    if (t < te) {
      if (++zl == d.nz) {
        zl = 0;
        rl = r;
      } else {
        rl += pst;
      }
#pragma unroll
      for (int j = 0; j < R; ++j) rnext[j] = ld2(rl + P.goff[j]);
    }
    float2 en[V + 1][R], dn[V + 1][R];
    // stage 1 (pointwise, e starts at zero): e_1 = d_1 = c2_0 D^-1 r
    {
      const float2 A = bcast(cf.a[0]), MB = bcast(-cf.b[0]), C1 = bcast(cf.c1[0]);
#pragma unroll
      for (int j = 0; j < R; ++j) {
        float2 dd = Z;
        en[1][j] = p_cheb(Z, rq[0][j], Z, Z, dd, A, MB, C1);
        dn[1][j] = dd;
        bc[j * WS] = en[1][j].x;
        bc[j * WS + HALF] = en[1][j].y;
      }
    }
    // stages 2..V: Chebyshev steps with the stencil on e_{s-1}
#pragma unroll
    for (int s = 2; s <= V; ++s) {
      const float* const sE = bp + (s - 2) * SP;
      float* const dE = bc + (s - 1) * SP;
      const float2 A = bcast(cf.a[s - 1]), MB = bcast(-cf.b[s - 1]), C1 = bcast(cf.c1[s - 1]);
#pragma unroll
      for (int j = 0; j < R; ++j) {
        const int o = j * WS;
        const float2 c = wc[s][j];
        const float2 ym = j > 0 ? wc[s][j - 1] : make_float2(sE[o - WS], sE[o - WS + HALF]);
        const float2 yp = j < R - 1 ? wc[s][j + 1] : make_float2(sE[o + WS], sE[o + WS + HALF]);
        const float2 sn = p_nbr_sum(sE[o - 1 + HALF], sE[o + 1], c, ym, yp, wp[s][j], en[s - 1][j]);
        float2 dd = dh[s][j];
        en[s][j] = p_cheb(c, rq[s - 1][j], sn, c, dd, A, MB, C1);
        dn[s][j] = dd;
        dE[o] = en[s][j].x;
        dE[o + HALF] = en[s][j].y;
      }
    }
    {
      const int zp = t - V + 1;                 // plane of e_V finished in this iteration
      if (zp >= z0 && zp < zend) {
        float* const ez = e_out + (size_t)zp * pst;
#pragma unroll
        for (int j = 0; j < R; ++j)
          if (P.tmask >> j & 1u) st2(ez + P.goff[j], en[V][j]);
      }
    }
    // residual stage at plane t - V, then z weights of the restriction at c = t - V - 1
    {
      const float* const sE = bp + (V - 1) * SP;
      float* const zE = bc + V * SP;
      const int c = t - V - 1;
      const bool cz = ((c & 1) == 0) && c >= z0 && c < zend;
#pragma unroll
      for (int j = 0; j < R; ++j) {
        const int o = j * WS;
        const float2 cc = wc[V + 1][j];
        const float2 ym = j > 0 ? wc[V + 1][j - 1] : make_float2(sE[o - WS], sE[o - WS + HALF]);
        const float2 yp = j < R - 1 ? wc[V + 1][j + 1] : make_float2(sE[o + WS], sE[o + WS + HALF]);
        const float2 sn = p_nbr_sum(sE[o - 1 + HALF], sE[o + 1], cc, ym, yp, wp[V + 1][j], en[V][j]);
        const float2 rn = p_resid(rq[V][j], sn, cc, MIH2);
        if (cz) {
          const float2 zw = p_fw3(rsp[j], rsc[j], rn);
          zE[o] = zw.x;
          zE[o + HALF] = zw.y;
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
        const float* const zE = sm + PAD + V * SP + (cur ? 0 : PLANE);
        float* const rcz = rc + (size_t)(c >> 1) * (cnx * cny);
#pragma unroll
        for (int i = 0; i < NQ; ++i) {
          if (qco[i] < 0) continue;
          const float* const e0 = zE + qpp[i];
          const float* const o0 = e0 + HALF;
          const float y0v = fw3(o0[-1 - WS], o0[-1], o0[-1 + WS]);
          const float y1v = fw3(e0[-WS], e0[0], e0[WS]);
          const float y2v = fw3(o0[-WS], o0[0], o0[WS]);
          rcz[qco[i]] = fw3(y0v, y1v, y2v);
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

// Coarse nodes under the haloed fine region: I in [CX0, CX0 + CU), J in [CY0, CY0 + CH),
// the +1 neighbour included; CH covers the rows of every thread column, idle ones too.
// The row stride CW >= CU is chosen like the planes' row stride: threads of a warp in
// the next row block read coarse rows about R/2 further on, and the jump should keep
// the warp's 32 loads on distinct banks.
constexpr int coarse_stride(int wxp, int r) {
  for (int cw = wxp + 1; cw < wxp + 33; ++cw)
    if (((r / 2) * cw - wxp) % 32 == 0) return cw;
  return wxp + 1;
}

template <class TL>
struct PCoarse {
  static constexpr int CU = TL::WXP + 1;                  // coarse columns used
  static constexpr int CW = coarse_stride(TL::WXP, TL::R);
  static constexpr int CH = (TL::ROWS + 1) / 2 + 2;
  static constexpr int CN = CW * CH;
  static constexpr int NXR = (TL::R + 1) / 2 + 1;        // coarse rows under a thread column
};

// e_0 = e + P e_c for the R pairs of a column: the trilinear prolongation as nested
// midpoints (x, then y, then z; stencil.cuh's prolong_value), the x midpoints of each
// coarse row formed once per column.  Row j of the column has y parity PAR ^ (j & 1)
// and first coarse row (PAR + j) / 2 relative to the column's.
template <int PAR, class TL>
__device__ __forceinline__ void prolong_column(const float* __restrict__ c0, const float* __restrict__ c1, bool zodd,
                                               float2 (&e)[TL::R]) {
  using CT = PCoarse<TL>;
  constexpr int R = TL::R, NXR = CT::NXR, CW = CT::CW;
  float2 X[NXR], Y[NXR];
#pragma unroll
  for (int k = 0; k < NXR; ++k) {
    const float v0 = c0[k * CW];
    X[k] = make_float2(v0, half_sum(v0, c0[k * CW + 1]));
  }
  if (zodd) {
#pragma unroll
    for (int k = 0; k < NXR; ++k) {
      const float v0 = c1[k * CW];
      Y[k] = make_float2(v0, half_sum(v0, c1[k * CW + 1]));
    }
  }
#pragma unroll
  for (int j = 0; j < R; ++j) {
    const int J = (PAR + j) >> 1;
    const bool dy = ((PAR + j) & 1) != 0;
    float2 pv = dy ? p_half_sum(X[J], X[J + 1]) : X[J];
    if (zodd) pv = p_half_sum(pv, dy ? p_half_sum(Y[J], Y[J + 1]) : Y[J]);
    e[j] = p_add(e[j], pv);
  }
}

template <int V, class TL>
__device__ __forceinline__ void up_segment(Dims d, const float* __restrict__ e_in, const float* __restrict__ ec,
                                           const float* __restrict__ r, float* __restrict__ e_out, int x0, int y0,
                                           int z0, int zend, float inv_h2, const Coef& cf, float* sm) {
  constexpr int H = V, R = TL::R, WS = TL::WS, HALF = TL::HALF, PLANE = TL::PLANE, PAD = TL::PAD;
  constexpr int NT = TL::NT, SP = 2 * PLANE;
  static_assert(TL::H == H, "up-leg halo");
  using CT = PCoarse<TL>;
  constexpr int CW = CT::CW, CN = CT::CN, CU = CT::CU, CH = CT::CH;
  constexpr int CL = (CU * CH + NT - 1) / NT;   // coarse cells a thread loads per plane
  // stage plane s (e_s, s = 0..V-1), buffer b at (2 s + b) PLANE; then three coarse planes
  float* const cring = sm + V * SP;

  const int tid = threadIdx.x;
  const int pst = d.nx * d.ny;
  const int cnx = d.nx >> 1, cny = d.ny >> 1, cnz = d.nz >> 1;
  const int cpst = cnx * cny;
  PPos<TL> P;
  P.init(d, x0, y0);
  float* const bs = sm + PAD + P.p0;
  // the column's rows: y parity of the first (tiles start on even rows) and the coarse
  // row under it, relative to the ring's first row
  const int CX0 = floor_half(x0 - TL::HX), CY0 = floor_half(y0 - H);
  const int par0 = (H + P.pyb * R) & 1;
  const int cb0 = tid < TL::NCOL ? (floor_half(y0 - H + P.pyb * R) - CY0) * CW + P.px : 0;
  // coarse cells of the ring this thread loads: in-plane offset (-1: none) and ring offset
  int cgo[CL], cso[CL];
#pragma unroll
  for (int i = 0; i < CL; ++i) {
    const int q = tid + i * NT;
    const int ci = q % CU, cj = q / CU;
    cso[i] = cj * CW + ci;
    cgo[i] = q < CU * CH ? wrapmod(CX0 + ci, cnx) + wrapmod(CY0 + cj, cny) * cnx : -1;
  }
  // coarse planes: slot of plane Ku (Ku = floor(t / 2)) and the plane of the next load
  const int tb = z0 - V, te = zend + V - 1;
  const int K0 = floor_half(tb);
  int ks = mod3(K0);
  int kl = wrapmod(K0, cnz);
  const float* ecl = ec + (size_t)kl * cpst;
  auto load_coarse = [&](float (&vals)[CL]) {
#pragma unroll
    for (int i = 0; i < CL; ++i) vals[i] = cgo[i] >= 0 ? __ldg(ecl + cgo[i]) : 0.f;
  };
  auto store_coarse = [&](int slot, const float (&vals)[CL]) {
    float* const dst = cring + slot * CN;
#pragma unroll
    for (int i = 0; i < CL; ++i)
      if (cgo[i] >= 0) dst[cso[i]] = vals[i];
  };
  auto next_coarse = [&]() {
    if (++kl == cnz) {
      kl = 0;
      ecl = ec;
    } else {
      ecl += cpst;
    }
  };
  const float2 Z = bcast(0.f);

  float2 rq[V + 1][R];
  float2 wp[V + 1][R], wc[V + 1][R];
  float2 dh[V + 1][R];
  float2 rnext[R], enext[R];
#pragma unroll
  for (int j = 0; j < R; ++j) {
#pragma unroll
    for (int i = 0; i <= V; ++i) rq[i][j] = Z, dh[i][j] = Z, wp[i][j] = Z, wc[i][j] = Z;
  }
  int zl = wrapmod(tb, d.nz);                   // plane of the latest fine loads
  size_t ol = (size_t)zl * pst;
  {
    float cv[CL];
    load_coarse(cv);
    store_coarse(ks, cv);
    next_coarse();
    load_coarse(cv);
    store_coarse(ks == 2 ? 0 : ks + 1, cv);
    next_coarse();
  }
#pragma unroll
  for (int j = 0; j < R; ++j) {
    rnext[j] = ld2(r + ol + P.goff[j]);
    enext[j] = ld2(e_in + ol + P.goff[j]);
  }
  __syncthreads();
  for (int t = tb; t <= te; ++t) {
    const int cur = (t - tb) & 1;
    float* const bc = bs + (cur ? PLANE : 0);
    const float* const bp = bs + (cur ? 0 : PLANE);
    const bool zodd = (t & 1) != 0;
    if (!zodd && t != tb) ks = ks == 2 ? 0 : ks + 1;   // Ku advanced
    const int ks1 = ks == 2 ? 0 : ks + 1;
    float2 en[V + 1][R], dn[V + 1][R];
    // next coarse plane (needed from the next even t on), stored at the end of this iteration
    float cv[CL];
    const bool need_c = zodd && t < te;
    if (need_c) {
      load_coarse(cv);
      next_coarse();
    }
#pragma unroll
    for (int j = 0; j < R; ++j) {
#pragma unroll
      for (int i = V; i > 0; --i) rq[i][j] = rq[i - 1][j];
      rq[0][j] = rnext[j];
      en[0][j] = enext[j];
    }
    if (t < te) {
      if (++zl == d.nz) {
        zl = 0;
        ol = 0;
      } else {
        ol += pst;
      }
#pragma unroll
      for (int j = 0; j < R; ++j) {
        rnext[j] = ld2(r + ol + P.goff[j]);
        enext[j] = ld2(e_in + ol + P.goff[j]);
      }
    }
    // stage 0: e_0 = e + P e_c (pointwise)
    {
      const float* const c0 = cring + ks * CN + cb0;
      const float* const c1 = cring + ks1 * CN + cb0;
      if constexpr (R % 2 == 0) {
        prolong_column<H & 1, TL>(c0, c1, zodd, en[0]);
      } else {
        if (par0) prolong_column<1, TL>(c0, c1, zodd, en[0]);
        else prolong_column<0, TL>(c0, c1, zodd, en[0]);
      }
#pragma unroll
      for (int j = 0; j < R; ++j) {
        bc[j * WS] = en[0][j].x;
        bc[j * WS + HALF] = en[0][j].y;
      }
    }
    // stages 1..V: Chebyshev post-smoothing steps at plane t - s
#pragma unroll
    for (int s = 1; s <= V; ++s) {
      const float* const sE = bp + (s - 1) * SP;
      float* const dE = bc + s * SP;
      const float2 A = bcast(cf.a[s - 1]), MB = bcast(-cf.b[s - 1]), C1 = bcast(cf.c1[s - 1]);
#pragma unroll
      for (int j = 0; j < R; ++j) {
        const int o = j * WS;
        const float2 c = wc[s][j];
        const float2 ym = j > 0 ? wc[s][j - 1] : make_float2(sE[o - WS], sE[o - WS + HALF]);
        const float2 yp = j < R - 1 ? wc[s][j + 1] : make_float2(sE[o + WS], sE[o + WS + HALF]);
        const float2 sn = p_nbr_sum(sE[o - 1 + HALF], sE[o + 1], c, ym, yp, wp[s][j], en[s - 1][j]);
        float2 dd = s == 1 ? Z : dh[s][j];
        en[s][j] = p_cheb(c, rq[s][j], sn, c, dd, A, MB, C1);
        dn[s][j] = dd;
        if (s < V) {
          dE[o] = en[s][j].x;
          dE[o + HALF] = en[s][j].y;
        }
      }
    }
    {
      const int zp = t - V;
      if (zp >= z0 && zp < zend) {
        float* const ez = e_out + (size_t)zp * pst;
#pragma unroll
        for (int j = 0; j < R; ++j)
          if (P.tmask >> j & 1u) st2(ez + P.goff[j], en[V][j]);
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
    if (need_c) store_coarse(ks1 == 2 ? 0 : ks1 + 1, cv);
    __syncthreads();
  }
}

}  // namespace legs
}  // namespace gbmg
