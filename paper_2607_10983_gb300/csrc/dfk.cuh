// Device code of the fused double-float update and residual of the finest level:
// tile geometry and one tile / z range of phi' = phi + e and r' = F - m - A phi'
// (Sec. 3.2 defect correction) on packed x-pairs.  Used by the per-level kernel of
// fused_kernels.cu and by the batched persistent kernel.
#pragma once
#include "kernels.h"
#include "packed.cuh"

namespace gbmg {
namespace dfk {

__device__ __forceinline__ int wrapmod(int i, int n) {
  const int r = i % n;
  return r < 0 ? r + n : r;
}

// Tile of the double-float kernel: x-pairs with a one-pair halo in x (one cell is
// needed), one row of halo in y, columns of R pairs per thread, even/odd cells and
// hi/lo parts in four separate arrays per plane, three planes in a ring (z - 1, z,
// z + 1 of the update).
template <int TX_, int TY_, int R_, int NT_>
struct DTile {
  static constexpr int TX = TX_, TY = TY_, R = R_, NT = NT_;
  static constexpr int WXP = TX / 2 + 2;                      // pairs per haloed row
  static constexpr int WY = TY + 2;                           // haloed rows
  static constexpr int NCOL = WXP * ((WY + R - 1) / R);
  static constexpr int WS = conflict_free_stride(WXP, R);     // row stride of the arrays
  static constexpr int ROWS = (NT + WXP - 1) / WXP * R;       // idle threads included
  static constexpr int PAD = WS + 1;
  static constexpr int ARR = ROWS * WS + 2 * PAD;             // floats of one array
  static constexpr int PLANE = 4 * ARR;                       // even hi, even lo, odd hi, odd lo
  static_assert(NCOL <= NT, "one column per thread");
};

__device__ __forceinline__ DF2 ld_df2(const float2* p) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  return DF2{make_float2(v.x, v.z), make_float2(v.y, v.w)};
}
__device__ __forceinline__ void st_df2(float2* p, const DF2& v) {
  *reinterpret_cast<float4*>(p) = make_float4(v.hi.x, v.lo.x, v.hi.y, v.lo.y);
}

// One tile (x0, y0) and z range [z0, zend) of the fused update and residual; the
// thread's sums of r'^2, phi' and (F - m)^2 are added to r2, ps, f2 (the caller
// reduces them).  smf: 3 * TL::PLANE floats of shared memory.  Ends with a barrier.
template <class TL>
__device__ __forceinline__ void df_segment(Dims d, const float2* __restrict__ phi_in, const float* __restrict__ e,
                                           const float2* __restrict__ F, const DF2 m, float2* __restrict__ phi_out,
                                           float* __restrict__ r_out, int x0, int y0, int z0, int zend, float* smf,
                                           float& r2, PAcc& ps, float& f2) {
  constexpr int R = TL::R, WXP = TL::WXP, WS = TL::WS, ARR = TL::ARR, PAD = TL::PAD;
  constexpr int PLANE = TL::PLANE;
  const int tid = threadIdx.x;
  const long long pst = (long long)d.nx * d.ny;
  // the thread's column of pairs
  const int px = tid % WXP, pyb = tid / WXP;
  const int p0 = pyb * R * WS + px;
  const int ux = x0 - 2 + 2 * px;
  int goff[R];
  unsigned tmask = 0;
#pragma unroll
  for (int j = 0; j < R; ++j) {
    const int py = pyb * R + j, uy = y0 - 1 + py;
    goff[j] = wrapmod(ux, d.nx) + wrapmod(uy, d.ny) * d.nx;
    if (tid < TL::NCOL && px >= 1 && px <= TL::TX / 2 && py >= 1 && py <= TL::TY && ux < d.nx && uy < d.ny)
      tmask |= 1u << j;
  }
  const float2 Z = bcast(0.f);
  DF2 W[3][R];        // the update at planes t (W[u]), t - 1, t - 2 of the ring
  DF2 nphi[R], fq[R];
  float2 ne[R];
#pragma unroll
  for (int j = 0; j < R; ++j) {
    fq[j] = DF2{Z, Z};
    ne[j] = Z;
#pragma unroll
    for (int u = 0; u < 3; ++u) W[u][j] = DF2{Z, Z};
  }
  const int tb = z0 - 1, te = zend;
  auto load = [&](int t) {
    const long long base = (long long)wrapmod(t, d.nz) * pst;
#pragma unroll
    for (int j = 0; j < R; ++j) {
      nphi[j] = ld_df2(phi_in + base + goff[j]);
      if (e) ne[j] = __ldg(reinterpret_cast<const float2*>(e + base + goff[j]));
    }
  };
  load(tb);
  int t = tb;
  while (t <= te) {
#pragma unroll
    for (int u = 0; u < 3; ++u, ++t) {
      if (t > te) break;
      float* const cur = smf + u * PLANE + PAD;            // plane t
      const float* const ctr = smf + ((u + 2) % 3) * PLANE + PAD;  // plane t - 1
      DF2 fcur[R];
#pragma unroll
      for (int j = 0; j < R; ++j) {
        W[u][j] = e ? p_df_add_f(nphi[j], ne[j]) : nphi[j];
        fcur[j] = fq[j];
      }
      const long long base = (long long)wrapmod(t, d.nz) * pst;
      if (t < te) {
        load(t + 1);
        // F of the plane whose residual the next iteration forms (plane t)
        if (t >= z0 && t < zend) {
#pragma unroll
          for (int j = 0; j < R; ++j) fq[j] = (tmask >> j & 1u) ? ld_df2(F + base + goff[j]) : DF2{Z, Z};
        }
      }
      const bool in_chunk = t >= z0 && t < zend;
#pragma unroll
      for (int j = 0; j < R; ++j) {
        const int p = p0 + j * WS;
        const DF2 v = W[u][j];
        cur[p] = v.hi.x;
        cur[p + ARR] = v.lo.x;
        cur[p + 2 * ARR] = v.hi.y;
        cur[p + 3 * ARR] = v.lo.y;
        if ((tmask >> j & 1u) && in_chunk) {
          if (phi_out) st_df2(phi_out + base + goff[j], v);
          ps.add(v.hi);
          ps.c = p_add(ps.c, v.lo);
        }
      }
      const int zp = t - 1;
      if (zp >= z0 && zp < zend) {
        const long long pbase = (long long)zp * pst;
        auto at = [&](int q) { return DF2{make_float2(ctr[q], ctr[q + 2 * ARR]), make_float2(ctr[q + ARR], ctr[q + 3 * ARR])}; };
#pragma unroll
        for (int j = 0; j < R; ++j) {
          if (!(tmask >> j & 1u)) continue;
          const int p = p0 + j * WS;
          const DF2 c = W[(u + 2) % 3][j];
          const DF2 ym = j > 0 ? W[(u + 2) % 3][j - 1] : at(p - WS);
          const DF2 yp = j < R - 1 ? W[(u + 2) % 3][j + 1] : at(p + WS);
          const float2 rv = p_df_resid(c, ctr[p - 1 + 2 * ARR], ctr[p - 1 + 3 * ARR], ctr[p + 1], ctr[p + 1 + ARR], ym,
                                       yp, W[(u + 1) % 3][j], W[u][j], fcur[j], m);
          *reinterpret_cast<float2*>(r_out + pbase + goff[j]) = rv;
          r2 = __fmaf_rn(rv.x, rv.x, r2);
          r2 = __fmaf_rn(rv.y, rv.y, r2);
          const float2 fv = p_add(p_sub(fcur[j].hi, m.hi), p_sub(fcur[j].lo, m.lo));
          f2 = __fmaf_rn(fv.x, fv.x, f2);
          f2 = __fmaf_rn(fv.y, fv.y, f2);
        }
      }
      __syncthreads();
    }
  }
}

}  // namespace dfk
}  // namespace gbmg
