// Packed FP32x2 arithmetic on the pair (even x, odd x) of neighbouring cells
// (f32x2 instructions of the sm_100 family).  Each lane rounds exactly like the
// scalar intrinsic of the same operation, so kernels written with these helpers
// reproduce the one-kernel-per-operation arithmetic bit for bit when they apply the
// operations in the same order.
#pragma once
#include "stencil.cuh"

namespace gbmg {

#define GBMG_PACKED_OP(name, op)                                                         \
  __device__ __forceinline__ float2 name(float2 a, float2 b) {                           \
    float2 d;                                                                            \
    asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t" op \
        " rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"                                     \
        : "=f"(d.x), "=f"(d.y)                                                           \
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));                                      \
    return d;                                                                            \
  }
GBMG_PACKED_OP(p_add, "add.rn.f32x2")
GBMG_PACKED_OP(p_sub, "sub.rn.f32x2")
GBMG_PACKED_OP(p_mul, "mul.rn.f32x2")
#undef GBMG_PACKED_OP

__device__ __forceinline__ float2 p_fma(float2 a, float2 b, float2 c) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "mov.b64 rc, {%6, %7};\n\tfma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}
__device__ __forceinline__ float2 bcast(float v) { return make_float2(v, v); }

// nbr_sum of the pair: the x neighbours of the even cell are (xm, c.y), those of
// the odd cell (c.x, xp); then y, then z, in the order of the scalar nbr_sum.
__device__ __forceinline__ float2 p_nbr_sum(float xm, float xp, float2 c, float2 ym, float2 yp, float2 zm,
                                            float2 zp) {
  float2 s = make_float2(t_add(xm, c.y), t_add(c.x, xp));
  s = p_add(s, p_add(ym, yp));
  return p_add(s, p_add(zm, zp));
}
// cheb_step on a pair (folded constants a, -b, c1 broadcast)
__device__ __forceinline__ float2 p_cheb(float2 e, float2 r, float2 s, float2 c, float2& d, float2 a, float2 mb,
                                         float2 c1) {
  const float2 q = p_fma(mb, p_fma(bcast(-6.f), c, s), p_mul(a, r));
  d = p_fma(c1, d, q);
  return p_add(e, d);
}
// resid_from_sum on a pair (mih2 = -1/h^2 broadcast)
__device__ __forceinline__ float2 p_resid(float2 r, float2 s, float2 c, float2 mih2) {
  return p_fma(mih2, p_fma(bcast(-6.f), c, s), r);
}
__device__ __forceinline__ float2 p_fw3(float2 a, float2 b, float2 c) {
  return p_fma(bcast(0.25f), p_add(a, c), p_mul(bcast(0.5f), b));
}
__device__ __forceinline__ float2 p_half_sum(float2 a, float2 b) { return p_mul(bcast(0.5f), p_add(a, b)); }

// ---- double-float pairs: hi parts of both cells, lo parts of both cells

struct DF2 {
  float2 hi, lo;
};

// two_sum of common.cuh, lane by lane
__device__ __forceinline__ void p_two_sum(float2 a, float2 b, float2& s, float2& e) {
  s = p_add(a, b);
  const float2 bb = p_sub(s, a);
  e = p_add(p_sub(a, p_sub(s, bb)), p_sub(b, bb));
}
// df_add_f of common.cuh: (hi, lo) + f, renormalised
__device__ __forceinline__ DF2 p_df_add_f(DF2 a, float2 b) {
  float2 s, e;
  p_two_sum(a.hi, b, s, e);
  e = p_add(e, a.lo);
  const float2 h = p_add(s, e);
  return DF2{h, p_sub(e, p_sub(h, s))};
}
// DfAcc of common.cuh, lane by lane.  add_neg(t) equals add(-t) bit for bit
// (x + (-y) = x - y and (-t) - bb = -(t + bb) exactly under round-to-nearest)
// without forming -t.
struct PAcc {
  float2 s, c;
  __device__ __forceinline__ void add(float2 t) {
    float2 ns, e;
    p_two_sum(s, t, ns, e);
    s = ns;
    c = p_add(c, e);
  }
  __device__ __forceinline__ void add_neg(float2 t) {
    const float2 ns = p_sub(s, t);
    const float2 bb = p_sub(ns, s);
    const float2 e = p_sub(p_sub(s, p_sub(ns, bb)), p_add(t, bb));
    s = ns;
    c = p_add(c, e);
  }
};
// df_resid of stencil.cuh on a pair: r = (F - m) - (sum of neighbours - 6 c), the hi
// parts summed error-free, the lo parts in plain FP32; x neighbours as in p_nbr_sum.
__device__ __forceinline__ float2 p_df_resid(DF2 c, float xm_hi, float xm_lo, float xp_hi, float xp_lo, DF2 ym,
                                             DF2 yp, DF2 zm, DF2 zp, DF2 f, DF2 m) {
  const float2 xmh = make_float2(xm_hi, c.hi.x), xph = make_float2(c.hi.y, xp_hi);
  const float2 xml = make_float2(xm_lo, c.lo.x), xpl = make_float2(c.lo.y, xp_lo);
  const float2 six = bcast(6.f);
  PAcc acc;
  acc.s = p_mul(six, c.hi);
  acc.c = p_fma(six, c.hi, make_float2(-acc.s.x, -acc.s.y));  // exact error of 6 hi
  acc.add_neg(xmh);
  acc.add_neg(xph);
  acc.add_neg(ym.hi);
  acc.add_neg(yp.hi);
  acc.add_neg(zm.hi);
  acc.add_neg(zp.hi);
  acc.add(f.hi);
  acc.add_neg(m.hi);
  float2 lo = p_add(p_add(xml, xpl), p_add(ym.lo, yp.lo));
  lo = p_add(lo, p_add(zm.lo, zp.lo));
  lo = p_sub(p_fma(six, c.lo, p_sub(f.lo, m.lo)), lo);
  return p_add(acc.s, p_add(acc.c, lo));
}

// Smallest row stride (in pairs) >= wxp for which a warp whose 32 consecutive
// threads straddle two row blocks still reads 32 distinct banks: the jump between
// the blocks, r * ws - (wxp - 1), must equal 1 modulo 32.  wxp itself if none exists.
constexpr int conflict_free_stride(int wxp, int r) {
  for (int ws = wxp; ws < wxp + 32; ++ws)
    if ((r * ws - wxp) % 32 == 0) return ws;
  return wxp;
}

}  // namespace gbmg
