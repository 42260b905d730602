// Per-cell arithmetic of the flat multigrid operations, shared by the one-kernel-
// per-operation path and the temporally blocked (fused) kernels so that both round
// identically.  Every operation is an explicitly rounded intrinsic (no FMA
// contraction decided by the compiler).
#pragma once
#include "common.cuh"

namespace gbmg {

__device__ __forceinline__ float t_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double t_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float t_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double t_sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float t_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double t_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float t_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double t_fma(double a, double b, double c) { return __fma_rn(a, b, c); }

// Sum of the six face neighbours, in the fixed order (x-, x+), (y-, y+), (z-, z+).
template <typename T>
__device__ __forceinline__ T nbr_sum(T xm, T xp, T ym, T yp, T zm, T zp) {
  T s = t_add(xm, xp);
  s = t_add(s, t_add(ym, yp));
  s = t_add(s, t_add(zm, zp));
  return s;
}

// (A_l u)_i = (sum of neighbours - 6 u_i) / h_l^2   (Sec. 2.1, Eq. linsys)
template <typename T>
__device__ __forceinline__ T lap_from_sum(T s, T c, T inv_h2) {
  return t_mul(t_fma(T(-6), c, s), inv_h2);
}

// r - A_l u = r - (s - 6c) / h^2
template <typename T>
__device__ __forceinline__ T resid_from_sum(T r, T s, T c, T inv_h2) {
  return t_fma(-inv_h2, t_fma(T(-6), c, s), r);
}

// One Chebyshev step (Sec. 2.3, Eq. flat_chebyshev, semi-iteration form)
//   z = D^-1 (r - A e);  d = c1 d + c2 z;  e += d,
// evaluated with the constants folded: a = c2 D^-1, b = a / h^2 (each rounded once
// on the host), q = a r - b (s - 6c), d = c1 d + q.  The first step of a pass has
// c1 = 0 (d = z / theta).  Returns the new e, updates d.
template <typename T>
__device__ __forceinline__ T cheb_step(T e, T r, T s, T c, T& d, T a, T b, T c1) {
  const T q = t_fma(-b, t_fma(T(-6), c, s), t_mul(a, r));
  d = t_fma(c1, d, q);
  return t_add(e, d);
}

// Weighted Jacobi (Sec. 2.3, Eq. flat_jacobi): e + omega D^-1 (r - A e), with
// wa = omega D^-1 and wb = wa / h^2: e + wa r - wb (s - 6c).
template <typename T>
__device__ __forceinline__ T jacobi_step(T e, T r, T s, T c, T wa, T wb) {
  return t_fma(-wb, t_fma(T(-6), c, s), t_fma(wa, r, e));
}

// One axis of full weighting: (a + c)/4 + b/2 (Appendix B).
template <typename T>
__device__ __forceinline__ T fw3(T a, T b, T c) {
  return t_fma(T(0.25), t_add(a, c), t_mul(T(0.5), b));
}

// One axis of trilinear interpolation between neighbouring coarse nodes.
template <typename T>
__device__ __forceinline__ T half_sum(T a, T b) {
  return t_mul(T(0.5), t_add(a, b));
}

// Trilinear prolongation: fine node 2I + d gets the mean over the coarse nodes
// I + d', d' <= d, evaluated as nested midpoints along x, then y, then z.
template <typename T>
__device__ __forceinline__ T prolong_value(const T* __restrict__ c, Dims dc, int x, int y, int z) {
  const int I = x >> 1, J = y >> 1, K = z >> 1;
  const int dx = x & 1, dy = y & 1, dz = z & 1;
  const int I1 = wrap_hi(I + 1, dc.nx), J1 = wrap_hi(J + 1, dc.ny), K1 = wrap_hi(K + 1, dc.nz);
  auto cx = [&](int jj, int kk) -> T {
    const T v0 = c[lin(dc, I, jj, kk)];
    return dx ? half_sum(v0, c[lin(dc, I1, jj, kk)]) : v0;
  };
  auto cy = [&](int kk) -> T {
    const T v0 = cx(J, kk);
    return dy ? half_sum(v0, cx(J1, kk)) : v0;
  };
  const T v0 = cy(K);
  return dz ? half_sum(v0, cy(K1)) : v0;
}

// Residual of the defect correction on the finest level (h = 1) in double-float:
//   r = (F - m) - (sum of neighbours of phi - 6 phi),
// summed with error-free transformations on the high parts (which cancel by a
// factor ~ (N/2pi)^2 for smooth potentials) and plain FP32 on the low parts.
// Returns r rounded to float.
__device__ __forceinline__ float df_resid(float2 c, float2 xm, float2 xp, float2 ym, float2 yp,
                                          float2 zm, float2 zp, float2 f, float2 m) {
  DfAcc acc;
  acc.s = __fmul_rn(6.0f, c.x);
  acc.c = __fmaf_rn(6.0f, c.x, -acc.s);   // exact error of 6*hi
  acc.add(-xm.x);
  acc.add(-xp.x);
  acc.add(-ym.x);
  acc.add(-yp.x);
  acc.add(-zm.x);
  acc.add(-zp.x);
  acc.add(f.x);
  acc.add(-m.x);
  float lo = __fadd_rn(__fadd_rn(xm.y, xp.y), __fadd_rn(ym.y, yp.y));
  lo = __fadd_rn(lo, __fadd_rn(zm.y, zp.y));
  lo = __fsub_rn(__fmaf_rn(6.0f, c.y, __fsub_rn(f.y, m.y)), lo);
  return __fadd_rn(acc.s, __fadd_rn(acc.c, lo));
}

}  // namespace gbmg
