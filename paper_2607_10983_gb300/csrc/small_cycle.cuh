// The bottom of the FP32 Chebyshev V-cycle (Sec. 2.3) by one CTA: the levels whose
// fields fit in shared memory (at most kSmallCells cells on the first of them, e.g.
// 16^3, 8^3, 4^3).  Every cell value is computed by the per-cell functions of the
// one-kernel-per-operation kernels in the same order, and the coarsest solve keeps
// their warp-per-row summation order, so the result is bit-identical to that chain.
// Used by the single-CTA kernel of small_cycle.cu and by the batched persistent kernel.
#pragma once
#include "kernels.h"
#include "stencil.cuh"

namespace gbmg {
namespace smallc {

template <typename V>
struct Nbrs6 {
  V xm, xp, ym, yp, zm, zp;
};

__device__ __forceinline__ Nbrs6<float> nbrs(const float* u, Dims d, int x, int y, int z, int i) {
  const int sy = d.nx, sz = d.nx * d.ny;
  Nbrs6<float> n;
  n.xm = u[i + ((x == 0 ? d.nx - 1 : x - 1) - x)];
  n.xp = u[i + ((x == d.nx - 1 ? 0 : x + 1) - x)];
  n.ym = u[i + ((y == 0 ? d.ny - 1 : y - 1) - y) * sy];
  n.yp = u[i + ((y == d.ny - 1 ? 0 : y + 1) - y) * sy];
  n.zm = u[i + ((z == 0 ? d.nz - 1 : z - 1) - z) * sz];
  n.zp = u[i + ((z == d.nz - 1 ? 0 : z + 1) - z) * sz];
  return n;
}
__device__ __forceinline__ float nsum6(const Nbrs6<float>& n) { return nbr_sum(n.xm, n.xp, n.ym, n.yp, n.zm, n.zp); }

__device__ __forceinline__ void cell_of(Dims d, int i, int& x, int& y, int& z) {
  x = i % d.nx;
  y = (i / d.nx) % d.ny;
  z = i / (d.nx * d.ny);
}

// The whole sub-cycle by the calling CTA (any block size, a multiple of 32); sm:
// small_cycle_smem(P) bytes of shared memory.  Ends with the result stored (no barrier
// after the last store).
__device__ __forceinline__ void block_vcycle(const SmallCycle& P, const float* __restrict__ r_in,
                                             float* __restrict__ e_out, float* sm) {
  const int tid = threadIdx.x, nt = blockDim.x;
  // per level: r, e, e2, d, t (the coarsest: r, e)
  float *R[kSmallMaxL], *E[kSmallMaxL], *E2[kSmallMaxL], *DV[kSmallMaxL], *T[kSmallMaxL];
  {
    float* p = sm;
    for (int l = 0; l < P.nl; ++l) {
      const int n = ncell(P.d[l]);
      R[l] = p;
      E[l] = p + n;
      p += 2 * n;
      if (l < P.nl - 1) {
        E2[l] = p;
        DV[l] = p + n;
        T[l] = p + 2 * n;
        p += 3 * n;
      }
    }
  }
  const int n0 = ncell(P.d[0]);
  for (int i = tid; i < n0; i += nt) {
    R[0][i] = r_in[i];
    E[0][i] = 0.f;
  }
  __syncthreads();
  auto smooth = [&](int l) {
    const Dims d = P.d[l];
    const int n = ncell(d);
    for (int k = 0; k < P.degree; ++k) {
      const float a = P.a[l][k], b = P.b[l][k], c1 = P.c1[k];
      for (int i = tid; i < n; i += nt) {
        int x, y, z;
        cell_of(d, i, x, y, z);
        const float c = E[l][i];
        float dv = c1 == 0.f ? 0.f : DV[l][i];
        E2[l][i] = cheb_step(c, R[l][i], nsum6(nbrs(E[l], d, x, y, z, i)), c, dv, a, b, c1);
        DV[l][i] = dv;
      }
      __syncthreads();
      float* s = E[l];
      E[l] = E2[l];
      E2[l] = s;
    }
  };
  // down: pre-smoothing, residual, restriction
  for (int l = 0; l + 1 < P.nl; ++l) {
    smooth(l);
    const Dims d = P.d[l];
    const int n = ncell(d);
    for (int i = tid; i < n; i += nt) {
      int x, y, z;
      cell_of(d, i, x, y, z);
      T[l][i] = resid_from_sum(R[l][i], nsum6(nbrs(E[l], d, x, y, z, i)), E[l][i], P.inv_h2[l]);
    }
    __syncthreads();
    const Dims dc = P.d[l + 1];
    const int nc = ncell(dc);
    for (int i = tid; i < nc; i += nt) {
      int X, Y, Z;
      cell_of(dc, i, X, Y, Z);
      int xs[3], ys[3], zs[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        xs[k] = wrapi(2 * X + k - 1, d.nx);
        ys[k] = wrapi(2 * Y + k - 1, d.ny);
        zs[k] = wrapi(2 * Z + k - 1, d.nz);
      }
      float yv[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        float zv[3];
#pragma unroll
        for (int b = 0; b < 3; ++b)
          zv[b] = fw3(T[l][(int)lin(d, xs[a], ys[b], zs[0])], T[l][(int)lin(d, xs[a], ys[b], zs[1])],
                      T[l][(int)lin(d, xs[a], ys[b], zs[2])]);
        yv[a] = fw3(zv[0], zv[1], zv[2]);
      }
      R[l + 1][i] = fw3(yv[0], yv[1], yv[2]);
      if (l + 2 < P.nl) E[l + 1][i] = 0.f;
    }
    __syncthreads();
  }
  // coarsest: e = G r, one warp per row, lanes stride the columns
  {
    const int lc = P.nl - 1;
    const int lane = tid & 31;
    for (int row = tid >> 5; row < P.nc; row += nt >> 5) {
      float acc = 0.f;
      for (int j = lane; j < P.nc; j += 32) acc = t_fma(P.G[(long long)row * P.nc + j], R[lc][j], acc);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc = t_add(acc, __shfl_xor_sync(0xffffffffu, acc, o));
      if (lane == 0) E[lc][row] = acc;
    }
    __syncthreads();
  }
  // up: prolongation + correction, post-smoothing
  for (int l = P.nl - 2; l >= 0; --l) {
    const Dims d = P.d[l], dc = P.d[l + 1];
    const int n = ncell(d);
    for (int i = tid; i < n; i += nt) {
      int x, y, z;
      cell_of(d, i, x, y, z);
      E[l][i] = t_add(E[l][i], prolong_value(E[l + 1], dc, x, y, z));
    }
    __syncthreads();
    smooth(l);
  }
  for (int i = tid; i < n0; i += nt) e_out[i] = E[0][i];
}


}  // namespace smallc
}  // namespace gbmg
