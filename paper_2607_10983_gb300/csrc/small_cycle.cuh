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


// Cells i = tid, tid + nt, ... of a level with their (x, y, z), advanced by mixed-radix
// addition of nt instead of a division per cell.
struct Walk {
  int i, x, y, z;
  int sx, sy, sz;
  __device__ __forceinline__ Walk(Dims d, int tid, int nt) : i(tid) {
    x = tid % d.nx;
    const int q = tid / d.nx;
    y = q % d.ny;
    z = q / d.ny;
    sx = nt % d.nx;
    const int q2 = nt / d.nx;
    sy = q2 % d.ny;
    sz = q2 / d.ny;
  }
  __device__ __forceinline__ void next(Dims d, int nt) {
    i += nt;
    x += sx;
    int c = 0;
    if (x >= d.nx) {
      x -= d.nx;
      c = 1;
    }
    y += sy + c;
    c = 0;
    if (y >= d.ny) {
      y -= d.ny;
      c = 1;
    }
    z += sz + c;
  }
};

// The whole sub-cycle by the calling CTA (any block size, a multiple of 32), NL levels;
// sm: small_cycle_smem(P) bytes of shared memory.  Ends with the result stored (no
// barrier after the last store).
template <int NL>
__device__ __forceinline__ void block_vcycle_n(const SmallCycle& P, const float* __restrict__ r_in,
                                               float* __restrict__ e_out, float* sm) {
  const int tid = threadIdx.x, nt = blockDim.x;
  // per level: r, e, e2, d, t (the coarsest: r, e), as offsets into sm
  int oR[NL], oE[NL], oE2[NL], oDV[NL], oT[NL];
  {
    int p = 0;
#pragma unroll
    for (int l = 0; l < NL; ++l) {
      const int n = ncell(P.d[l]);
      oR[l] = p;
      oE[l] = p + n;
      p += 2 * n;
      oE2[l] = oDV[l] = oT[l] = 0;
      if (l < NL - 1) {
        oE2[l] = p;
        oDV[l] = p + n;
        oT[l] = p + 2 * n;
        p += 3 * n;
      }
    }
  }
  const int n0 = ncell(P.d[0]);
  for (int i = tid; i < n0; i += nt) {
    sm[oR[0] + i] = r_in[i];
    sm[oE[0] + i] = 0.f;
  }
  __syncthreads();
  auto smooth = [&](int l) {
    const Dims d = P.d[l];
    const int n = ncell(d);
    for (int k = 0; k < P.degree; ++k) {
      const float a = P.a[l][k], b = P.b[l][k], c1 = P.c1[k];
      const float* E = sm + oE[l];
      float* E2 = sm + oE2[l];
      float* DV = sm + oDV[l];
      const float* R = sm + oR[l];
      for (Walk w(d, tid, nt); w.i < n; w.next(d, nt)) {
        const int i = w.i;
        const float c = E[i];
        float dv = c1 == 0.f ? 0.f : DV[i];
        E2[i] = cheb_step(c, R[i], nsum6(nbrs(E, d, w.x, w.y, w.z, i)), c, dv, a, b, c1);
        DV[i] = dv;
      }
      __syncthreads();
      const int t = oE[l];
      oE[l] = oE2[l];
      oE2[l] = t;
    }
  };
  // down: pre-smoothing, residual, restriction
#pragma unroll
  for (int l = 0; l + 1 < NL; ++l) {
    smooth(l);
    const Dims d = P.d[l];
    const int n = ncell(d);
    {
      const float* E = sm + oE[l];
      const float* R = sm + oR[l];
      float* T = sm + oT[l];
      const float ih2 = P.inv_h2[l];
      for (Walk w(d, tid, nt); w.i < n; w.next(d, nt))
        T[w.i] = resid_from_sum(R[w.i], nsum6(nbrs(E, d, w.x, w.y, w.z, w.i)), E[w.i], ih2);
    }
    __syncthreads();
    const Dims dc = P.d[l + 1];
    const int nc = ncell(dc);
    {
      const float* T = sm + oT[l];
      float* Rc = sm + oR[l + 1];
      float* Ec = sm + oE[l + 1];
      for (Walk w(dc, tid, nt); w.i < nc; w.next(dc, nt)) {
        int xs[3], ys[3], zs[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          xs[k] = wrapi(2 * w.x + k - 1, d.nx);
          ys[k] = wrapi(2 * w.y + k - 1, d.ny);
          zs[k] = wrapi(2 * w.z + k - 1, d.nz);
        }
        float yv[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          float zv[3];
#pragma unroll
          for (int b = 0; b < 3; ++b)
            zv[b] = fw3(T[(int)lin(d, xs[a], ys[b], zs[0])], T[(int)lin(d, xs[a], ys[b], zs[1])],
                        T[(int)lin(d, xs[a], ys[b], zs[2])]);
          yv[a] = fw3(zv[0], zv[1], zv[2]);
        }
        Rc[w.i] = fw3(yv[0], yv[1], yv[2]);
        if (l + 2 < NL) Ec[w.i] = 0.f;
      }
    }
    __syncthreads();
  }
  // coarsest: e = G r, one warp per row, lanes stride the columns
  {
    const float* R = sm + oR[NL - 1];
    float* E = sm + oE[NL - 1];
    const int lane = tid & 31;
    for (int row = tid >> 5; row < P.nc; row += nt >> 5) {
      float acc = 0.f;
      for (int j = lane; j < P.nc; j += 32) acc = t_fma(P.G[(long long)row * P.nc + j], R[j], acc);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc = t_add(acc, __shfl_xor_sync(0xffffffffu, acc, o));
      if (lane == 0) E[row] = acc;
    }
    __syncthreads();
  }
  // up: prolongation + correction, post-smoothing
#pragma unroll
  for (int l = NL - 2; l >= 0; --l) {
    const Dims d = P.d[l], dc = P.d[l + 1];
    const int n = ncell(d);
    {
      float* E = sm + oE[l];
      const float* Ec = sm + oE[l + 1];
      for (Walk w(d, tid, nt); w.i < n; w.next(d, nt)) E[w.i] = t_add(E[w.i], prolong_value(Ec, dc, w.x, w.y, w.z));
    }
    __syncthreads();
    smooth(l);
  }
  for (int i = tid; i < n0; i += nt) e_out[i] = sm[oE[0] + i];
}

__device__ __forceinline__ void block_vcycle(const SmallCycle& P, const float* __restrict__ r_in,
                                             float* __restrict__ e_out, float* sm) {
  switch (P.nl) {
    case 2: block_vcycle_n<2>(P, r_in, e_out, sm); break;
    case 3: block_vcycle_n<3>(P, r_in, e_out, sm); break;
    default: block_vcycle_n<4>(P, r_in, e_out, sm); break;
  }
}

}  // namespace smallc
}  // namespace gbmg
