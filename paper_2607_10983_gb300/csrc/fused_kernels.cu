// Fused double-float kernel of the finest level: phi' = phi + e in double-float and
// the next defect-correction residual r' = F - m - A phi' (Sec. 3.2) in one pass.
//
// A CTA owns an output tile of TX x TY cells in (x, y) and a chunk of z planes; it
// updates phi on the tile plus a one-cell halo and forms the residual one plane
// behind.  Work unit: the pair of x-neighbouring cells, with the error-free
// double-float sums done by packed FP32x2 instructions lane by lane (bit-identical to
// the scalar double-float kernels).  A thread owns a column of R pairs; shared memory
// holds the updated planes split by x parity and hi/lo part, in a ring of three; the
// z window stays in registers.  One barrier per plane.
#include <cstdio>

#include "dfk.cuh"

namespace gbmg {

namespace {

using namespace dfk;

// ------------------------------------------------------------------ finest level, double-float

// phi' = phi + e (double-float) on the tile plus a one-cell halo, then
// r' = F - m - A phi' on the tile, one plane behind; block partial sums of r'^2,
// of phi' and (pf2 non-null) of (F - m)^2.  e NULL: phi' = phi (first residual of a
// solve); phi_out NULL: phi' is not stored.
template <class TL>
__global__ void __launch_bounds__(TL::NT, 2)
k_df_update_residual(Dims d, const float2* __restrict__ phi_in, const float* __restrict__ e,
                     const float2* __restrict__ F, const double* __restrict__ m_dev, float2* __restrict__ phi_out,
                     float* __restrict__ r_out, double* __restrict__ pr2, double* __restrict__ psum,
                     double* __restrict__ pf2, int zc) {
  extern __shared__ float smf[];
  __shared__ double shr[32];
  const int x0 = blockIdx.x * TL::TX, y0 = blockIdx.y * TL::TY, z0 = blockIdx.z * zc;
  const int zend = min(z0 + zc, d.nz);
  const float2 m1 = f64_to_df(m_dev[0]);
  const DF2 m{bcast(m1.x), bcast(m1.y)};
  float r2 = 0.f, f2 = 0.f;
  PAcc ps{bcast(0.f), bcast(0.f)};
  df_segment<TL>(d, phi_in, e, F, m, phi_out, r_out, x0, y0, z0, zend, smf, r2, ps, f2);
  DfAcc acc{ps.s.x, ps.c.x};
  acc.add(ps.s.y);
  acc.c += ps.c.y;
  const double b2 = block_sum_f(r2, shr);
  const double bs = block_sum_acc(acc, shr);
  const double bf = pf2 ? block_sum_f(f2, shr) : 0.0;
  if (threadIdx.x == 0) {
    const int bid = block_linear_id();
    pr2[bid] = b2;
    psum[bid] = bs;
    if (pf2) pf2[bid] = bf;
  }
}

using DFT = DTile<64, 16, 2, 320>;


}  // namespace

// ---- double-float update

// z chunk of the double-float update: at least four waves of two CTAs per SM, so that
// enough loads are in flight; the warm-up costs one plane per chunk.
int df_zchunk(Dims d) {
  const long long tiles = (long long)((d.nx + DFT::TX - 1) / DFT::TX) * ((d.ny + DFT::TY - 1) / DFT::TY);
  int zc = d.nz;
  while (zc > 16 && tiles * ((d.nz + zc - 1) / zc) < 4 * 2 * 152) zc = (zc + 1) / 2;
  return zc;
}

long long df_update_residual_partials(Dims d) {
  const int zc = df_zchunk(d);
  return (long long)((d.nx + DFT::TX - 1) / DFT::TX) * ((d.ny + DFT::TY - 1) / DFT::TY) * ((d.nz + zc - 1) / zc);
}

cudaError_t launch_df_update_residual(cudaStream_t st, Dims d, const float2* phi_in, const float* e, const float2* F,
                                      const double* m_dev, float2* phi_out, float* r_out, double* pr2, double* psum,
                                      double* pf2) {
  if (d.nx % 2) return cudaErrorInvalidValue;  // x-pairs
  static bool attr = false;
  const size_t sm = 3 * (size_t)DFT::PLANE * sizeof(float);
  if (!attr) {
    cudaError_t err = cudaFuncSetAttribute(k_df_update_residual<DFT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (err != cudaSuccess) return err;
    attr = true;
  }
  const int zc = df_zchunk(d);
  const dim3 grid((d.nx + DFT::TX - 1) / DFT::TX, (d.ny + DFT::TY - 1) / DFT::TY, (d.nz + zc - 1) / zc);
  k_df_update_residual<DFT><<<grid, DFT::NT, sm, st>>>(d, phi_in, e, F, m_dev, phi_out, r_out, pr2, psum, pf2, zc);
  note_launch();
  return cudaGetLastError();
}

}  // namespace gbmg
