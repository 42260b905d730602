// Single-CTA kernel of the bottom of the FP32 V-cycle (the levels that fit in shared
// memory): a level visit of the one-kernel-per-operation chain costs a launch per
// operation while each operation is a few thousand cells; here the same operations run
// as phases of one CTA separated by __syncthreads (device code in small_cycle.cuh).
#include "small_cycle.cuh"

namespace gbmg {

namespace {

__global__ void __launch_bounds__(kSmallThreads, 1) k_small_vcycle(SmallCycle P, const float* __restrict__ r_in,
                                                                   float* __restrict__ e_out) {
  extern __shared__ __align__(16) float sm[];
  smallc::block_vcycle(P, r_in, e_out, sm);
}

}  // namespace

size_t small_cycle_smem(const SmallCycle& P) {
  size_t f = 0;
  for (int l = 0; l < P.nl; ++l) f += (size_t)ncell(P.d[l]) * (l < P.nl - 1 ? 5 : 2);
  return f * sizeof(float);
}

cudaError_t launch_small_vcycle(cudaStream_t st, const SmallCycle& P, const float* r_in, float* e_out) {
  if (P.nl < 2 || P.nl > kSmallMaxL || ncell(P.d[0]) > kSmallCells || P.degree < 1 || P.degree > 16 ||
      P.nc != ncell(P.d[P.nl - 1]))
    return cudaErrorInvalidValue;
  const size_t sm = small_cycle_smem(P);
  if (sm > kSmallSmem) return cudaErrorInvalidValue;
  static bool attr = false;
  if (!attr) {
    cudaError_t err = cudaFuncSetAttribute(k_small_vcycle, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmallSmem);
    if (err != cudaSuccess) return err;
    attr = true;
  }
  k_small_vcycle<<<1, kSmallThreads, sm, st>>>(P, r_in, e_out);
  note_launch();
  return cudaGetLastError();
}

}  // namespace gbmg
