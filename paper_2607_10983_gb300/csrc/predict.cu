// Warm-start predictors (Sec. 3.2 "Predictors"): recycling, the growth-scaled
// previous solution (Eq. growth) and linear / quadratic extrapolation over the
// previous solutions, one FP64 pass.  Explicitly rounded operations, left to right,
// so the result does not depend on FMA contraction.
#include "kernels.h"
#include "solver.h"

namespace gbmg {

namespace {

template <int ORDER>
__global__ void k_predict(long long n, double growth, const double* __restrict__ h0, const double* __restrict__ h1,
                          const double* __restrict__ h2, double* out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double v;
    if (ORDER == 0) v = __dmul_rn(growth, h0[i]);
    else if (ORDER == 1) v = __dsub_rn(__dmul_rn(2.0, h0[i]), h1[i]);
    else v = __dadd_rn(__dsub_rn(__dmul_rn(3.0, h0[i]), __dmul_rn(3.0, h1[i])), h2[i]);
    out[i] = v;
  }
}

}  // namespace

}  // namespace gbmg

using namespace gbmg;

extern "C" gbmg_status mg_predict(gbmg_ctx* c, int order, double growth, const double* const* hist, int nh,
                                  double* out) {
  if (!c || !hist || !out || order < 0 || order > 2 || nh < order + 1)
    return fail(GBMG_ERR_INVALID_ARG, "mg_predict: bad argument");
  for (int k = 0; k <= order; ++k)
    if (!hist[k]) return fail(GBMG_ERR_INVALID_ARG, "mg_predict: NULL history field");
  DeviceGuard g(c->device);
  const long long n = ncell(c->lv[0].d);
  const int blocks = (int)df_partial_count(n);
  if (order == 0) k_predict<0><<<blocks, 256, 0, c->stream>>>(n, growth, hist[0], nullptr, nullptr, out);
  else if (order == 1) k_predict<1><<<blocks, 256, 0, c->stream>>>(n, growth, hist[0], hist[1], nullptr, out);
  else k_predict<2><<<blocks, 256, 0, c->stream>>>(n, growth, hist[0], hist[1], hist[2], out);
  note_launch();
  TRY(cudaGetLastError());
  return GBMG_OK;
}
