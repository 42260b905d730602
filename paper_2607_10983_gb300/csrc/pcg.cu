// Vector kernels of the V-cycle-preconditioned conjugate-gradient correction (Sec. 3.2:
// multigrid as the preconditioner of a conjugate-gradient iteration).  FP32 vectors,
// FP64 dot products and scalars kept on the device.
#include "kernels.h"

namespace gbmg {

namespace {

constexpr int PT = 256;

__global__ void k_dot_f32(long long n, const float* __restrict__ a, const float* __restrict__ b,
                          double* __restrict__ partials) {
  __shared__ double sh[32];
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    s += (double)a[i] * (double)b[i];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// e = (first ? 0 : e) + alpha p;  r -= alpha q;  alpha = num / den (device scalars)
__global__ void k_pcg_update(long long n, float* __restrict__ e, float* __restrict__ r, const float* __restrict__ p,
                             const float* __restrict__ q, const double* __restrict__ num,
                             const double* __restrict__ den, int first) {
  const float alpha = den[0] != 0.0 ? (float)(num[0] / den[0]) : 0.f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float pi = p[i];
    e[i] = first ? alpha * pi : fmaf(alpha, pi, e[i]);
    r[i] = fmaf(-alpha, q[i], r[i]);
  }
}

// p = z + beta p, beta = num / den
__global__ void k_pcg_dir(long long n, float* __restrict__ p, const float* __restrict__ z,
                          const double* __restrict__ num, const double* __restrict__ den) {
  const float beta = den[0] != 0.0 ? (float)(num[0] / den[0]) : 0.f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    p[i] = fmaf(beta, p[i], z[i]);
}

}  // namespace

cudaError_t launch_dot_f32(cudaStream_t st, long long n, const float* a, const float* b, double* partials) {
  k_dot_f32<<<(int)df_partial_count(n), PT, 0, st>>>(n, a, b, partials);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_pcg_update(cudaStream_t st, long long n, float* e, float* r, const float* p, const float* q,
                              const double* num, const double* den, int first) {
  k_pcg_update<<<(int)df_partial_count(n), PT, 0, st>>>(n, e, r, p, q, num, den, first);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_pcg_dir(cudaStream_t st, long long n, float* p, const float* z, const double* num,
                           const double* den) {
  k_pcg_dir<<<(int)df_partial_count(n), PT, 0, st>>>(n, p, z, num, den);
  note_launch();
  return cudaGetLastError();
}

}  // namespace gbmg
