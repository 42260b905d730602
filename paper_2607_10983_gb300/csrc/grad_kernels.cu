// Finite-difference gradients on the periodic finest level (spacing 1) and their
// transposes, for losses of the form sum(w . grad phi):
//   order 4: (-u_{i+2} + 8 u_{i+1} - 8 u_{i-1} + u_{i-2}) / 12, the one-exchange
//            fourth-order gradient of the force evaluation (Sec. 3.4);
//   order 2: (u_{i+1} - u_{i-1}) / 2, the central difference of Sec. 4.1.
// Both stencils are antisymmetric on the periodic mesh, so the transpose is the
// negated divergence with the same stencil.  FP64 in and out (w in FP32), once per
// loss evaluation, outside the V-cycle.
#include "kernels.h"
#include "solver.h"

namespace gbmg {

namespace {

constexpr int BX = 32, BY = 8;
inline dim3 cell_grid(Dims d) { return dim3((d.nx + BX - 1) / BX, (d.ny + BY - 1) / BY, d.nz); }

// |s| <= 2 <= n: one conditional wrap instead of a modulo
__device__ __forceinline__ int wrap2(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }
__device__ __forceinline__ long long shifted(Dims d, int x, int y, int z, int axis, int s) {
  if (axis == 0) x = wrap2(x + s, d.nx);
  else if (axis == 1) y = wrap2(y + s, d.ny);
  else z = wrap2(z + s, d.nz);
  return lin(d, x, y, z);
}

template <typename V>
__device__ __forceinline__ double dstencil(const V* u, Dims d, int x, int y, int z, int axis, int order, int sign) {
  auto U = [&](int s) { return (double)u[shifted(d, x, y, z, axis, sign * s)]; };
  if (order == 4) return (-U(2) + 8.0 * U(1) - 8.0 * U(-1) + U(-2)) / 12.0;
  return (U(1) - U(-1)) * 0.5;
}

__global__ void k_grad(Dims d, int order, const double* __restrict__ u, double* __restrict__ out) {
  const int x = blockIdx.x * BX + threadIdx.x, y = blockIdx.y * BY + threadIdx.y, z = blockIdx.z;
  if (x >= d.nx || y >= d.ny) return;
  const long long n = ncell(d), i = lin(d, x, y, z);
  for (int a = 0; a < 3; ++a) out[a * n + i] = dstencil(u, d, x, y, z, a, order, 1);
}

// grad^T w = -div w with the same antisymmetric stencil
__global__ void k_grad_T(Dims d, int order, const float* __restrict__ w, double* __restrict__ out) {
  const int x = blockIdx.x * BX + threadIdx.x, y = blockIdx.y * BY + threadIdx.y, z = blockIdx.z;
  if (x >= d.nx || y >= d.ny) return;
  const long long n = ncell(d), i = lin(d, x, y, z);
  double v = 0.0;
  for (int a = 0; a < 3; ++a) v += dstencil(w + a * n, d, x, y, z, a, order, -1);
  out[i] = v;
}

// block partials of sum(w . grad u)
__global__ void k_grad_dot(Dims d, int order, const double* __restrict__ u, const float* __restrict__ w,
                           double* __restrict__ partials) {
  __shared__ double sh[32];
  const int x = blockIdx.x * BX + threadIdx.x, y = blockIdx.y * BY + threadIdx.y, z = blockIdx.z;
  double v = 0.0;
  if (x < d.nx && y < d.ny) {
    const long long n = ncell(d), i = lin(d, x, y, z);
    for (int a = 0; a < 3; ++a) v += (double)w[a * n + i] * dstencil(u, d, x, y, z, a, order, 1);
  }
  v = block_sum(v, sh);
  if (is_thread0()) partials[block_linear_id()] = v;
}

}  // namespace

}  // namespace gbmg

using namespace gbmg;

extern "C" gbmg_status mg_grad(gbmg_ctx* c, int order, int transpose, const void* in_dev, double* out_dev) {
  if (!c || !in_dev || !out_dev || (order != 2 && order != 4)) return fail(GBMG_ERR_INVALID_ARG, "mg_grad: bad argument");
  DeviceGuard g(c->device);
  const Dims d = c->lv[0].d;
  if (transpose) k_grad_T<<<cell_grid(d), dim3(BX, BY), 0, c->stream>>>(d, order, (const float*)in_dev, out_dev);
  else k_grad<<<cell_grid(d), dim3(BX, BY), 0, c->stream>>>(d, order, (const double*)in_dev, out_dev);
  note_launch();
  TRY(cudaGetLastError());
  return GBMG_OK;
}

extern "C" gbmg_status mg_grad_dot(gbmg_ctx* c, int order, const double* u_dev, const float* w_dev, double* out_dev) {
  if (!c || !u_dev || !w_dev || !out_dev || (order != 2 && order != 4))
    return fail(GBMG_ERR_INVALID_ARG, "mg_grad_dot: bad argument");
  DeviceGuard g(c->device);
  const Dims d = c->lv[0].d;
  k_grad_dot<<<cell_grid(d), dim3(BX, BY), 0, c->stream>>>(d, order, u_dev, w_dev, c->partials);
  note_launch();
  TRY(cudaGetLastError());
  TRY(launch_finalize(c->stream, c->partials, partial_count(d), out_dev, 1.0));
  return GBMG_OK;
}
