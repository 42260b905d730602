// Allocation-free evaluation of the relative residual ||F - m - A phi|| / ||F - m||
// (m = mean(F), A the 7-point periodic Laplacian, h = 1), for callers that must not
// allocate device memory: for example a time-step loop that runs inside a fixed,
// pre-reserved memory budget, or code hosted by another framework whose allocator
// owns the device.  It needs no context and no mg_setup.
//
// Scratch: the per-plane partial sums and the mean live in the file-scope device
// array below.  Every GPU that loads the library holds it (about 64 KiB) until the
// process exits.  Host code may not use the symbol as an address; the address of
// the array on each device is obtained once with cudaGetSymbolAddress, on the first
// call made on that device, with that device current.
#include <atomic>
#include <cmath>
#include <cstring>

#include "gbmg.h"
#include "kernels.h"
#include "solver.h"
#include "stencil.cuh"

namespace {

constexpr int NOALLOC_MAX_NZ = GBMG_NOALLOC_MAX_NZ;
// [0, nz): plane sums of F (then of (F - m)^2), [MAX, MAX + nz): plane sums of r^2, [2 MAX]: mean
constexpr int SCRATCH_DOUBLES = 2 * NOALLOC_MAX_NZ + 8;

static __device__ __align__(256) double g_noalloc_scratch[SCRATCH_DOUBLES];

constexpr int MAX_DEVICES = 64;
// Device address of g_noalloc_scratch per device, looked up on the first call there.
// Atomic: first calls from several host threads may race; each stores the same value.
std::atomic<double*> g_scratch_addr[MAX_DEVICES];

constexpr int NT = 256;

// One block per z plane: compensated sum of F over the plane.
__global__ void k_plane_sum(gbmg::Dims d, const double* __restrict__ F, double* __restrict__ scratch) {
  __shared__ double sh[32];
  const int z = blockIdx.x;
  const long long base = (long long)z * d.nx * d.ny;
  const long long np = (long long)d.nx * d.ny;
  gbmg::DfAcc s{0.f, 0.f};
  for (long long i = threadIdx.x; i < np; i += blockDim.x) {
    const float2 v = gbmg::f64_to_df(F[base + i]);
    s.add(v.x);
    s.c += v.y;
  }
  const double b = gbmg::block_sum_acc(s, sh);
  if (threadIdx.x == 0) scratch[z] = b;
}

// mean = (sum of the plane sums) / n, in a fixed order.
__global__ void k_mean(int nz, double inv_n, double* __restrict__ scratch) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int z = threadIdx.x; z < nz; z += blockDim.x) s += scratch[z];
  s = gbmg::block_sum(s, sh);
  if (threadIdx.x == 0) scratch[2 * NOALLOC_MAX_NZ] = s * inv_n;
}

// One block per z plane: sums of (F - m)^2 and of r^2, r = F - m - A phi in double-float;
// each square is rounded to FP32 and accumulated in a compensated (double-float) sum.
__global__ void k_plane_resid(gbmg::Dims d, const double* __restrict__ F, const double* __restrict__ phi,
                              double* __restrict__ scratch) {
  __shared__ double sh[32];
  const int z = blockIdx.x;
  const long long np = (long long)d.nx * d.ny;
  const long long pst = np;
  const long long base = (long long)z * pst;
  const long long zm = (long long)(z == 0 ? d.nz - 1 : z - 1) * pst, zp = (long long)(z == d.nz - 1 ? 0 : z + 1) * pst;
  const float2 m = gbmg::f64_to_df(scratch[2 * NOALLOC_MAX_NZ]);
  gbmg::DfAcc f2{0.f, 0.f}, r2{0.f, 0.f};
  for (long long i = threadIdx.x; i < np; i += blockDim.x) {
    const int x = (int)(i % d.nx), y = (int)(i / d.nx);
    const int xm = x == 0 ? d.nx - 1 : x - 1, xp = x == d.nx - 1 ? 0 : x + 1;
    const int ym = y == 0 ? d.ny - 1 : y - 1, yp = y == d.ny - 1 ? 0 : y + 1;
    auto P = [&](long long zo, int xx, int yy) { return gbmg::f64_to_df(phi[zo + (long long)yy * d.nx + xx]); };
    const float2 f = gbmg::f64_to_df(F[base + i]);
    const float r = gbmg::df_resid(P(base, x, y), P(base, xm, y), P(base, xp, y), P(base, x, ym), P(base, x, yp),
                                   P(zm, x, y), P(zp, x, y), f, m);
    const float fm = __fadd_rn(__fsub_rn(f.x, m.x), __fsub_rn(f.y, m.y));
    f2.add(fm * fm);
    r2.add(r * r);
  }
  const double bf = gbmg::block_sum_acc(f2, sh);
  const double br = gbmg::block_sum_acc(r2, sh);
  if (threadIdx.x == 0) {
    scratch[z] = bf;
    scratch[NOALLOC_MAX_NZ + z] = br;
  }
}

// rel = sqrt(sum r^2 / sum (F - m)^2), written to the caller's device scalar.
__global__ void k_rel(int nz, const double* __restrict__ scratch, double* __restrict__ out) {
  __shared__ double sh[32];
  double f = 0.0, r = 0.0;
  for (int z = threadIdx.x; z < nz; z += blockDim.x) {
    f += scratch[z];
    r += scratch[NOALLOC_MAX_NZ + z];
  }
  f = gbmg::block_sum(f, sh);
  r = gbmg::block_sum(r, sh);
  if (threadIdx.x == 0) out[0] = f > 0.0 ? sqrt(r / f) : sqrt(r);
}

}  // namespace

extern "C" gbmg_status mg_rel_residual_noalloc(int nx, int ny, int nz, const double* source_dev,
                                               const double* phi_dev, double* rel_out_dev, void* cuda_stream) {
  if (!source_dev || !phi_dev || !rel_out_dev)
    return gbmg::fail(GBMG_ERR_INVALID_ARG, "mg_rel_residual_noalloc: NULL argument");
  if (nx < 4 || ny < 4 || nz < 4) return gbmg::fail(GBMG_ERR_INVALID_ARG, "mg_rel_residual_noalloc: every side must be >= 4");
  if (nz > NOALLOC_MAX_NZ)
    return gbmg::fail(GBMG_ERR_INVALID_ARG,
                      "mg_rel_residual_noalloc: nz exceeds the 4096 planes its fixed scratch holds");
  if ((long long)nx * ny > 0x7fffffffll)
    return gbmg::fail(GBMG_ERR_INVALID_ARG, "mg_rel_residual_noalloc: a z plane exceeds 2^31 - 1 cells");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return gbmg::cuda_fail(e, "mg_rel_residual_noalloc: cudaGetDevice");
  if (dev < 0 || dev >= MAX_DEVICES) return gbmg::fail(GBMG_ERR_INVALID_ARG, "mg_rel_residual_noalloc: device index above 63");
  double* scratch = g_scratch_addr[dev].load(std::memory_order_acquire);
  if (!scratch) {
    // set-up on the first call on this device (this device is current)
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return gbmg::cuda_fail(e, "mg_rel_residual_noalloc: cudaGetSymbolAddress");
    scratch = (double*)p;
    g_scratch_addr[dev].store(scratch, std::memory_order_release);
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const gbmg::Dims d{nx, ny, nz};
  k_plane_sum<<<nz, NT, 0, st>>>(d, source_dev, scratch);
  k_mean<<<1, 1024, 0, st>>>(nz, 1.0 / ((double)nx * ny * nz), scratch);
  k_plane_resid<<<nz, NT, 0, st>>>(d, source_dev, phi_dev, scratch);
  k_rel<<<1, 1024, 0, st>>>(nz, scratch, rel_out_dev);
  for (int i = 0; i < 4; ++i) gbmg::note_launch();
  e = cudaGetLastError();
  if (e != cudaSuccess) return gbmg::cuda_fail(e, "mg_rel_residual_noalloc: launch");
  return GBMG_OK;
}
