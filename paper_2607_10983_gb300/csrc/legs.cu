// Temporally blocked FP32 level kernels (the single-GPU form of the paper's
// communication-avoiding whole-level fusion, Sec. 3.4 implementation list): one
// HBM pass per level visit and leg instead of one per operation.
//
//   k_down_fused : Chebyshev pre-smoothing from e = 0 (degree V), residual and
//                  full-weighting restriction.  Reads r, writes e and R(r - A e).
//   k_up_fused   : trilinear prolongation + correction and Chebyshev
//                  post-smoothing.  Reads e, e_c, r; writes the new e.
//
// Blocking scheme.  A CTA owns an output tile of TX x TY cells in (x, y) and a range
// of z planes; it computes on the tile plus a halo (H cells in y, H rounded up to
// whole pairs in x), so that every stage, which needs its input on one more ring of
// cells, still produces valid values on the tile.  The CTA streams through z: each
// iteration loads one input plane and every stage advances one plane, stage s one
// plane behind stage s-1.  One barrier per iteration.
//
// Work unit: the pair of x-neighbouring cells (even x, odd x), computed with packed
// FP32x2 instructions; a thread owns a column of R pairs stacked in y.  Shared
// memory holds each stage's current plane split by x parity (even cells, odd cells),
// so the x neighbours of a pair are two conflict-free scalar loads; y neighbours
// inside the column and the two older z planes stay in registers.  Every lane of a
// packed instruction rounds like the scalar intrinsic of the one-kernel-per-operation
// path, in the same order, so the results are bit-identical to it.
//
// Schedule: persistent grid of one CTA per SM; the (tile, plane) pairs form one
// tile-major list and CTA b runs the contiguous range [b T / G, (b+1) T / G), as one
// z segment per tile it touches (each segment with its own warm-up planes).  Each
// tile's z stream starts at its own phase (tile_phase), so that neighbouring tiles
// stream the same planes at about the same time and their shared halo rows are read
// from DRAM about once.
#include <type_traits>

#include "legs.cuh"

namespace gbmg {

namespace {

using namespace legs;

template <int V, class TL>
__global__ void __maxnreg__(65536 / ((TL::NT + 127) / 128 * 128) / 8 * 8)
k_down_fused(Dims d, const float* __restrict__ r, float* __restrict__ e_out, float* __restrict__ rc, Sched sc,
             float inv_h2, Coef cf) {
  extern __shared__ float sm[];
  long long a = (long long)blockIdx.x * sc.total / gridDim.x;
  const long long b = (long long)(blockIdx.x + 1) * sc.total / gridDim.x;
  while (a < b) {
    const long long tile = a / d.nz;
    const int p0 = (int)(a - tile * d.nz);
    const int z0 = (tile_phase(tile * d.nz, d.nz, sc.total, gridDim.x) + p0) % d.nz;
    int len = (int)(b - a < d.nz - p0 ? b - a : d.nz - p0);
    if (len > d.nz - z0) len = d.nz - z0;  // not taken (tile_phase): a run never crosses plane nz
    down_segment<V, TL>(d, r, e_out, rc, (int)(tile % sc.tiles_x) * TL::TX, (int)(tile / sc.tiles_x) * TL::TY, z0,
                        z0 + len, inv_h2, cf, sm);
    a += len;
    __syncthreads();
  }
}

template <int V, class TL>
__global__ void __maxnreg__(65536 / ((TL::NT + 127) / 128 * 128) / 8 * 8)
k_up_fused(Dims d, const float* __restrict__ e_in, const float* __restrict__ ec, const float* __restrict__ r,
           float* __restrict__ e_out, Sched sc, float inv_h2, Coef cf) {
  extern __shared__ float sm[];
  long long a = (long long)blockIdx.x * sc.total / gridDim.x;
  const long long b = (long long)(blockIdx.x + 1) * sc.total / gridDim.x;
  while (a < b) {
    const long long tile = a / d.nz;
    const int p0 = (int)(a - tile * d.nz);
    const int z0 = (tile_phase(tile * d.nz, d.nz, sc.total, gridDim.x) + p0) % d.nz;
    int len = (int)(b - a < d.nz - p0 ? b - a : d.nz - p0);
    if (len > d.nz - z0) len = d.nz - z0;  // not taken (tile_phase): a run never crosses plane nz
    up_segment<V, TL>(d, e_in, ec, r, e_out, (int)(tile % sc.tiles_x) * TL::TX, (int)(tile / sc.tiles_x) * TL::TY,
                      z0, z0 + len, inv_h2, cf, sm);
    a += len;
    __syncthreads();
  }
}

// ------------------------------------------------------------------ launch

// Tiles per degree: 64 x 32 cells; block sizes are multiples of 128 threads
// (registers are granted to groups of four warps).  Down leg (degrees 1-3): columns of
// R = 3 pairs, 512 threads: 16 warps per SM within 128 registers (0.554 ms at 512^3
// against 0.595 with 4-pair columns in 384 threads, 12 warps at 168 registers: the leg
// is bound by dependency latency, which more warps hide); degree 4 (halo 5) keeps 4-pair
// columns, 384 threads and a 64 x 24 tile, which fit its shared memory.  Up leg: columns
// of R = 4 pairs, 384 threads (even R makes each row's y parity, and with it the
// prolongation's coarse-row pattern, a compile-time constant).
template <int V>
struct DownTile {
  using T = typename std::conditional<(V >= 4), PTile<64, 24, V + 1, 384, 4>, PTile<64, 32, V + 1, 512, 3>>::type;
};
template <int V>
struct UpTile {
  using T = PTile<64, 32, V, 384, 4>;
};

template <int V>
size_t down_smem() {
  return (size_t)(V + 1) * 2 * DownTile<V>::T::PLANE * sizeof(float);
}
template <int V>
size_t up_smem() {
  using TL = typename UpTile<V>::T;
  return ((size_t)V * 2 * TL::PLANE + 3 * PCoarse<TL>::CN) * sizeof(float);
}

Coef make_coef(const double* c1, const double* c2, int v, double h) {
  Coef cf{};
  for (int i = 0; i < v && i < 16; ++i) {
    double a, b;
    cheb_constants(c2[i], h, a, b);
    cf.c1[i] = (float)c1[i];
    cf.a[i] = (float)a;
    cf.b[i] = (float)b;
  }
  return cf;
}

int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1)
      n = 152;
  }
  return n;
}

template <class TL>
Sched make_sched(Dims d, int& ctas) {
  Sched sc;
  sc.tiles_x = (d.nx + TL::TX - 1) / TL::TX;
  sc.total = (long long)sc.tiles_x * ((d.ny + TL::TY - 1) / TL::TY) * d.nz;
  const long long g = sc.total < sm_count() ? sc.total : sm_count();
  ctas = (int)g;
  return sc;
}

template <int V>
cudaError_t down_v(cudaStream_t st, Dims d, const float* r, float* e, float* rc, float ih2, const Coef& cf) {
  using TL = typename DownTile<V>::T;
  static bool attr = false;
  const size_t sm = down_smem<V>();
  if (!attr) {
    cudaError_t err = cudaFuncSetAttribute(k_down_fused<V, TL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (err != cudaSuccess) return err;
    attr = true;
  }
  int ctas = 0;
  const Sched sc = make_sched<TL>(d, ctas);
  k_down_fused<V, TL><<<ctas, TL::NT, sm, st>>>(d, r, e, rc, sc, ih2, cf);
  note_launch();
  return cudaGetLastError();
}

template <int V>
cudaError_t up_v(cudaStream_t st, Dims d, const float* e_in, const float* ec, const float* r, float* e_out,
                 float ih2, const Coef& cf) {
  using TL = typename UpTile<V>::T;
  static bool attr = false;
  const size_t sm = up_smem<V>();
  if (!attr) {
    cudaError_t err = cudaFuncSetAttribute(k_up_fused<V, TL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (err != cudaSuccess) return err;
    attr = true;
  }
  int ctas = 0;
  const Sched sc = make_sched<TL>(d, ctas);
  k_up_fused<V, TL><<<ctas, TL::NT, sm, st>>>(d, e_in, ec, r, e_out, sc, ih2, cf);
  note_launch();
  return cudaGetLastError();
}

}  // namespace

bool fused_degree_supported(int degree) { return degree >= 1 && degree <= 4; }

cudaError_t launch_down_fused(cudaStream_t st, int degree, Dims d, const float* r, float* e, float* rc, double h,
                              const double* c1, const double* c2) {
  if (d.nx % 2 || d.ny % 2 || d.nz % 2) return cudaErrorInvalidValue;  // levels that are coarsened are even
  const Coef cf = make_coef(c1, c2, degree, h);
  const float ih2 = (float)(1.0 / (h * h));
  switch (degree) {
    case 1: return down_v<1>(st, d, r, e, rc, ih2, cf);
    case 2: return down_v<2>(st, d, r, e, rc, ih2, cf);
    case 3: return down_v<3>(st, d, r, e, rc, ih2, cf);
    case 4: return down_v<4>(st, d, r, e, rc, ih2, cf);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_up_fused(cudaStream_t st, int degree, Dims d, const float* e_in, const float* ec, const float* r,
                            float* e_out, double h, const double* c1, const double* c2) {
  if (d.nx % 2 || d.ny % 2 || d.nz % 2) return cudaErrorInvalidValue;
  const Coef cf = make_coef(c1, c2, degree, h);
  const float ih2 = (float)(1.0 / (h * h));
  switch (degree) {
    case 1: return up_v<1>(st, d, e_in, ec, r, e_out, ih2, cf);
    case 2: return up_v<2>(st, d, e_in, ec, r, e_out, ih2, cf);
    case 3: return up_v<3>(st, d, e_in, ec, r, e_out, ih2, cf);
    case 4: return up_v<4>(st, d, e_in, ec, r, e_out, ih2, cf);
  }
  return cudaErrorInvalidValue;
}

}  // namespace gbmg
