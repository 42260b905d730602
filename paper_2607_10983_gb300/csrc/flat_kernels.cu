// One-kernel-per-operation flat multigrid kernels (T = float or double), reductions
// and the double-float kernels of the mixed-precision defect correction.
//
// These are the plain path: every operation of the V-cycle (Sec. 2.3) is its own
// launch, one thread per cell, periodic neighbours by explicit index wrap.  In FP64
// they form the baseline "plain FP64 V-cycle"; in FP32 they are the reference
// against which the temporally blocked kernels are checked bit for bit.
#include <cstdint>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "kernels.h"
#include "stencil.cuh"

namespace gbmg {

namespace {

constexpr int BX = 32, BY = 8;
constexpr int RED_THREADS = 256;
constexpr long long RED_MAX_BLOCKS = 152 * 16;

inline dim3 cell_grid(Dims d) { return dim3((d.nx + BX - 1) / BX, (d.ny + BY - 1) / BY, d.nz); }

inline int red_blocks(long long n) {
  long long b = (n + RED_THREADS - 1) / RED_THREADS;
  if (b > RED_MAX_BLOCKS) b = RED_MAX_BLOCKS;
  return (int)(b < 1 ? 1 : b);
}

// Load the six face neighbours of (x, y, z) from a periodic field.
template <typename V>
struct Nbrs {
  V xm, xp, ym, yp, zm, zp;
};

template <typename V>
__device__ __forceinline__ Nbrs<V> load_nbrs(const V* __restrict__ u, Dims d, int x, int y, int z,
                                              long long i) {
  const long long sy = d.nx, sz = (long long)d.nx * d.ny;
  Nbrs<V> n;
  n.xm = u[i + ((x == 0 ? d.nx - 1 : x - 1) - x)];
  n.xp = u[i + ((x == d.nx - 1 ? 0 : x + 1) - x)];
  n.ym = u[i + (long long)((y == 0 ? d.ny - 1 : y - 1) - y) * sy];
  n.yp = u[i + (long long)((y == d.ny - 1 ? 0 : y + 1) - y) * sy];
  n.zm = u[i + (long long)((z == 0 ? d.nz - 1 : z - 1) - z) * sz];
  n.zp = u[i + (long long)((z == d.nz - 1 ? 0 : z + 1) - z) * sz];
  return n;
}

template <typename T>
__device__ __forceinline__ T nsum(const Nbrs<T>& n) {
  return nbr_sum(n.xm, n.xp, n.ym, n.yp, n.zm, n.zp);
}

template <typename T>
__device__ __forceinline__ float sq_as_float(T v) { return (float)v * (float)v; }

template <typename T>
__global__ void k_apply(Dims d, const T* __restrict__ u, T* __restrict__ out, T inv_h2) {
  const int x = blockIdx.x * BX + threadIdx.x, y = blockIdx.y * BY + threadIdx.y, z = blockIdx.z;
  if (x >= d.nx || y >= d.ny) return;
  const long long i = lin(d, x, y, z);
  out[i] = lap_from_sum(nsum(load_nbrs(u, d, x, y, z, i)), u[i], inv_h2);
}

template <typename T>
__global__ void k_residual(Dims d, const T* __restrict__ f, const T* __restrict__ u, T* __restrict__ out,
                           T inv_h2, double* __restrict__ partials) {
  __shared__ double sh[32];
  const int x = blockIdx.x * BX + threadIdx.x, y = blockIdx.y * BY + threadIdx.y, z = blockIdx.z;
  T r = T(0);
  if (x < d.nx && y < d.ny) {
    const long long i = lin(d, x, y, z);
    r = resid_from_sum(f[i], nsum(load_nbrs(u, d, x, y, z, i)), u[i], inv_h2);
    out[i] = r;
  }
  if (partials) {
    double s;
    if constexpr (sizeof(T) == 8) s = block_sum((double)r * (double)r, sh);
    else s = block_sum_f(r * r, sh);
    if (is_thread0()) partials[block_linear_id()] = s;
  }
}

template <typename T>
__global__ void k_cheb_step(Dims d, const T* __restrict__ r, const T* __restrict__ e_in, T* __restrict__ e_out,
                            T* __restrict__ dvec, T a, T b, T c1) {
  const int x = blockIdx.x * BX + threadIdx.x, y = blockIdx.y * BY + threadIdx.y, z = blockIdx.z;
  if (x >= d.nx || y >= d.ny) return;
  const long long i = lin(d, x, y, z);
  const T c = e_in[i];
  T dv = c1 == T(0) ? T(0) : dvec[i];
  e_out[i] = cheb_step(c, r[i], nsum(load_nbrs(e_in, d, x, y, z, i)), c, dv, a, b, c1);
  dvec[i] = dv;
}

template <typename T>
__global__ void k_jacobi(Dims d, const T* __restrict__ r, const T* __restrict__ e_in, T* __restrict__ e_out,
                         T wa, T wb) {
  const int x = blockIdx.x * BX + threadIdx.x, y = blockIdx.y * BY + threadIdx.y, z = blockIdx.z;
  if (x >= d.nx || y >= d.ny) return;
  const long long i = lin(d, x, y, z);
  const T c = e_in[i];
  e_out[i] = jacobi_step(c, r[i], nsum(load_nbrs(e_in, d, x, y, z, i)), c, wa, wb);
}

// Full weighting, one thread per coarse cell: z-axis weights first, then y, then x
// (the order the fused kernels use).
template <typename T>
__global__ void k_restrict(Dims df, const T* __restrict__ f, T* __restrict__ c) {
  const Dims dc{df.nx / 2, df.ny / 2, df.nz / 2};
  const int X = blockIdx.x * BX + threadIdx.x, Y = blockIdx.y * BY + threadIdx.y, Z = blockIdx.z;
  if (X >= dc.nx || Y >= dc.ny) return;
  int xs[3], ys[3], zs[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    xs[k] = wrapi(2 * X + k - 1, df.nx);
    ys[k] = wrapi(2 * Y + k - 1, df.ny);
    zs[k] = wrapi(2 * Z + k - 1, df.nz);
  }
  T yv[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    T zv[3];
#pragma unroll
    for (int b = 0; b < 3; ++b)
      zv[b] = fw3(f[lin(df, xs[a], ys[b], zs[0])], f[lin(df, xs[a], ys[b], zs[1])], f[lin(df, xs[a], ys[b], zs[2])]);
    yv[a] = fw3(zv[0], zv[1], zv[2]);
  }
  c[lin(dc, X, Y, Z)] = fw3(yv[0], yv[1], yv[2]);
}

template <typename T>
__global__ void k_prolong_add(Dims dc, const T* __restrict__ c, T* __restrict__ f) {
  const Dims df{dc.nx * 2, dc.ny * 2, dc.nz * 2};
  const int x = blockIdx.x * BX + threadIdx.x, y = blockIdx.y * BY + threadIdx.y, z = blockIdx.z;
  if (x >= df.nx || y >= df.ny) return;
  const long long i = lin(df, x, y, z);
  f[i] = t_add(f[i], prolong_value(c, dc, x, y, z));
}

// f += P c in FP32 with one thread per coarse cell (I, J, K): the eight coarse values at
// I..I+1, J..J+1, K..K+1 (periodic) are loaded once and give the fine cells {2I, 2I+1} x
// {2J, 2J+1} x {2K, 2K+1}, each formed like prolong_value (x, then y, then z midpoints,
// the same roundings), so the results are the same bits as k_prolong_add's; the fine
// rows are read and written as x-pairs (f 8-byte aligned).
__global__ void k_prolong_add_blocks(Dims dc, const float* __restrict__ c, float* __restrict__ f) {
  const int I = blockIdx.x * BX + threadIdx.x, J = blockIdx.y * BY + threadIdx.y, K = blockIdx.z;
  if (I >= dc.nx || J >= dc.ny) return;
  const Dims df{dc.nx * 2, dc.ny * 2, dc.nz * 2};
  const int I1 = wrap_hi(I + 1, dc.nx), J1 = wrap_hi(J + 1, dc.ny), K1 = wrap_hi(K + 1, dc.nz);
  // (fine x = 2I, fine x = 2I + 1) on the coarse row (jj, kk)
  auto xpair = [&](int jj, int kk) {
    const float v0 = c[lin(dc, I, jj, kk)];
    return make_float2(v0, half_sum(v0, c[lin(dc, I1, jj, kk)]));
  };
  auto mid = [](float2 a, float2 b) { return make_float2(half_sum(a.x, b.x), half_sum(a.y, b.y)); };
  const float2 xJK = xpair(J, K), xJ1K = xpair(J1, K), xJK1 = xpair(J, K1), xJ1K1 = xpair(J1, K1);
  // fine rows 2J (dy = 0) and 2J + 1 (dy = 1) on the coarse planes K and K1
  const float2 yK[2] = {xJK, mid(xJK, xJ1K)};
  const float2 yK1[2] = {xJK1, mid(xJK1, xJ1K1)};
#pragma unroll
  for (int dz = 0; dz < 2; ++dz)
#pragma unroll
    for (int dy = 0; dy < 2; ++dy) {
      const float2 v = dz ? mid(yK[dy], yK1[dy]) : yK[dy];
      float2* const p = reinterpret_cast<float2*>(f + lin(df, 2 * I, 2 * J + dy, 2 * K + dz));
      const float2 o = *p;
      *p = make_float2(t_add(o.x, v.x), t_add(o.y, v.y));
    }
}

// e = G r, one warp per row, lanes stride the columns; fixed summation order.
template <typename T>
__global__ void k_coarse_matvec(int n, const T* __restrict__ G, const T* __restrict__ r, T* __restrict__ e) {
  const int row = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  T acc = T(0);
  for (int j = lane; j < n; j += 32) acc = t_fma(G[(long long)row * n + j], r[j], acc);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc = t_add(acc, __shfl_xor_sync(0xffffffffu, acc, o));
  if (lane == 0) e[row] = acc;
}

template <typename T>
__global__ void k_sum(long long n, const T* __restrict__ x, double* __restrict__ ps, double* __restrict__ pq) {
  __shared__ double sh[32];
  T s = T(0), q = T(0);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const T v = x[i];
    s += v;
    q += v * v;
  }
  double bs, bq;
  if constexpr (sizeof(T) == 8) {
    bs = block_sum((double)s, sh);
    bq = block_sum((double)q, sh);
  } else {
    bs = block_sum_f(s, sh);
    bq = block_sum_f(q, sh);
  }
  if (threadIdx.x == 0) {
    if (ps) ps[blockIdx.x] = bs;
    if (pq) pq[blockIdx.x] = bq;
  }
}

template <typename T>
__global__ void k_shift(long long n, const T* __restrict__ x, const double* __restrict__ shift, T* __restrict__ out) {
  const T s = (T)shift[0];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = t_sub(x[i], s);
}

// Storage of a coarse-level correction in a 16-bit format: each value rounded to
// nearest (ties to even) in BF16 (mode 1) or FP16 (mode 2) and held as FP32 again.
template <int MODE>
__global__ void k_round16(long long n, float* __restrict__ e) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float v = e[i];
    e[i] = MODE == 1 ? __bfloat162float(__float2bfloat16_rn(v)) : __half2float(__float2half_rn(v));
  }
}

// A few device scalars into page-locked host memory through its device address (no copy
// engine: the scalars do not queue behind large copies of other streams).
__global__ void k_scalars_to_host(const double* __restrict__ src, double* __restrict__ dst, int n) {
  if ((int)threadIdx.x < n) dst[threadIdx.x] = src[threadIdx.x];
  __threadfence_system();
}

__global__ void k_finalize(const double* __restrict__ p, long long count, double* __restrict__ out, double scale) {
  __shared__ double sh[32];
  double s = 0.0;
  for (long long i = threadIdx.x; i < count; i += blockDim.x) s += p[i];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) out[0] = s * scale;
}

// ---- double-float ----

// One element per access (any alignment); elements are visited in the pair order of
// k_f64_to_df_x2 (pair q = elements 2q, 2q + 1) so that the partial sums, and with them
// the mean, do not depend on the alignment of x.
__global__ void k_f64_to_df(long long n, const double* __restrict__ x, float2* __restrict__ out,
                            double* __restrict__ ps) {
  __shared__ double sh[32];
  DfAcc s{0.f, 0.f};
  const long long n2 = n / 2;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n2; q += (long long)gridDim.x * blockDim.x) {
    const float2 a = f64_to_df(x[2 * q]), b = f64_to_df(x[2 * q + 1]);
    out[2 * q] = a;
    out[2 * q + 1] = b;
    s.add(a.x);
    s.c += a.y;
    s.add(b.x);
    s.c += b.y;
  }
  if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
    const float2 a = f64_to_df(x[n - 1]);
    out[n - 1] = a;
    s.add(a.x);
    s.c += a.y;
  }
  if (ps) {
    const double b = block_sum_acc(s, sh);
    if (threadIdx.x == 0) ps[blockIdx.x] = b;
  }
}

// Two consecutive elements per thread and iteration (16-byte accesses; x, out 16-byte
// aligned, n2 = n / 2 pairs, the odd last element by thread 0 of block 0).
__global__ void k_f64_to_df_x2(long long n, const double2* __restrict__ x, float4* __restrict__ out,
                               double* __restrict__ ps) {
  __shared__ double sh[32];
  DfAcc s{0.f, 0.f};
  const long long n2 = n / 2;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n2; i += (long long)gridDim.x * blockDim.x) {
    const double2 v = x[i];
    const float2 a = f64_to_df(v.x), b = f64_to_df(v.y);
    out[i] = make_float4(a.x, a.y, b.x, b.y);
    s.add(a.x);
    s.c += a.y;
    s.add(b.x);
    s.c += b.y;
  }
  if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
    const float2 a = f64_to_df(reinterpret_cast<const double*>(x)[n - 1]);
    reinterpret_cast<float2*>(out)[n - 1] = a;
    s.add(a.x);
    s.c += a.y;
  }
  if (ps) {
    const double b = block_sum_acc(s, sh);
    if (threadIdx.x == 0) ps[blockIdx.x] = b;
  }
}

__global__ void k_df_to_f64_x2(long long n, const float4* __restrict__ in, const double* __restrict__ shift,
                               double2* __restrict__ out) {
  float2 ms = make_float2(0.f, 0.f);
  if (shift) {
    ms = f64_to_df(shift[0]);
    ms.x = -ms.x;
    ms.y = -ms.y;
  }
  const long long n2 = n / 2;
  auto conv = [&](float4 v) {
    float2 a = make_float2(v.x, v.y), b = make_float2(v.z, v.w);
    if (shift) {
      a = df_add(a, ms);
      b = df_add(b, ms);
    }
    return make_double2(df_to_f64(a), df_to_f64(b));
  };
  // two grid strides per iteration: both loads are in flight before either conversion
  const long long G = (long long)gridDim.x * blockDim.x;
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  for (; i + G < n2; i += 2 * G) {
    const float4 v0 = in[i], v1 = in[i + G];
    out[i] = conv(v0);
    out[i + G] = conv(v1);
  }
  if (i < n2) out[i] = conv(in[i]);
  if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
    float2 a = reinterpret_cast<const float2*>(in)[n - 1];
    if (shift) a = df_add(a, ms);
    reinterpret_cast<double*>(out)[n - 1] = df_to_f64(a);
  }
}

__global__ void k_df_to_f64(long long n, const float2* __restrict__ in, const double* __restrict__ shift,
                            double* __restrict__ out) {
  float2 ms = make_float2(0.f, 0.f);
  if (shift) {
    ms = f64_to_df(shift[0]);
    ms.x = -ms.x;
    ms.y = -ms.y;
  }
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    float2 v = in[i];
    if (shift) v = df_add(v, ms);
    out[i] = df_to_f64(v);
  }
}

__global__ void k_df_residual(Dims d, const float2* __restrict__ F, const double* __restrict__ m_dev,
                              const float2* __restrict__ phi, float* __restrict__ r,
                              double* __restrict__ pr2, double* __restrict__ pf2) {
  __shared__ double sh[32];
  const float2 m = f64_to_df(m_dev ? m_dev[0] : 0.0);
  const int x = blockIdx.x * BX + threadIdx.x, y = blockIdx.y * BY + threadIdx.y, z = blockIdx.z;
  float rv = 0.f, fv = 0.f;
  if (x < d.nx && y < d.ny) {
    const long long i = lin(d, x, y, z);
    const Nbrs<float2> nb = load_nbrs(phi, d, x, y, z, i);
    const float2 f = F[i];
    rv = df_resid(phi[i], nb.xm, nb.xp, nb.ym, nb.yp, nb.zm, nb.zp, f, m);
    r[i] = rv;
    fv = __fadd_rn(__fsub_rn(f.x, m.x), __fsub_rn(f.y, m.y));
  }
  if (pr2) {
    const double s = block_sum_f(rv * rv, sh);
    if (is_thread0()) pr2[block_linear_id()] = s;
  }
  if (pf2) {
    const double s = block_sum_f(fv * fv, sh);
    if (is_thread0()) pf2[block_linear_id()] = s;
  }
}

__global__ void k_df_update(long long n, float2* __restrict__ phi, const float* __restrict__ e,
                            double* __restrict__ ps) {
  __shared__ double sh[32];
  DfAcc s{0.f, 0.f};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    float2 v = phi[i];
    if (e) {
      v = df_add_f(v, e[i]);
      phi[i] = v;
    }
    s.add(v.x);
    s.c += v.y;
  }
  if (ps) {
    const double b = block_sum_acc(s, sh);
    if (threadIdx.x == 0) ps[blockIdx.x] = b;
  }
}

}  // namespace

long long partial_count(Dims d) {
  const dim3 g = cell_grid(d);
  return (long long)g.x * g.y * g.z;
}

long long df_partial_count(long long n) { return red_blocks(n); }

template <typename T>
cudaError_t launch_apply(cudaStream_t st, Dims d, const T* u, T* out, T inv_h2) {
  k_apply<T><<<cell_grid(d), dim3(BX, BY), 0, st>>>(d, u, out, inv_h2);
  note_launch();
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_residual(cudaStream_t st, Dims d, const T* f, const T* u, T* out, T inv_h2, double* p) {
  k_residual<T><<<cell_grid(d), dim3(BX, BY), 0, st>>>(d, f, u, out, inv_h2, p);
  note_launch();
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_cheb_step(cudaStream_t st, Dims d, const T* r, const T* e_in, T* e_out, T* dvec, T a, T b, T c1) {
  k_cheb_step<T><<<cell_grid(d), dim3(BX, BY), 0, st>>>(d, r, e_in, e_out, dvec, a, b, c1);
  note_launch();
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_jacobi(cudaStream_t st, Dims d, const T* r, const T* e_in, T* e_out, T wa, T wb) {
  k_jacobi<T><<<cell_grid(d), dim3(BX, BY), 0, st>>>(d, r, e_in, e_out, wa, wb);
  note_launch();
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_restrict(cudaStream_t st, Dims fine, const T* f, T* c) {
  const Dims dc{fine.nx / 2, fine.ny / 2, fine.nz / 2};
  k_restrict<T><<<cell_grid(dc), dim3(BX, BY), 0, st>>>(fine, f, c);
  note_launch();
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_prolong_add(cudaStream_t st, Dims coarse, const T* c, T* f) {
  const Dims df{coarse.nx * 2, coarse.ny * 2, coarse.nz * 2};
  if (sizeof(T) == 4 && ((uintptr_t)f & 7) == 0)
    k_prolong_add_blocks<<<cell_grid(coarse), dim3(BX, BY), 0, st>>>(coarse, (const float*)c, (float*)f);
  else
    k_prolong_add<T><<<cell_grid(df), dim3(BX, BY), 0, st>>>(coarse, c, f);
  note_launch();
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_coarse_matvec(cudaStream_t st, int n, const T* G, const T* r, T* e) {
  const int rows_per_block = 8;
  k_coarse_matvec<T><<<(n + rows_per_block - 1) / rows_per_block, 32 * rows_per_block, 0, st>>>(n, G, r, e);
  note_launch();
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_sum(cudaStream_t st, long long n, const T* x, double* ps, double* pq) {
  k_sum<T><<<red_blocks(n), RED_THREADS, 0, st>>>(n, x, ps, pq);
  note_launch();
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_shift(cudaStream_t st, long long n, const T* x, const double* shift, T* out) {
  k_shift<T><<<red_blocks(n), RED_THREADS, 0, st>>>(n, x, shift, out);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_round16(cudaStream_t st, long long n, float* e, int mode) {
  if (mode == 1) k_round16<1><<<red_blocks(n), RED_THREADS, 0, st>>>(n, e);
  else if (mode == 2) k_round16<2><<<red_blocks(n), RED_THREADS, 0, st>>>(n, e);
  else return cudaErrorInvalidValue;
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_finalize(cudaStream_t st, const double* p, long long count, double* out, double scale) {
  k_finalize<<<1, 1024, 0, st>>>(p, count, out, scale);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_scalars_to_host(cudaStream_t st, const double* src, double* dst_mapped, int n) {
  if (n < 0 || n > 32) return cudaErrorInvalidValue;
  k_scalars_to_host<<<1, 32, 0, st>>>(src, dst_mapped, n);
  note_launch();
  return cudaGetLastError();
}

static bool aligned16(const void* a, const void* b) {
  return ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b)) & 15) == 0;
}

// df_partial_count(n) partials either way (the pair form runs red_blocks(n) blocks too)
cudaError_t launch_f64_to_df(cudaStream_t st, long long n, const double* x, float2* out, double* ps) {
  if (aligned16(x, out))
    k_f64_to_df_x2<<<red_blocks(n), RED_THREADS, 0, st>>>(n, reinterpret_cast<const double2*>(x),
                                                           reinterpret_cast<float4*>(out), ps);
  else
    k_f64_to_df<<<red_blocks(n), RED_THREADS, 0, st>>>(n, x, out, ps);
  note_launch();
  return cudaGetLastError();
}
cudaError_t launch_df_to_f64(cudaStream_t st, long long n, const float2* in, const double* shift, double* out) {
  if (aligned16(in, out))
    k_df_to_f64_x2<<<red_blocks(n), RED_THREADS, 0, st>>>(n, reinterpret_cast<const float4*>(in), shift,
                                                           reinterpret_cast<double2*>(out));
  else
    k_df_to_f64<<<red_blocks(n), RED_THREADS, 0, st>>>(n, in, shift, out);
  note_launch();
  return cudaGetLastError();
}
cudaError_t launch_df_residual(cudaStream_t st, Dims d, const float2* F, const double* m_dev, const float2* phi,
                               float* r, double* pr2, double* pf2) {
  k_df_residual<<<cell_grid(d), dim3(BX, BY), 0, st>>>(d, F, m_dev, phi, r, pr2, pf2);
  note_launch();
  return cudaGetLastError();
}
cudaError_t launch_df_update(cudaStream_t st, long long n, float2* phi, const float* e, double* ps) {
  k_df_update<<<red_blocks(n), RED_THREADS, 0, st>>>(n, phi, e, ps);
  note_launch();
  return cudaGetLastError();
}

#define GBMG_INSTANTIATE(T)                                                                           \
  template cudaError_t launch_apply<T>(cudaStream_t, Dims, const T*, T*, T);                         \
  template cudaError_t launch_residual<T>(cudaStream_t, Dims, const T*, const T*, T*, T, double*);   \
  template cudaError_t launch_cheb_step<T>(cudaStream_t, Dims, const T*, const T*, T*, T*, T, T, T);  \
  template cudaError_t launch_jacobi<T>(cudaStream_t, Dims, const T*, const T*, T*, T, T);           \
  template cudaError_t launch_restrict<T>(cudaStream_t, Dims, const T*, T*);                         \
  template cudaError_t launch_prolong_add<T>(cudaStream_t, Dims, const T*, T*);                      \
  template cudaError_t launch_coarse_matvec<T>(cudaStream_t, int, const T*, const T*, T*);           \
  template cudaError_t launch_sum<T>(cudaStream_t, long long, const T*, double*, double*);           \
  template cudaError_t launch_shift<T>(cudaStream_t, long long, const T*, const double*, T*);
GBMG_INSTANTIATE(float)
GBMG_INSTANTIATE(double)
#undef GBMG_INSTANTIATE

}  // namespace gbmg
