// Particle-mesh steps around the Poisson solve (Sec. 2.1 "The PM gravity solve";
// Sec. 3.4, force evaluation = paint, solve, gradient, read): cloud-in-cell paint
// and read on the finest level of a context.  Positions in cell units, node
// (i, j, k) at position (i, j, k), periodic; per axis node floor(x) gets weight
// 1 - f and node floor(x) + 1 weight f, f = x - floor(x), formed in FP64 from the
// FP32 position (exact).  Read is the transpose of paint.
#include "kernels.h"
#include "solver.h"

namespace gbmg {

namespace {

struct Corners {
  long long off[8];
  double w[8];
};

// the 8 corners in the order dz, dy, dx (dx fastest) with their weights (wx wy) wz
__device__ __forceinline__ Corners cic_corners(Dims d, const float* __restrict__ pos, long long p) {
  Corners c;
  double f[3];
  int i0[3], i1[3];  // node floor(x) and floor(x) + 1, wrapped onto the mesh
  const int n[3] = {d.nx, d.ny, d.nz};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double x = (double)pos[3 * p + a];
    const double fl = floor(x);
    f[a] = __dsub_rn(x, fl);
    int i = (int)fl % n[a];
    i = i < 0 ? i + n[a] : i;
    i0[a] = i;
    i1[a] = i + 1 == n[a] ? 0 : i + 1;
  }
  int k = 0;
#pragma unroll
  for (int dz = 0; dz < 2; ++dz) {
    const double wz = dz ? f[2] : __dsub_rn(1.0, f[2]);
    const long long iz = dz ? i1[2] : i0[2];
#pragma unroll
    for (int dy = 0; dy < 2; ++dy) {
      const double wy = dy ? f[1] : __dsub_rn(1.0, f[1]);
      const long long iy = dy ? i1[1] : i0[1];
#pragma unroll
      for (int dx = 0; dx < 2; ++dx) {
        const double wx = dx ? f[0] : __dsub_rn(1.0, f[0]);
        const long long ix = dx ? i1[0] : i0[0];
        c.off[k] = (iz * d.ny + iy) * d.nx + ix;
        c.w[k] = __dmul_rn(__dmul_rn(wx, wy), wz);
        ++k;
      }
    }
  }
  return c;
}

__global__ void k_cic_paint(Dims d, const float* __restrict__ pos, const float* __restrict__ mass, double m0,
                            long long np, double* __restrict__ rho) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < np; p += (long long)gridDim.x * blockDim.x) {
    const Corners c = cic_corners(d, pos, p);
    const double m = mass ? (double)mass[p] : m0;
#pragma unroll
    for (int k = 0; k < 8; ++k) atomicAdd(rho + c.off[k], __dmul_rn(m, c.w[k]));
  }
}

__global__ void k_cic_read(Dims d, const double* __restrict__ field, int ncomp, const float* __restrict__ pos,
                           long long np, double* __restrict__ out) {
  const long long n = ncell(d);
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < np; p += (long long)gridDim.x * blockDim.x) {
    const Corners c = cic_corners(d, pos, p);
    for (int q = 0; q < ncomp; ++q) {
      const double* f = field + q * n;
      double v = 0.0;
#pragma unroll
      for (int k = 0; k < 8; ++k) v = __dadd_rn(v, __dmul_rn(c.w[k], f[c.off[k]]));
      out[p * ncomp + q] = v;
    }
  }
}

// ---- single-precision force path: phi -> FP32, fourth-order gradient in FP32, CIC read in FP32

__global__ void k_phi_to_f32(long long n, const double* __restrict__ phi, float* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = (float)phi[i];
}

__device__ __forceinline__ int wrap_any(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// g[a] = -(-u_{i+2} + 8 u_{i+1} - 8 u_{i-1} + u_{i-2}) / 12 along axis a (the force, h = 1)
__global__ void k_force_grid(Dims d, const float* __restrict__ u, float* __restrict__ g) {
  const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y, z = blockIdx.z;
  if (x >= d.nx || y >= d.ny) return;
  const long long n = ncell(d), sy = d.nx, sz = (long long)d.nx * d.ny;
  const long long i = z * sz + (long long)y * sy + x;
  const long long bx = i - x, by = i - (long long)y * sy, bz = i - z * sz;
  auto fx = [&](int s) { return u[bx + wrap_any(x + s, d.nx)]; };
  auto fy = [&](int s) { return u[by + (long long)wrap_any(y + s, d.ny) * sy]; };
  auto fz = [&](int s) { return u[bz + (long long)wrap_any(z + s, d.nz) * sz]; };
  const float c8 = 8.f / 12.f, c1 = 1.f / 12.f;
  g[i] = c8 * (fx(-1) - fx(1)) + c1 * (fx(2) - fx(-2));
  g[n + i] = c8 * (fy(-1) - fy(1)) + c1 * (fy(2) - fy(-2));
  g[2 * n + i] = c8 * (fz(-1) - fz(1)) + c1 * (fz(2) - fz(-2));
}

__global__ void k_force_read(Dims d, const float* __restrict__ g, const float* __restrict__ pos, long long np,
                             float* __restrict__ out) {
  const long long n = ncell(d);
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < np; p += (long long)gridDim.x * blockDim.x) {
    int i0[3], i1[3];
    float f[3];
    const int nn[3] = {d.nx, d.ny, d.nz};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float x = pos[3 * p + a];
      const float fl = floorf(x);
      f[a] = x - fl;
      int i = (int)fl % nn[a];
      i = i < 0 ? i + nn[a] : i;
      i0[a] = i;
      i1[a] = i + 1 == nn[a] ? 0 : i + 1;
    }
    float acc[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int dz = 0; dz < 2; ++dz) {
      const float wz = dz ? f[2] : 1.f - f[2];
      const long long oz = (long long)(dz ? i1[2] : i0[2]) * d.ny;
#pragma unroll
      for (int dy = 0; dy < 2; ++dy) {
        const float wzy = wz * (dy ? f[1] : 1.f - f[1]);
        const long long oy = (oz + (dy ? i1[1] : i0[1])) * d.nx;
#pragma unroll
        for (int dx = 0; dx < 2; ++dx) {
          const float w = wzy * (dx ? f[0] : 1.f - f[0]);
          const long long o = oy + (dx ? i1[0] : i0[0]);
#pragma unroll
          for (int q = 0; q < 3; ++q) acc[q] = fmaf(w, g[q * n + o], acc[q]);
        }
      }
    }
    out[3 * p] = acc[0];
    out[3 * p + 1] = acc[1];
    out[3 * p + 2] = acc[2];
  }
}

int particle_blocks(long long np) {
  long long b = (np + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace

}  // namespace gbmg

using namespace gbmg;

extern "C" gbmg_status mg_cic_paint(gbmg_ctx* c, const float* pos_dev, const float* mass_dev, double mass,
                                    long long n_particles, double* rho_dev) {
  if (!c || !rho_dev || n_particles < 0 || (n_particles > 0 && !pos_dev))
    return fail(GBMG_ERR_INVALID_ARG, "mg_cic_paint: bad argument");
  DeviceGuard g(c->device);
  const Dims d = c->lv[0].d;
  TRY(cudaMemsetAsync(rho_dev, 0, (size_t)ncell(d) * sizeof(double), c->stream));
  if (n_particles == 0) return GBMG_OK;
  k_cic_paint<<<particle_blocks(n_particles), 256, 0, c->stream>>>(d, pos_dev, mass_dev, mass, n_particles, rho_dev);
  note_launch();
  TRY(cudaGetLastError());
  return GBMG_OK;
}

extern "C" gbmg_status mg_cic_read(gbmg_ctx* c, const double* field_dev, int ncomp, const float* pos_dev,
                                   long long n_particles, double* out_dev) {
  if (!c || !field_dev || ncomp < 1 || ncomp > 3 || n_particles < 0 || (n_particles > 0 && (!pos_dev || !out_dev)))
    return fail(GBMG_ERR_INVALID_ARG, "mg_cic_read: bad argument");
  DeviceGuard g(c->device);
  if (n_particles == 0) return GBMG_OK;
  k_cic_read<<<particle_blocks(n_particles), 256, 0, c->stream>>>(c->lv[0].d, field_dev, ncomp, pos_dev, n_particles,
                                                                 out_dev);
  note_launch();
  TRY(cudaGetLastError());
  return GBMG_OK;
}

extern "C" gbmg_status mg_force(gbmg_ctx* c, const double* phi_dev, const float* pos_dev, long long n_particles,
                                float* force_out_dev) {
  if (!c || !phi_dev || n_particles < 0 || (n_particles > 0 && (!pos_dev || !force_out_dev)))
    return fail(GBMG_ERR_INVALID_ARG, "mg_force: bad argument");
  DeviceGuard g(c->device);
  const Dims d = c->lv[0].d;
  const long long n = ncell(d);
  if (!c->force_scratch) {
    TRY(cudaMalloc((void**)&c->force_scratch, (size_t)n * 4 * sizeof(float)));
    c->owned.push_back(c->force_scratch);
  }
  float* u = c->force_scratch;
  float* gr = c->force_scratch + n;
  k_phi_to_f32<<<(int)df_partial_count(n), 256, 0, c->stream>>>(n, phi_dev, u);
  note_launch();
  TRY(cudaGetLastError());
  k_force_grid<<<dim3((d.nx + 31) / 32, (d.ny + 7) / 8, d.nz), dim3(32, 8), 0, c->stream>>>(d, u, gr);
  note_launch();
  TRY(cudaGetLastError());
  if (n_particles == 0) return GBMG_OK;
  k_force_read<<<particle_blocks(n_particles), 256, 0, c->stream>>>(d, gr, pos_dev, n_particles, force_out_dev);
  note_launch();
  TRY(cudaGetLastError());
  return GBMG_OK;
}
