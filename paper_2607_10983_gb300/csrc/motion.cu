// Mesh motion (Sec. 4.4): the deformation-rate potential solves the curvilinear
// equation L_psi[psidot] = kappa (m_init - sqrt(g) rho) (Eq. calcdefp) with the same
// operator and solver as the gravitational potential, its source smoothed first;
// then psi <- Z[psi + dtau psidot] with Z removing the mean (Eq. defadvance).
// The paper does not say how the source is smoothed: here by passes of the
// separable [1/4, 1/2, 1/4] filter (the one-axis weights of the full-weighting
// restriction, Appendix B, without decimation).
#include <cstring>
#include <utility>

#include "kernels.h"
#include "solver.h"

namespace gbmg {

namespace {

constexpr int S_MOTION_MEAN = 12;  // device scalar slot of the mean of psi

__global__ void k_motion_source(long long n, const double* __restrict__ rho, const float* __restrict__ J, double kappa,
                                double m_init, double* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = kappa * (m_init - (double)J[i] * rho[i]);
}

// one axis of the binomial filter: (u_{i-1} + u_{i+1}) / 4 + u_i / 2, periodic
__global__ void k_binomial_axis(Dims d, int axis, const double* __restrict__ in, double* __restrict__ out) {
  const long long n = ncell(d);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % d.nx), y = (int)((i / d.nx) % d.ny), z = (int)(i / ((long long)d.nx * d.ny));
    long long m, p;
    if (axis == 0) {
      m = i + (wrap_lo(x - 1, d.nx) - x);
      p = i + (wrap_hi(x + 1, d.nx) - x);
    } else if (axis == 1) {
      m = i + (long long)(wrap_lo(y - 1, d.ny) - y) * d.nx;
      p = i + (long long)(wrap_hi(y + 1, d.ny) - y) * d.nx;
    } else {
      m = i + (long long)(wrap_lo(z - 1, d.nz) - z) * d.nx * d.ny;
      p = i + (long long)(wrap_hi(z + 1, d.nz) - z) * d.nx * d.ny;
    }
    out[i] = 0.25 * (in[m] + in[p]) + 0.5 * in[i];
  }
}

__global__ void k_axpy_inplace(long long n, double* __restrict__ y, double a, const double* __restrict__ x) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = y[i] + a * x[i];
}

}  // namespace

}  // namespace gbmg

using namespace gbmg;

extern "C" gbmg_status mg_mesh_motion(gbmg_ctx* c, const double* rho_dev, double kappa, double m_init,
                                      int smooth_passes, double dtau, double* psi_inout_dev, double* psidot_inout_dev,
                                      double tol, int max_vcycles, gbmg_stats* stats) {
  g_last_error.clear();
  if (!c || !rho_dev || !psi_inout_dev || !psidot_inout_dev || smooth_passes < 0 || !(tol >= 0.0))
    return fail(GBMG_ERR_INVALID_ARG, "mg_mesh_motion: bad argument");
  if (c->o.op != GBMG_OP_CURV19) return fail(GBMG_ERR_INVALID_ARG, "mg_mesh_motion: needs a curvilinear context");
  DeviceGuard g(c->device);
  const Dims d = c->lv[0].d;
  const long long n = ncell(d);
  if (!c->motion) {
    TRY(cudaMalloc((void**)&c->motion, (size_t)n * 2 * sizeof(double)));
    c->owned.push_back(c->motion);
  }
  // geometry of the current mesh (J on every level, coarse operators)
  TRYS(mg_set_geometry(c, psi_inout_dev));
  double* a = c->motion;
  double* b = c->motion + n;
  const int blocks = (int)df_partial_count(n);
  k_motion_source<<<blocks, 256, 0, c->stream>>>(n, rho_dev, c->lv[0].cc.J, kappa, m_init, a);
  note_launch();
  TRY(cudaGetLastError());
  for (int p = 0; p < smooth_passes; ++p)
    for (int axis = 0; axis < 3; ++axis) {
      k_binomial_axis<<<blocks, 256, 0, c->stream>>>(d, axis, a, b);
      note_launch();
      TRY(cudaGetLastError());
      std::swap(a, b);
    }
  // L psidot = source (volume-weighted projection inside the solve), warm-started
  gbmg_stats st;
  std::memset(&st, 0, sizeof(st));
  TRYS(curv_solve(c, a, psidot_inout_dev, tol, max_vcycles, st));
  // psi <- psi + dtau psidot, then remove the mean
  k_axpy_inplace<<<blocks, 256, 0, c->stream>>>(n, psi_inout_dev, dtau, psidot_inout_dev);
  note_launch();
  TRY(cudaGetLastError());
  double* part = c->partials;
  TRY(launch_sum<double>(c->stream, n, psi_inout_dev, part, nullptr));
  TRY(launch_finalize(c->stream, part, df_partial_count(n), c->scal + S_MOTION_MEAN, 1.0 / (double)n));
  TRY(launch_shift<double>(c->stream, n, psi_inout_dev, c->scal + S_MOTION_MEAN, psi_inout_dev));
  TRY(cudaStreamSynchronize(c->stream));
  c->geom_ready = false;  // psi moved: the next curvilinear solve must set the geometry again
  c->geom_from_psi = false;
  c->last = st;
  if (stats) *stats = st;
  return (gbmg_status)st.status;
}
