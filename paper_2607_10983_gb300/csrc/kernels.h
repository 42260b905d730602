// Launch functions of the multigrid kernels (host-callable, internal to the library).
// Each queues one kernel on `st` and returns the launch status.
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace gbmg {

// Counts kernel launches made by this library (process-wide, for measurement).
void note_launch();
void note_launches(long long k);  // k launches at once (graph replays; negative: captured, not run)
long long launch_count();

// Number of per-block partial sums a reduction-producing launch writes for a level.
long long partial_count(Dims d);

// ---- one kernel per operation, T = float or double (flat 7-point operator) ----
template <typename T>
cudaError_t launch_apply(cudaStream_t st, Dims d, const T* u, T* out, T inv_h2);
template <typename T>
cudaError_t launch_residual(cudaStream_t st, Dims d, const T* f, const T* u, T* out, T inv_h2,
                            double* partials_sq);
// Chebyshev step with folded constants a = c2 D^-1, b = a / h^2 (see cheb_step).
template <typename T>
cudaError_t launch_cheb_step(cudaStream_t st, Dims d, const T* r, const T* e_in, T* e_out, T* dvec, T a, T b, T c1);
// Weighted Jacobi with wa = omega D^-1, wb = wa / h^2.
template <typename T>
cudaError_t launch_jacobi(cudaStream_t st, Dims d, const T* r, const T* e_in, T* e_out, T wa, T wb);
// Folded Chebyshev constants of step k on a level of spacing h.
inline void cheb_constants(double c2, double h, double& a, double& b) {
  const double dinv = -(h * h) / 6.0;
  a = c2 * dinv;
  b = a * (1.0 / (h * h));
}
template <typename T>
cudaError_t launch_restrict(cudaStream_t st, Dims fine, const T* f, T* c);
template <typename T>
cudaError_t launch_prolong_add(cudaStream_t st, Dims coarse, const T* c, T* f);
template <typename T>
cudaError_t launch_coarse_matvec(cudaStream_t st, int n, const T* G, const T* r, T* e);

// The bottom of the FP32 Chebyshev V-cycle in one CTA (levels that fit in shared
// memory): levels 0 .. nl-1 of the sub-hierarchy, the last the coarsest (e = G r).
// Bit-identical to the one-kernel-per-operation chain from e = 0 on level 0.
constexpr int kSmallMaxL = 4;               // levels of the sub-hierarchy
constexpr int kSmallCells = 4096;           // cells of its first level at most (16^3)
constexpr int kSmallThreads = 1024;
constexpr size_t kSmallSmem = 200 * 1024;   // shared memory bound (bytes)
struct SmallCycle {
  int nl;
  Dims d[kSmallMaxL];
  float inv_h2[kSmallMaxL];
  float a[kSmallMaxL][16], b[kSmallMaxL][16];  // folded Chebyshev constants per level and step
  float c1[16];
  int degree;
  int nc;           // unknowns of the coarsest level
  const float* G;   // its nc x nc pseudo-inverse (FP32, row-major)
};
size_t small_cycle_smem(const SmallCycle& P);
// e_out = V-cycle(r_in) on level 0 of P (device buffers of level 0's size)
cudaError_t launch_small_vcycle(cudaStream_t st, const SmallCycle& P, const float* r_in, float* e_out);
template <typename T>
cudaError_t launch_sum(cudaStream_t st, long long n, const T* x, double* partials_sum,
                       double* partials_sq);
template <typename T>
cudaError_t launch_shift(cudaStream_t st, long long n, const T* x, const double* shift_dev, T* out);

// e[i] = e[i] rounded to BF16 (mode 1) or FP16 (mode 2), kept as FP32.
cudaError_t launch_round16(cudaStream_t st, long long n, float* e, int mode);
// out[0] = scale * (sum of `count` partials), summed in a fixed order (one block).
cudaError_t launch_finalize(cudaStream_t st, const double* partials, long long count, double* out, double scale);
// n <= 32 doubles from device memory into page-locked host memory (its device address)
cudaError_t launch_scalars_to_host(cudaStream_t st, const double* src, double* dst_mapped, int n);

// ---- double-float path (finest level, h = 1) ----
cudaError_t launch_f64_to_df(cudaStream_t st, long long n, const double* x, float2* out,
                             double* partials_sum);
cudaError_t launch_df_to_f64(cudaStream_t st, long long n, const float2* in, const double* shift_dev,
                             double* out);
cudaError_t launch_df_residual(cudaStream_t st, Dims d, const float2* F, const double* m_dev,
                               const float2* phi, float* r, double* partials_r2,
                               double* partials_f2);
// phi += e (e NULL: phi unchanged); partials_sum (nullable) gets the block sums of phi.
cudaError_t launch_df_update(cudaStream_t st, long long n, float2* phi, const float* e,
                             double* partials_sum);
long long df_partial_count(long long n);

// ---- conjugate-gradient vectors (FP32, device scalars): partials of a . b
// (df_partial_count(n) blocks); e = (first ? 0 : e) + (num/den) p, r -= (num/den) q;
// p = z + (num/den) p
cudaError_t launch_dot_f32(cudaStream_t st, long long n, const float* a, const float* b, double* partials);
cudaError_t launch_pcg_update(cudaStream_t st, long long n, float* e, float* r, const float* p, const float* q,
                              const double* num, const double* den, int first);
cudaError_t launch_pcg_dir(cudaStream_t st, long long n, float* p, const float* z, const double* num,
                           const double* den);

// ---- temporally blocked FP32 level kernels (Chebyshev smoother) ----
bool fused_degree_supported(int degree);
// e = Chebyshev pre-smoothing of A e = r from e = 0; rc = R (r - A e) on the next level.
cudaError_t launch_down_fused(cudaStream_t st, int degree, Dims d, const float* r, float* e, float* rc,
                              double h, const double* c1, const double* c2);
// e_out = Chebyshev post-smoothing of A e = r starting from e_in + P ec.
cudaError_t launch_up_fused(cudaStream_t st, int degree, Dims d, const float* e_in, const float* ec,
                            const float* r, float* e_out, double h, const double* c1, const double* c2);
// Finest level: phi_out = phi_in + e (double-float), r_out = F - m - A phi_out, with block partials
// of ||r_out||^2, sum(phi_out) and (pf2 nullable) ||F - m||^2, df_update_residual_partials(d) each.
// e NULL: no update (phi_out may then be NULL: not written).
long long df_update_residual_partials(Dims d);
cudaError_t launch_df_update_residual(cudaStream_t st, Dims d, const float2* phi_in, const float* e,
                                      const float2* F, const double* m_dev, float2* phi_out, float* r_out,
                                      double* partials_r2, double* partials_sum, double* partials_f2);

// ---- curvilinear operator (moving mesh) ----
// Per-level geometry: J = det A and the packed symmetric B = J A^-2 (xx, yy, zz, xy, xz, yz).
struct CurvCoef {
  const float* J;
  const float* B[6];
  float h2;  // h_l^2
};
struct CurvCoefOut {
  float* J;
  float* B[6];
};
cudaError_t launch_geom(cudaStream_t st, Dims d, const double* psi, double h, CurvCoefOut out);
// Curvilinear operator form: 0 = M (the paper's scheme), 1 = its exact transpose M^T,
// 2 = the symmetric variant S (its own transpose).
// out = op(u) (/ J when divide_J)
template <typename T>
cudaError_t launch_curv_apply(cudaStream_t st, Dims d, CurvCoef cf, const T* u, T* out, int form, int divide_J);
// out = r - op(u) / J; partials (nullable): block sums of out^2
template <typename T>
cudaError_t launch_curv_residual(cudaStream_t st, Dims d, CurvCoef cf, const T* r, const T* u, T* out, int form,
                                 double* partials);
template <typename T>
cudaError_t launch_curv_jacobi(cudaStream_t st, Dims d, CurvCoef cf, const T* r, const T* e_in, T* e_out, int form,
                               T omega);
// dense n x n matrix of op / J on a (small) level, FP64 row-major
// e_out = the weighted-Jacobi sweep of an iterate that is zero (pointwise; FP32)
cudaError_t launch_curv_jacobi_zero(cudaStream_t st, Dims d, CurvCoef cf, const float* r, float* e_out, int form,
                                    float omega);
cudaError_t launch_curv_dense(cudaStream_t st, Dims d, CurvCoef cf, int form, double* out);
// double-float outer residual: r = b - op(u)/J with b = J (src - m) (scale_J) or src
// block partial sums written by launch_curv_df_residual and launch_curv_residual<float>
long long curv_partial_count(Dims d);
cudaError_t launch_curv_df_residual(cudaStream_t st, Dims d, CurvCoef cf, const float2* src, const double* m_dev,
                                    int scale_J, const float2* u, int form, float* r, double* pr2, double* pf2);
// partial sums of x * J and of J (df_partial_count(n) blocks each)
cudaError_t launch_wsum(cudaStream_t st, long long n, const double* x, const float* J, double* pxj, double* pj);
// psi_bar of the curvilinear adjoint on the finest level from the forward solution phi
// (FP64) and the transposed-solve solution lam (double-float); S: 6 n pairs of scratch;
// sym: the operator is the symmetric variant; h a power of two.
cudaError_t launch_psibar(cudaStream_t st, Dims d, const double* psi, const double* phi, const float2* lam,
                          const double* delta, const double* mw_dev, const double* slam_dev, double h, int sym,
                          float2* S, double* out);
// out = J (lam - s) (nullable) and lam64 = lam (nullable), from double-float lam
cudaError_t launch_jscale(cudaStream_t st, long long n, const float2* lam, const float* J, const double* s_dev,
                          double* out, double* lam64);
// out[0] = a[0] / b[0] (0 if b[0] == 0)
cudaError_t launch_ratio(cudaStream_t st, const double* a, const double* b, double* out);

}  // namespace gbmg
