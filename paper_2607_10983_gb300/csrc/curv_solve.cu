// Curvilinear (moving-mesh) solve and the adjoint solves.
//
// Geometry (Sec. 4.2, Appendix B): psi is restricted to every level by full
// weighting and the triad, volume element and B = sqrt(g) g^-1 are rebuilt there;
// the coarsest level's operator is inverted exactly (pseudo-inverse).
// Solve (Sec. 4.3): L phi = f with L = M / J, f = delta - sum(delta J)/sum(J)
// (Eq. solvability), weighted-Jacobi V-cycles in FP32 inside a double-float
// defect correction, gauge: mean of phi removed.
// Adjoint (Sec. 4.8, Eq. adj_rhs / adj_op, written with the exact transpose):
// M^T lam = phi_bar - mean(phi_bar) by the same V-cycle on M^T / J,
// delta_bar = J (lam - sum(J lam)/sum(J)), psi_bar through the geometry.
// With the symmetric variant (opts.curv_sym) both solves use S, its own transpose.
#include <cstring>
#include <vector>

#include "kernels.h"
#include "solver.h"

using namespace gbmg;

namespace {

enum CurvScal { S_SUMJ = 6, S_MW = 9, S_SLAM = 10 };

// operator form of the forward (tr false) or transposed (tr true) problem: 0 = M, 1 = M^T, 2 = S
int curv_form(const gbmg_ctx* c, bool tr) { return c->o.curv_sym ? 2 : (tr ? 1 : 0); }

template <typename T>
const T* curv_G(const gbmg_ctx* c, bool tr);
template <>
const float* curv_G<float>(const gbmg_ctx* c, bool tr) { return tr ? c->G32T : c->G32; }
template <>
const double* curv_G<double>(const gbmg_ctx* c, bool tr) { return tr ? c->G64T : c->G64; }

// nu weighted-Jacobi sweeps; from_zero: the iterate is zero, so the first sweep is the
// pointwise one (no read of e; the same values as a full sweep of zeros)
template <typename T>
gbmg_status curv_smooth(gbmg_ctx* c, int l, T*& e, T*& eo, const T* r, int nu, bool tr, bool from_zero) {
  const Level& L = c->lv[l];
  for (int k = 0; k < nu; ++k) {
    if (k == 0 && from_zero) {
      if constexpr (sizeof(T) == 4) {
        TRY(launch_curv_jacobi_zero(c->stream, L.d, L.cc, r, eo, curv_form(c, tr), (float)c->o.omega));
        std::swap(e, eo);
        continue;
      }
    }
    ProfScope ps(c, l == 0 ? GBMG_PROF_CURV0 : GBMG_PROF_OFF);
    TRY(launch_curv_jacobi<T>(c->stream, L.d, L.cc, r, e, eo, curv_form(c, tr), (T)c->o.omega));
    std::swap(e, eo);
  }
  return GBMG_OK;
}

// Curvilinear V-cycle for L_l e = r (or the transposed-solve operator), one kernel
// per operation (Sec. 4.3, Eq. curv_error; Appendix B), from e = 0: the iterate's
// content is not read when nu1 > 0 (the first sweep is the pointwise one), and must be
// zero otherwise.
template <typename T>
gbmg_status vcycle_curv(gbmg_ctx* c, int l, T*& e, T*& eo, const T* r, bool tr) {
  const Level& L = c->lv[l];
  if (l == c->L - 1) {
    TRY(launch_coarse_matvec<T>(c->stream, c->nc, curv_G<T>(c, tr), r, e));
    return GBMG_OK;
  }
  TRYS(curv_smooth<T>(c, l, e, eo, r, c->o.nu1, tr, true));
  TRY(launch_curv_residual<T>(c->stream, L.d, L.cc, r, e, (T*)L.t, curv_form(c, tr), nullptr));
  const Level& C = c->lv[l + 1];
  TRY(launch_restrict<T>(c->stream, L.d, (const T*)L.t, (T*)C.r));
  T* ce = (T*)C.e;
  T* ceo = (T*)C.e2;
  if (l + 1 < c->L - 1 && c->o.nu1 == 0) TRY(cudaMemsetAsync(ce, 0, (size_t)ncell(C.d) * sizeof(T), c->stream));
  TRYS(vcycle_curv<T>(c, l + 1, ce, ceo, (const T*)C.r, tr));
  TRY(launch_prolong_add<T>(c->stream, C.d, ce, e));
  TRYS(curv_smooth<T>(c, l, e, eo, r, c->o.nu2, tr, false));
  return GBMG_OK;
}

// Mixed-precision solve of L u = f (forward, f = src - weighted mean) or of the
// transposed problem M^T u = src - mean(src) (tr).  u_in NULL starts from zero;
// u_out NULL leaves the result in c->phi_df only.
// One cycle of the curvilinear solve on c->stream: FP32 V-cycle on r0, phi += e in
// double-float, r0 = the double-float residual and its norm, the scalars copied to pinned
// host memory.  Its launches depend only on the context and the orientation, so after a
// cycle has run eagerly it is captured once as a CUDA graph per orientation and replayed
// (the coefficients change in place; timed families are timed by event nodes).
gbmg_status curv_cycle(gbmg_ctx* c, bool tr, float* r0) {
  const Level& L0 = c->lv[0];
  const long long n = ncell(L0.d);
  double* sc = c->scal;
  float* e = (float*)L0.e;
  float* eo = (float*)L0.e2;
  if (c->o.nu1 == 0) TRY(cudaMemsetAsync(e, 0, (size_t)n * sizeof(float), c->stream));
  TRYS(vcycle_curv<float>(c, 0, e, eo, r0, tr));
  TRY(launch_df_update(c->stream, n, c->phi_df, e, nullptr));
  {
    ProfScope ps(c, GBMG_PROF_DF0);
    TRY(launch_curv_df_residual(c->stream, L0.d, L0.cc, c->F_df, sc + S_MEAN_F, tr ? 0 : 1, c->phi_df, curv_form(c, tr),
                                r0, c->partials, nullptr));
  }
  TRY(launch_finalize(c->stream, c->partials, curv_partial_count(L0.d), sc + S_R2, 1.0));
  TRY(launch_scalars_to_host(c->stream, c->scal, c->host_scal_dev, 8));
  return GBMG_OK;
}

gbmg_status curv_solve_impl(gbmg_ctx* c, const double* src, const double* u_in, double* u_out, double tol, int maxv,
                            gbmg_stats& st, bool tr) {
  const Level& L0 = c->lv[0];
  const long long n = ncell(L0.d);
  double* part = c->partials;
  double* part1 = c->partials + c->npart;
  double* part2 = c->partials + 2 * c->npart;
  double* sc = c->scal;
  const long long pr = df_partial_count(n), pc = curv_partial_count(L0.d);
  TRY(launch_f64_to_df(c->stream, n, src, c->F_df, part));
  if (!tr) {
    TRY(launch_wsum(c->stream, n, src, L0.cc.J, part, part1));
    TRY(launch_finalize(c->stream, part, pr, sc + S_SUM_F, 1.0));
    TRY(launch_finalize(c->stream, part1, pr, sc + S_SUMJ, 1.0));
    TRY(launch_ratio(c->stream, sc + S_SUM_F, sc + S_SUMJ, sc + S_MEAN_F));
  } else {
    TRY(launch_finalize(c->stream, part, pr, sc + S_MEAN_F, 1.0 / (double)n));
  }
  if (u_in) {
    TRY(launch_f64_to_df(c->stream, n, u_in, c->phi_df, nullptr));
  } else {
    TRY(cudaMemsetAsync(c->phi_df, 0, (size_t)n * sizeof(float2), c->stream));
  }
  float* r0 = (float*)L0.r;
  const int itr = curv_form(c, tr);
  TRY(launch_curv_df_residual(c->stream, L0.d, L0.cc, c->F_df, sc + S_MEAN_F, tr ? 0 : 1, c->phi_df, itr, r0, part,
                              part1));
  TRY(launch_finalize(c->stream, part, pc, sc + S_R2, 1.0));
  TRY(launch_finalize(c->stream, part1, pc, sc + S_F2, 1.0));
  double rel = 0.0;
  TRYS(read_rel(c, rel));
  Monitor mon(st, tol, maxv);
  mon.start(rel);
  const int k = tr ? 1 : 0;
  while (!mon.done()) {
    sync_graph_mask(c);
    const bool graphs = c->curv_warm[k] && !c->cyc_off;
    if (graphs && !c->curv_exec[k])
      TRYS(capture_graph(c, 2 + k, [&]() { return curv_cycle(c, tr, r0); }, c->curv_exec[k], c->curv_kernels[k]));
    const bool replay = graphs && c->curv_exec[k];
    if (replay) {
      TRY(cudaGraphLaunch(c->curv_exec[k], c->stream));
      note_launches(c->curv_kernels[k]);
    } else {
      TRYS(curv_cycle(c, tr, r0));
      c->curv_warm[k] = true;
    }
    TRYS(rel_from_host(c, rel));
    if (replay) gprof_collect(c, 2 + k);
    if (mon.record(rel)) break;
  }
  if (u_out) {
    TRY(launch_df_update(c->stream, n, c->phi_df, nullptr, part2));
    TRY(launch_finalize(c->stream, part2, pr, sc + S_MEAN_PHI, 1.0 / (double)n));
    TRY(launch_df_to_f64(c->stream, n, c->phi_df, sc + S_MEAN_PHI, u_out));
  }
  return GBMG_OK;
}

gbmg_status ensure_adjoint_scratch(gbmg_ctx* c) {
  const long long n = ncell(c->lv[0].d);
  if (!c->adj_lam) {
    TRY(cudaMalloc((void**)&c->adj_lam, (size_t)n * sizeof(double)));
    c->owned.push_back(c->adj_lam);
  }
  if (!c->adj_S) {
    TRY(cudaMalloc((void**)&c->adj_S, (size_t)n * 6 * sizeof(double)));
    c->owned.push_back(c->adj_S);
  }
  return GBMG_OK;
}

}  // namespace

gbmg_status gbmg::curv_solve(gbmg_ctx* c, const double* F, double* phi, double tol, int maxv, gbmg_stats& st) {
  return curv_solve_impl(c, F, phi, phi, tol, maxv, st, false);
}

namespace {

// Exact inverses of the coarsest operator and of its transposed-solve twin (minimum-norm,
// left null vector J), built from the coarsest level's coefficients.  Waits for the stream.
gbmg_status build_coarsest(gbmg_ctx* c, const char* who) {
  const Level& C = c->lv[c->L - 1];
  const int nc = c->nc;
  std::vector<float> Jc(nc);
  TRY(cudaMemcpyAsync(Jc.data(), C.cc.J, (size_t)nc * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
  std::vector<double> Lm((size_t)nc * nc), G;
  for (int tr = 0; tr < 2; ++tr) {
    TRY(launch_curv_dense(c->stream, C.d, C.cc, curv_form(c, tr != 0), c->dense));
    TRY(cudaMemcpyAsync(Lm.data(), c->dense, Lm.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    TRY(cudaStreamSynchronize(c->stream));
    std::vector<double> w(Jc.begin(), Jc.end());
    for (float v : Jc)
      if (!(v > 0.f)) return fail(GBMG_ERR_INVALID_ARG, std::string(who) + ": non-positive volume element on the coarsest level");
    if (!dense_pinv(nc, Lm, w, G)) return fail(GBMG_ERR_INVALID_ARG, std::string(who) + ": coarsest operator is singular");
    std::vector<float> G32(G.begin(), G.end());
    TRY(cudaMemcpy(tr ? c->G64T : c->G64, G.data(), G.size() * sizeof(double), cudaMemcpyHostToDevice));
    TRY(cudaMemcpy(tr ? c->G32T : c->G32, G32.data(), G32.size() * sizeof(float), cudaMemcpyHostToDevice));
  }
  return GBMG_OK;
}

}  // namespace

extern "C" gbmg_status mg_set_geometry(gbmg_ctx* c, const double* psi_dev) {
  if (!c || !psi_dev) return fail(GBMG_ERR_INVALID_ARG, "mg_set_geometry: NULL argument");
  if (c->o.op != GBMG_OP_CURV19) return fail(GBMG_ERR_STATE, "mg_set_geometry: context is not curvilinear");
  DeviceGuard g(c->device);
  c->geom_ready = false;
  for (int l = 0; l < c->L; ++l) {
    Level& L = c->lv[l];
    if (l == 0) {
      TRY(cudaMemcpyAsync(L.psi, psi_dev, (size_t)ncell(L.d) * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    } else {
      TRY(launch_restrict<double>(c->stream, c->lv[l - 1].d, c->lv[l - 1].psi, L.psi));
    }
    CurvCoefOut o;
    o.J = (float*)L.cc.J;
    for (int k = 0; k < 6; ++k) o.B[k] = (float*)L.cc.B[k];
    TRY(launch_geom(c->stream, L.d, L.psi, L.h, o));
  }
  TRYS(build_coarsest(c, "mg_set_geometry"));
  c->geom_ready = true;
  c->geom_from_psi = true;
  return GBMG_OK;
}

extern "C" gbmg_status mg_set_coefficients(gbmg_ctx* c, const float* J_dev, const float* B_dev) {
  if (!c || !J_dev || !B_dev) return fail(GBMG_ERR_INVALID_ARG, "mg_set_coefficients: NULL argument");
  if (c->o.op != GBMG_OP_CURV19) return fail(GBMG_ERR_STATE, "mg_set_coefficients: context is not curvilinear");
  DeviceGuard g(c->device);
  c->geom_ready = false;
  c->geom_from_psi = false;
  const size_t b0 = (size_t)ncell(c->lv[0].d) * sizeof(float);
  for (int l = 0; l < c->L; ++l) {
    Level& L = c->lv[l];
    if (l == 0) {
      TRY(cudaMemcpyAsync((float*)L.cc.J, J_dev, b0, cudaMemcpyDeviceToDevice, c->stream));
      for (int k = 0; k < 6; ++k)
        TRY(cudaMemcpyAsync((float*)L.cc.B[k], (const char*)B_dev + k * b0, b0, cudaMemcpyDeviceToDevice, c->stream));
    } else {
      // coarse coefficients: full-weighting restriction of the finer level's coefficients
      const Level& F = c->lv[l - 1];
      TRY(launch_restrict<float>(c->stream, F.d, F.cc.J, (float*)L.cc.J));
      for (int k = 0; k < 6; ++k) TRY(launch_restrict<float>(c->stream, F.d, F.cc.B[k], (float*)L.cc.B[k]));
    }
  }
  TRYS(build_coarsest(c, "mg_set_coefficients"));
  c->geom_ready = true;
  return GBMG_OK;
}

extern "C" gbmg_status mg_solve_adjoint(gbmg_ctx* c, const double* phi_bar_dev, double* source_bar_dev,
                                        double* psi_bar_dev, const double* phi_dev, const double* source_dev,
                                        double tol, int max_vcycles, gbmg_stats* stats) {
  g_last_error.clear();
  if (!c || !phi_bar_dev || !source_bar_dev) return fail(GBMG_ERR_INVALID_ARG, "mg_solve_adjoint: NULL argument");
  if (!(tol >= 0.0)) return fail(GBMG_ERR_INVALID_ARG, "mg_solve_adjoint: tol must be >= 0");
  DeviceGuard g(c->device);
  const Level& L0 = c->lv[0];
  const long long n = ncell(L0.d);
  if (c->o.op == GBMG_OP_FLAT7) {
    // A is symmetric: source_bar = P A^+ P phi_bar is the same solve on the cotangent
    if (psi_bar_dev) return fail(GBMG_ERR_INVALID_ARG, "mg_solve_adjoint: psi_bar is only defined for the curvilinear operator");
    TRY(cudaMemsetAsync(source_bar_dev, 0, (size_t)n * sizeof(double), c->stream));
    return mg_solve(c, phi_bar_dev, nullptr, source_bar_dev, tol, max_vcycles, stats);
  }
  if (!c->geom_ready) return fail(GBMG_ERR_STATE, "mg_solve_adjoint: no geometry set");
  if (psi_bar_dev && (!phi_dev || !source_dev))
    return fail(GBMG_ERR_INVALID_ARG, "mg_solve_adjoint: psi_bar needs the forward solution and source");
  if (psi_bar_dev && !c->geom_from_psi)
    return fail(GBMG_ERR_STATE, "mg_solve_adjoint: psi_bar needs a geometry set from psi, not raw coefficients");
  TRYS(ensure_adjoint_scratch(c));
  gbmg_stats st;
  std::memset(&st, 0, sizeof(st));
  TRYS(curv_solve_impl(c, phi_bar_dev, nullptr, nullptr, tol, max_vcycles, st, true));
  double* part = c->partials;
  double* part1 = c->partials + c->npart;
  double* sc = c->scal;
  const long long pr = df_partial_count(n);
  // lam in FP64, s_lam = sum(J lam) / sum(J), delta_bar = J (lam - s_lam)
  TRY(launch_jscale(c->stream, n, c->phi_df, L0.cc.J, nullptr, nullptr, c->adj_lam));
  TRY(launch_wsum(c->stream, n, c->adj_lam, L0.cc.J, part, part1));
  TRY(launch_finalize(c->stream, part, pr, sc + S_SUM_F, 1.0));
  TRY(launch_finalize(c->stream, part1, pr, sc + S_SUMJ, 1.0));
  TRY(launch_ratio(c->stream, sc + S_SUM_F, sc + S_SUMJ, sc + S_SLAM));
  TRY(launch_jscale(c->stream, n, c->phi_df, L0.cc.J, sc + S_SLAM, source_bar_dev, nullptr));
  if (psi_bar_dev) {
    TRY(launch_wsum(c->stream, n, source_dev, L0.cc.J, part, part1));
    TRY(launch_finalize(c->stream, part, pr, sc + S_SUM_F, 1.0));
    TRY(launch_finalize(c->stream, part1, pr, sc + S_SUMJ, 1.0));
    TRY(launch_ratio(c->stream, sc + S_SUM_F, sc + S_SUMJ, sc + S_MW));
    TRY(launch_psibar(c->stream, L0.d, L0.psi, phi_dev, c->phi_df, source_dev, sc + S_MW, sc + S_SLAM, L0.h,
                      c->o.curv_sym, (float2*)c->adj_S, psi_bar_dev));
  }
  TRY(cudaStreamSynchronize(c->stream));
  c->last = st;
  if (stats) *stats = st;
  return (gbmg_status)st.status;
}

// ------------------------------------------------------------------ components

extern "C" gbmg_status mg_curv_apply(gbmg_ctx* c, int level, int dtype, int transpose, int divide_by_J,
                                     const void* u, void* out) {
  if (!c || !u || !out || level < 0 || level >= c->L || (dtype != GBMG_F32 && dtype != GBMG_F64))
    return fail(GBMG_ERR_INVALID_ARG, "mg_curv_apply: bad argument");
  if (c->o.op != GBMG_OP_CURV19 || !c->geom_ready) return fail(GBMG_ERR_STATE, "mg_curv_apply: no geometry set");
  DeviceGuard g(c->device);
  const Level& L = c->lv[level];
  if (dtype == GBMG_F64)
    TRY(launch_curv_apply<double>(c->stream, L.d, L.cc, (const double*)u, (double*)out, curv_form(c, transpose != 0), divide_by_J ? 1 : 0));
  else
    TRY(launch_curv_apply<float>(c->stream, L.d, L.cc, (const float*)u, (float*)out, curv_form(c, transpose != 0), divide_by_J ? 1 : 0));
  return GBMG_OK;
}

// FP32 tiled kernels of the V-cycle's levels, one launch each (for tests and composition).
static gbmg_status curv_component_check(gbmg_ctx* c, int level, const void* a, const void* b, const void* o,
                                        const char* who) {
  if (!c || !a || !b || !o || level < 0 || level >= c->L) return fail(GBMG_ERR_INVALID_ARG, std::string(who) + ": bad argument");
  if (c->o.op != GBMG_OP_CURV19 || !c->geom_ready) return fail(GBMG_ERR_STATE, std::string(who) + ": no geometry set");
  return GBMG_OK;
}

extern "C" gbmg_status mg_curv_residual(gbmg_ctx* c, int level, int transpose, const float* r, const float* u,
                                        float* out) {
  TRYS(curv_component_check(c, level, r, u, out, "mg_curv_residual"));
  DeviceGuard g(c->device);
  const Level& L = c->lv[level];
  TRY(launch_curv_residual<float>(c->stream, L.d, L.cc, r, u, out, curv_form(c, transpose != 0), nullptr));
  return GBMG_OK;
}

extern "C" gbmg_status mg_curv_smooth(gbmg_ctx* c, int level, int transpose, const float* e_in, const float* r,
                                      float* e_out) {
  TRYS(curv_component_check(c, level, r, r, e_out, "mg_curv_smooth"));
  if (e_in == e_out) return fail(GBMG_ERR_INVALID_ARG, "mg_curv_smooth: e_in and e_out must differ");
  DeviceGuard g(c->device);
  const Level& L = c->lv[level];
  const int form = curv_form(c, transpose != 0);
  if (e_in) TRY(launch_curv_jacobi<float>(c->stream, L.d, L.cc, r, e_in, e_out, form, (float)c->o.omega));
  else TRY(launch_curv_jacobi_zero(c->stream, L.d, L.cc, r, e_out, form, (float)c->o.omega));
  return GBMG_OK;
}

extern "C" gbmg_status mg_curv_geometry(gbmg_ctx* c, int level, float* J_out, float* B_out) {
  if (!c || level < 0 || level >= c->L) return fail(GBMG_ERR_INVALID_ARG, "mg_curv_geometry: bad argument");
  if (c->o.op != GBMG_OP_CURV19 || !c->geom_ready) return fail(GBMG_ERR_STATE, "mg_curv_geometry: no geometry set");
  DeviceGuard g(c->device);
  const Level& L = c->lv[level];
  const size_t b = (size_t)ncell(L.d) * sizeof(float);
  if (J_out) TRY(cudaMemcpyAsync(J_out, L.cc.J, b, cudaMemcpyDeviceToDevice, c->stream));
  if (B_out)
    for (int k = 0; k < 6; ++k)
      TRY(cudaMemcpyAsync((char*)B_out + k * b, L.cc.B[k], b, cudaMemcpyDeviceToDevice, c->stream));
  return GBMG_OK;
}

extern "C" gbmg_status mg_curv_vcycle(gbmg_ctx* c, int transpose, const float* r, float* e_out) {
  if (!c || !r || !e_out) return fail(GBMG_ERR_INVALID_ARG, "mg_curv_vcycle: NULL argument");
  if (c->o.op != GBMG_OP_CURV19 || !c->geom_ready) return fail(GBMG_ERR_STATE, "mg_curv_vcycle: no geometry set");
  DeviceGuard g(c->device);
  const Level& L0 = c->lv[0];
  const long long n = ncell(L0.d);
  float* e = (float*)L0.e;
  float* eo = (float*)L0.e2;
  TRY(cudaMemsetAsync(e, 0, (size_t)n * 4, c->stream));
  TRYS(vcycle_curv<float>(c, 0, e, eo, r, transpose != 0));
  TRY(cudaMemcpyAsync(e_out, e, (size_t)n * 4, cudaMemcpyDeviceToDevice, c->stream));
  return GBMG_OK;
}
