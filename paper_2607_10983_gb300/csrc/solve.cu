// V-cycle level loop, solve drivers and the component entry points of the C ABI.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "kernels.h"
#include "solver.h"

using namespace gbmg;

namespace {

template <typename T>
const T* coarse_G(const gbmg_ctx* c);
template <>
const float* coarse_G<float>(const gbmg_ctx* c) { return c->G32; }
template <>
const double* coarse_G<double>(const gbmg_ctx* c) { return c->G64; }

// One smoothing pass on level l (pre: nu1 Jacobi sweeps, post: nu2), one kernel per
// step, ping-ponging e and eo.
template <typename T>
gbmg_status smooth_pass(gbmg_ctx* c, int l, T*& e, T*& eo, const T* r, T* dv, bool post) {
  const Level& L = c->lv[l];
  if (c->o.smoother == GBMG_SMOOTH_CHEBYSHEV) {
    for (int k = 0; k < c->o.degree; ++k) {
      ProfScope ps(c, l == 0 ? GBMG_PROF_SMOOTH0 : GBMG_PROF_OFF);
      double a, b;
      cheb_constants(c->cc2[k], L.h, a, b);
      TRY(launch_cheb_step<T>(c->stream, L.d, r, e, eo, dv, (T)a, (T)b, (T)c->cc1[k]));
      std::swap(e, eo);
    }
  } else {
    const int nu = post ? c->o.nu2 : c->o.nu1;
    const double wa = c->o.omega * (-(L.h * L.h) / 6.0);
    const double wb = wa * (1.0 / (L.h * L.h));
    for (int k = 0; k < nu; ++k) {
      TRY(launch_jacobi<T>(c->stream, L.d, r, e, eo, (T)wa, (T)wb));
      std::swap(e, eo);
    }
  }
  return GBMG_OK;
}

// With the fused path on, the levels from l down, when they fit in shared memory, run
// as one single-CTA kernel (bit-identical to the chain below).
bool small_cycle_from(const gbmg_ctx* c, int l, SmallCycle* out) {
  return c->o.fused && small_cycle_params(c, l, out);
}

}  // namespace

// Parameters of the single-CTA bottom cycle from level l of c's hierarchy, when the
// Chebyshev smoother runs and levels l .. L-1 fit (false otherwise).
bool gbmg::small_cycle_params(const gbmg_ctx* c, int l, SmallCycle* out) {
  if (c->o.smoother != GBMG_SMOOTH_CHEBYSHEV || c->o.degree > 16) return false;
  const int nl = c->L - l;
  if (nl < 2 || nl > kSmallMaxL || ncell(c->lv[l].d) > kSmallCells) return false;
  SmallCycle P{};
  P.nl = nl;
  P.degree = c->o.degree;
  for (int k = 0; k < c->o.degree; ++k) P.c1[k] = (float)c->cc1[k];
  for (int i = 0; i < nl; ++i) {
    const Level& L = c->lv[l + i];
    P.d[i] = L.d;
    P.inv_h2[i] = (float)(1.0 / (L.h * L.h));
    for (int k = 0; k < c->o.degree; ++k) {
      double a, b;
      cheb_constants(c->cc2[k], L.h, a, b);
      P.a[i][k] = (float)a;
      P.b[i][k] = (float)b;
    }
  }
  P.nc = c->nc;
  P.G = c->G32;
  if (small_cycle_smem(P) > kSmallSmem) return false;
  if (out) *out = P;
  return true;
}

namespace {

// With opts.coarse_store, the correction of a level with fewer than 128^3 cells is held
// in BF16 or FP16 from the moment it is handed up to the next finer level.
constexpr long long kCoarseStoreCells = 128ll * 128 * 128;
gbmg_status store_coarse_correction(gbmg_ctx* c, int l, float* e) {
  if (!c->o.coarse_store || ncell(c->lv[l].d) >= kCoarseStoreCells) return GBMG_OK;
  TRY(launch_round16(c->stream, ncell(c->lv[l].d), e, c->o.coarse_store));
  return GBMG_OK;
}

// V-cycle (Sec. 2.3) on level l for A_l e = r, one kernel per operation.  e / eo are
// the level's ping-pong buffers; on return e points at the result.
template <typename T>
gbmg_status vcycle_unfused(gbmg_ctx* c, int l, T*& e, T*& eo, const T* r) {
  const Level& L = c->lv[l];
  if (l == c->L - 1) {
    TRY(launch_coarse_matvec<T>(c->stream, c->nc, coarse_G<T>(c), r, e));
    return GBMG_OK;
  }
  if constexpr (sizeof(T) == 4) {
    SmallCycle P;
    if (small_cycle_from(c, l, &P)) {
      TRY(launch_small_vcycle(c->stream, P, r, e));
      return GBMG_OK;
    }
  }
  T* dv = (T*)L.dv;
  TRYS(smooth_pass<T>(c, l, e, eo, r, dv, false));
  const T inv_h2 = (T)(1.0 / (L.h * L.h));
  TRY(launch_residual<T>(c->stream, L.d, r, e, (T*)L.t, inv_h2, nullptr));
  const Level& C = c->lv[l + 1];
  TRY(launch_restrict<T>(c->stream, L.d, (const T*)L.t, (T*)C.r));
  T* ce = (T*)C.e;
  T* ceo = (T*)C.e2;
  if (l + 1 < c->L - 1 && !(sizeof(T) == 4 && small_cycle_from(c, l + 1, nullptr)))
    TRY(cudaMemsetAsync(ce, 0, (size_t)ncell(C.d) * sizeof(T), c->stream));
  TRYS(vcycle_unfused<T>(c, l + 1, ce, ceo, (const T*)C.r));
  if constexpr (sizeof(T) == 4) TRYS(store_coarse_correction(c, l + 1, (float*)ce));
  TRY(launch_prolong_add<T>(c->stream, C.d, ce, e));
  TRYS(smooth_pass<T>(c, l, e, eo, r, dv, true));
  return GBMG_OK;
}

// Levels of at least 2^18 cells (64^3) use the temporally blocked kernels; below
// that a level visit is latency-bound and the one-kernel-per-operation chain is as
// fast.  Measured on the 512^3 / 256^3 warm sequences: thresholds 2^23 / 2^21 / 2^18
// gave 64.0 / 65.3 / 65.3 and 280 / 303 / 309 solves/s.
constexpr long long kFusedMinCells = 1ll << 18;
bool level_fused(const gbmg_ctx* c, int l) {
  const Dims d = c->lv[l].d;
  return c->o.fused && l < c->L - 1 && d.nx >= 16 && d.ny >= 16 && d.nz >= 16 &&
         (ncell(d) >= kFusedMinCells || c->fused_all);
}

// V-cycle in FP32 with the temporally blocked kernels on large levels (one launch per
// level visit on each leg) and the one-kernel-per-operation path below them.  e
// receives the pointer to the level's correction.
gbmg_status vcycle_fused(gbmg_ctx* c, int l, float*& e, const float* r) {
  const Level& L = c->lv[l];
  if (!level_fused(c, l)) {
    float* ee = (float*)L.e;
    float* eo = (float*)L.e2;
    if (l < c->L - 1 && !small_cycle_from(c, l, nullptr))
      TRY(cudaMemsetAsync(ee, 0, (size_t)ncell(L.d) * sizeof(float), c->stream));
    TRYS(vcycle_unfused<float>(c, l, ee, eo, r));
    e = ee;
    return GBMG_OK;
  }
  const Level& C = c->lv[l + 1];
  {
    ProfScope ps(c, l == 0 ? GBMG_PROF_DOWN0 : GBMG_PROF_OFF);
    TRY(launch_down_fused(c->stream, c->o.degree, L.d, r, (float*)L.e, (float*)C.r, L.h, c->cc1.data(),
                          c->cc2.data()));
  }
  float* ce = nullptr;
  TRYS(vcycle_fused(c, l + 1, ce, (const float*)C.r));
  TRYS(store_coarse_correction(c, l + 1, ce));
  {
    ProfScope ps(c, l == 0 ? GBMG_PROF_UP0 : GBMG_PROF_OFF);
    TRY(launch_up_fused(c->stream, c->o.degree, L.d, (const float*)L.e, ce, r, (float*)L.e2, L.h,
                        c->cc1.data(), c->cc2.data()));
  }
  e = (float*)L.e2;
  return GBMG_OK;
}

// Device scalar slots of the conjugate-gradient correction.
enum PcgScal { S_RZ = 16, S_RZ_NEW = 17, S_PQ = 18 };

// k = c->o.krylov steps of conjugate gradients for the finest FP32 error equation
// A e = r, preconditioned by one V-cycle from zero (Sec. 3.2).  A and the V-cycle are
// both negative definite on zero-mean fields, so these are the iterates of CG on -A
// with the preconditioner -M.  r is overwritten by the inner residual; e receives the
// pointer to the correction.
gbmg_status pcg_correction(gbmg_ctx* c, float* r, float*& e_out) {
  const Level& L0 = c->lv[0];
  const long long n = ncell(L0.d);
  if (!c->pcg) {
    TRY(cudaMalloc((void**)&c->pcg, (size_t)n * 3 * sizeof(float)));
    c->owned.push_back(c->pcg);
  }
  float* E = c->pcg;
  float* P = c->pcg + n;
  float* Q = c->pcg + 2 * n;
  double* part = c->partials;
  double* sc = c->scal;
  const long long pr = df_partial_count(n);
  // z = M r: one V-cycle from zero (fused legs where the level is large enough)
  auto precond = [&](float*& z) -> gbmg_status {
    if (c->o.fused) return vcycle_fused(c, 0, z, r);
    float* e = (float*)L0.e;
    float* eo = (float*)L0.e2;
    TRY(cudaMemsetAsync(e, 0, (size_t)n * sizeof(float), c->stream));
    TRYS(vcycle_unfused<float>(c, 0, e, eo, r));
    z = e;
    return GBMG_OK;
  };
  float* z = nullptr;
  TRYS(precond(z));
  TRY(cudaMemcpyAsync(P, z, (size_t)n * sizeof(float), cudaMemcpyDeviceToDevice, c->stream));
  TRY(launch_dot_f32(c->stream, n, r, z, part));
  TRY(launch_finalize(c->stream, part, pr, sc + S_RZ, 1.0));
  const int k = c->o.krylov;
  for (int j = 0; j < k; ++j) {
    TRY(launch_apply<float>(c->stream, L0.d, P, Q, 1.0f));
    TRY(launch_dot_f32(c->stream, n, P, Q, part));
    TRY(launch_finalize(c->stream, part, pr, sc + S_PQ, 1.0));
    TRY(launch_pcg_update(c->stream, n, E, r, P, Q, sc + S_RZ, sc + S_PQ, j == 0 ? 1 : 0));
    if (j == k - 1) break;
    TRYS(precond(z));
    TRY(launch_dot_f32(c->stream, n, r, z, part));
    TRY(launch_finalize(c->stream, part, pr, sc + S_RZ_NEW, 1.0));
    TRY(launch_pcg_dir(c->stream, n, P, z, sc + S_RZ_NEW, sc + S_RZ));
    TRY(cudaMemcpyAsync(sc + S_RZ, sc + S_RZ_NEW, sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  }
  e_out = E;
  return GBMG_OK;
}

gbmg_status solve_fp64(gbmg_ctx* c, const double* F, double* phi, double tol, int maxv, gbmg_stats& st) {
  const Level& L0 = c->lv[0];
  const long long n = ncell(L0.d);
  double* part = c->partials;
  double* sc = c->scal;
  const long long pr = df_partial_count(n);
  TRY(launch_sum<double>(c->stream, n, F, part, nullptr));
  TRY(launch_finalize(c->stream, part, pr, sc + S_MEAN_F, 1.0 / (double)n));
  double* f0 = (double*)L0.r;
  TRY(launch_shift<double>(c->stream, n, F, sc + S_MEAN_F, f0));
  TRY(launch_sum<double>(c->stream, n, f0, nullptr, part));
  TRY(launch_finalize(c->stream, part, pr, sc + S_F2, 1.0));
  double* u = (double*)L0.e;
  double* uo = (double*)L0.e2;
  TRY(cudaMemcpyAsync(u, phi, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  auto resnorm = [&]() -> gbmg_status {
    TRY(launch_residual<double>(c->stream, L0.d, f0, u, (double*)L0.t, 1.0, part));
    TRY(launch_finalize(c->stream, part, partial_count(L0.d), sc + S_R2, 1.0));
    return GBMG_OK;
  };
  TRYS(resnorm());
  double rel = 0.0;
  TRYS(read_rel(c, rel));
  Monitor mon(st, tol, maxv);
  mon.start(rel);
  while (!mon.done()) {
    TRYS(vcycle_unfused<double>(c, 0, u, uo, f0));
    TRYS(resnorm());
    TRYS(read_rel(c, rel));
    if (mon.record(rel)) break;
  }
  TRY(launch_sum<double>(c->stream, n, u, part, nullptr));
  TRY(launch_finalize(c->stream, part, pr, sc + S_MEAN_PHI, 1.0 / (double)n));
  TRY(launch_shift<double>(c->stream, n, u, sc + S_MEAN_PHI, phi));
  return GBMG_OK;
}

// One cycle of the fused mixed solve on c->stream: the correction e of r0 (a V-cycle from
// zero, or the preconditioned CG steps of krylov, which overwrite r0), phi_nxt = phi_cur +
// e and r_nxt = F - m - A phi_nxt in double-float with their norms, and the scalars copied
// to pinned host memory (read after the stream is synchronised).
gbmg_status fused_cycle(gbmg_ctx* c, const float2* phi_cur, float2* phi_nxt, float* r0, float* r_nxt) {
  const Level& L0 = c->lv[0];
  double* sc = c->scal;
  double* part = c->partials;
  double* part2 = c->partials + 2 * c->npart;
  float* e = nullptr;
  if (c->o.krylov) TRYS(pcg_correction(c, r0, e));
  else TRYS(vcycle_fused(c, 0, e, r0));
  {
    ProfScope ps(c, GBMG_PROF_DF0);
    TRY(launch_df_update_residual(c->stream, L0.d, phi_cur, e, c->F_df, sc + S_MEAN_F, phi_nxt, r_nxt, part, part2,
                                  nullptr));
  }
  TRY(launch_finalize(c->stream, part, df_update_residual_partials(L0.d), sc + S_R2, 1.0));
  TRY(launch_scalars_to_host(c->stream, c->scal, c->host_scal_dev, 8));
  return GBMG_OK;
}

// Cycles run as CUDA graphs (on small meshes the kernels are short, so launching them
// one by one from the host would leave the GPU waiting; on large ones the host is ahead
// except right after each cycle's convergence check): one graph per parity of the
// potential buffers, captured the first time that parity comes up after a cycle of the
// context has run eagerly (which sets every kernel's one-time attributes), then launched
// on c->stream.  Their arguments are the context's own buffers and constants, so the
// same graphs serve every later solve.  Timed kernel families are timed by event nodes
// of the graphs (read after each replay).  A failed capture leaves the context on eager
// launches.
bool cycle_graphs(const gbmg_ctx* c) { return !c->cyc_off; }

gbmg_status solve_mixed(gbmg_ctx* c, const double* F, const double* phi, double* phi_out, double tol, int maxv,
                        gbmg_stats& st) {
  const Level& L0 = c->lv[0];
  const long long n = ncell(L0.d);
  double* part = c->partials;
  double* part1 = c->partials + c->npart;
  double* part2 = c->partials + 2 * c->npart;
  double* sc = c->scal;
  const long long pr = df_partial_count(n), pc = partial_count(L0.d);
  // prologue: F and phi to double-float, mean of F, first residual and ||F - mean||
  TRY(launch_f64_to_df(c->stream, n, F, c->F_df, part));
  TRY(launch_finalize(c->stream, part, pr, sc + S_MEAN_F, 1.0 / (double)n));
  TRY(launch_f64_to_df(c->stream, n, phi, c->phi_df, nullptr));
  float* r0 = (float*)L0.r;
  const long long pu = df_update_residual_partials(L0.d);
  if (c->o.fused) {
    TRY(launch_df_update_residual(c->stream, L0.d, c->phi_df, nullptr, c->F_df, sc + S_MEAN_F, nullptr, r0, part,
                                  part2, part1));
    TRY(launch_finalize(c->stream, part, pu, sc + S_R2, 1.0));
    TRY(launch_finalize(c->stream, part1, pu, sc + S_F2, 1.0));
  } else {
    TRY(launch_df_residual(c->stream, L0.d, c->F_df, sc + S_MEAN_F, c->phi_df, r0, part, part1));
    TRY(launch_finalize(c->stream, part, pc, sc + S_R2, 1.0));
    TRY(launch_finalize(c->stream, part1, pc, sc + S_F2, 1.0));
  }
  double rel = 0.0;
  TRYS(read_rel(c, rel));
  Monitor mon(st, tol, maxv);
  mon.start(rel);
  float2* phi_cur = c->phi_df;
  float2* phi_nxt = c->phi_df2;
  float* r_alt = c->r_alt;
  bool have_sum = c->o.fused;  // the fused residual kernels also sum phi
  while (!mon.done()) {
    if (c->o.fused) {
      const int par = phi_cur == c->phi_df ? 0 : 1;
      sync_graph_mask(c);
      if (c->cyc_warm && cycle_graphs(c) && !c->cyc_exec[par])
        TRYS(capture_graph(c, par, [&]() { return fused_cycle(c, phi_cur, phi_nxt, r0, r_alt); }, c->cyc_exec[par],
                           c->cyc_kernels[par]));
      const bool replay = c->cyc_warm && cycle_graphs(c) && c->cyc_exec[par];
      if (replay) {
        TRY(cudaGraphLaunch(c->cyc_exec[par], c->stream));
        note_launches(c->cyc_kernels[par]);
      } else {
        TRYS(fused_cycle(c, phi_cur, phi_nxt, r0, r_alt));
        c->cyc_warm = true;
      }
      std::swap(phi_cur, phi_nxt);
      std::swap(r0, r_alt);
      TRYS(rel_from_host(c, rel));
      if (replay) gprof_collect(c, par);
      if (mon.record(rel)) break;
      continue;
    }
    {
      float* e = (float*)L0.e;
      float* eo = (float*)L0.e2;
      if (c->o.krylov) {
        TRYS(pcg_correction(c, r0, e));
      } else {
        TRY(cudaMemsetAsync(e, 0, (size_t)n * sizeof(float), c->stream));
        TRYS(vcycle_unfused<float>(c, 0, e, eo, r0));
      }
      TRY(launch_df_update(c->stream, n, phi_cur, e, nullptr));
      {
        ProfScope ps(c, GBMG_PROF_DF0);
        TRY(launch_df_residual(c->stream, L0.d, c->F_df, sc + S_MEAN_F, phi_cur, r0, part, nullptr));
      }
      TRY(launch_finalize(c->stream, part, pc, sc + S_R2, 1.0));
    }
    TRYS(read_rel(c, rel));
    if (mon.record(rel)) break;
  }
  // epilogue: gauge (remove the mean of phi) and convert back to FP64
  if (have_sum) {
    TRY(launch_finalize(c->stream, part2, pu, sc + S_MEAN_PHI, 1.0 / (double)n));
  } else {
    TRY(launch_df_update(c->stream, n, phi_cur, nullptr, part2));
    TRY(launch_finalize(c->stream, part2, pr, sc + S_MEAN_PHI, 1.0 / (double)n));
  }
  TRY(launch_df_to_f64(c->stream, n, phi_cur, sc + S_MEAN_PHI, phi_out));
  return GBMG_OK;
}

gbmg_status check_level(const gbmg_ctx* c, int level, int dtype, const char* who) {
  if (!c) return fail(GBMG_ERR_INVALID_ARG, std::string(who) + ": ctx is NULL");
  if (level < 0 || level >= c->L) return fail(GBMG_ERR_INVALID_ARG, std::string(who) + ": bad level");
  if (dtype != GBMG_F32 && dtype != GBMG_F64) return fail(GBMG_ERR_INVALID_ARG, std::string(who) + ": bad dtype");
  return GBMG_OK;
}

gbmg_status comp_scratch(gbmg_ctx* c, int dtype, void** out) {
  if (!c->comp_scratch[dtype]) {
    const size_t esz = dtype == GBMG_F64 ? 8 : 4;
    void* p = nullptr;
    TRY(cudaMalloc(&p, 2 * (size_t)ncell(c->lv[0].d) * esz));
    c->owned.push_back(p);
    c->comp_scratch[dtype] = p;
  }
  *out = c->comp_scratch[dtype];
  return GBMG_OK;
}

// One solve on the context's stream, without waiting for it: phi_in is the initial
// guess, phi_out receives the result (the same buffer for the in-place mg_solve).
gbmg_status solve_core(gbmg_ctx* c, const double* F, const double* phi_in, double* phi_out, double tol, int maxv,
                       gbmg_stats& st) {
  std::memset(&st, 0, sizeof(st));
  if (c->o.op == GBMG_OP_FLAT7 && c->o.prec != GBMG_FP64) return solve_mixed(c, F, phi_in, phi_out, tol, maxv, st);
  if (c->o.op == GBMG_OP_CURV19 && !c->geom_ready)
    return fail(GBMG_ERR_STATE, "mg_solve: curvilinear solve before mg_set_geometry");
  // the FP64 and curvilinear solves iterate in place
  if (phi_out != phi_in)
    TRY(cudaMemcpyAsync(phi_out, phi_in, (size_t)ncell(c->lv[0].d) * sizeof(double), cudaMemcpyDeviceToDevice,
                        c->stream));
  return c->o.op == GBMG_OP_CURV19 ? curv_solve(c, F, phi_out, tol, maxv, st) : solve_fp64(c, F, phi_out, tol, maxv, st);
}

}  // namespace

// ------------------------------------------------------------------ solve

extern "C" gbmg_status mg_solve(gbmg_ctx* ctx, const double* source_dev, const double* coeffs_dev,
                                double* phi_inout_dev, double tol, int max_vcycles, gbmg_stats* stats) {
  g_last_error.clear();
  if (!ctx || !source_dev || !phi_inout_dev) return fail(GBMG_ERR_INVALID_ARG, "mg_solve: NULL argument");
  if (coeffs_dev && ctx->o.op != GBMG_OP_CURV19)
    return fail(GBMG_ERR_INVALID_ARG, "mg_solve: coeffs must be NULL for the flat operator");
  if (!(tol >= 0.0)) return fail(GBMG_ERR_INVALID_ARG, "mg_solve: tol must be >= 0");
  DeviceGuard g(ctx->device);
  gbmg_stats st;
  if (ctx->o.op == GBMG_OP_CURV19 && coeffs_dev) {
    gbmg_status s = mg_set_geometry(ctx, coeffs_dev);
    if (s != GBMG_OK) return s;
  }
  gbmg_status s = solve_core(ctx, source_dev, phi_inout_dev, phi_inout_dev, tol, max_vcycles, st);
  if (s != GBMG_OK) return s;
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(e, "mg_solve");
  ctx->last = st;
  if (stats) *stats = st;
  if (st.status != GBMG_OK) {
    char buf[160];
    std::snprintf(buf, sizeof(buf), "mg_solve: %s after %d cycles, relative residual %.3e",
                  mg_status_string((gbmg_status)st.status), st.cycles, st.rel_res);
    g_last_error = buf;
  }
  return (gbmg_status)st.status;
}

// The device address of a page-locked host buffer (cudaHostAlloc, cudaHostRegister,
// a pinned torch tensor), or NULL for memory the device cannot address.
static void* device_view(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

extern "C" gbmg_status mg_solve_host(gbmg_ctx* ctx, const double* source_host, double* phi_inout_host, double tol,
                                     int max_vcycles, gbmg_stats* stats) {
  g_last_error.clear();
  if (!ctx || !source_host || !phi_inout_host) return fail(GBMG_ERR_INVALID_ARG, "mg_solve_host: NULL argument");
  DeviceGuard g(ctx->device);
  // Mixed precision touches the FP64 source and phi only in the conversions to and from
  // double-float: with page-locked buffers those kernels read and write host memory
  // over the host link themselves, and no staging copy is made.
  if (ctx->o.prec == GBMG_MIXED) {
    void* Fv = device_view(source_host);
    void* Pv = device_view(phi_inout_host);
    if (Fv && Pv) return mg_solve(ctx, (const double*)Fv, nullptr, (double*)Pv, tol, max_vcycles, stats);
  }
  const size_t bytes = (size_t)ncell(ctx->lv[0].d) * sizeof(double);
  if (!ctx->stage_F) {
    TRY(cudaMalloc((void**)&ctx->stage_F, bytes));
    ctx->owned.push_back(ctx->stage_F);
    TRY(cudaMalloc((void**)&ctx->stage_phi, bytes));
    ctx->owned.push_back(ctx->stage_phi);
  }
  // an error exit first waits for the copies that may still read the host buffers
  cudaError_t e = cudaMemcpyAsync(ctx->stage_F, source_host, bytes, cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ctx->stage_phi, phi_inout_host, bytes, cudaMemcpyHostToDevice, ctx->stream);
  if (e != cudaSuccess) {
    cudaStreamSynchronize(ctx->stream);
    return cuda_fail(e, "mg_solve_host: copy to the device");
  }
  const gbmg_status s = mg_solve(ctx, ctx->stage_F, nullptr, ctx->stage_phi, tol, max_vcycles, stats);
  if (s != GBMG_OK && s != GBMG_ERR_NOT_CONVERGED && s != GBMG_ERR_NONFINITE && s != GBMG_ERR_DIVERGED) {
    cudaStreamSynchronize(ctx->stream);
    return s;
  }
  TRY(cudaMemcpyAsync(phi_inout_host, ctx->stage_phi, bytes, cudaMemcpyDeviceToHost, ctx->stream));
  TRY(cudaStreamSynchronize(ctx->stream));
  return s;
}

// Lazily created copy streams, events and device buffers of mg_solve_host_sequence.
static gbmg_status seq_resources(gbmg_ctx* c) {
  const size_t bytes = (size_t)ncell(c->lv[0].d) * sizeof(double);
  for (int k = 0; k < 2; ++k) {
    if (!c->seq_F[k]) {
      TRY(cudaMalloc((void**)&c->seq_F[k], bytes));
      c->owned.push_back(c->seq_F[k]);
    }
    if (!c->seq_phi[k]) {
      TRY(cudaMalloc((void**)&c->seq_phi[k], bytes));
      c->owned.push_back(c->seq_phi[k]);
    }
  }
  for (cudaEvent_t& e : c->seq_ev)
    if (!e) TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  if (!c->seq_d2h) TRY(cudaStreamCreateWithFlags(&c->seq_d2h, cudaStreamNonBlocking));
  if (!c->seq_h2d) TRY(cudaStreamCreateWithFlags(&c->seq_h2d, cudaStreamNonBlocking));
  return GBMG_OK;
}

extern "C" gbmg_status mg_solve_host_sequence(gbmg_ctx* ctx, int count, const double* const* sources_host,
                                              double* const* phi_host, const double* phi0_host, double tol,
                                              int max_vcycles, gbmg_stats* stats) {
  g_last_error.clear();
  if (!ctx || count < 0 || (count > 0 && (!sources_host || !phi_host)))
    return fail(GBMG_ERR_INVALID_ARG, "mg_solve_host_sequence: bad argument");
  for (int t = 0; t < count; ++t)
    if (!sources_host[t] || !phi_host[t]) return fail(GBMG_ERR_INVALID_ARG, "mg_solve_host_sequence: NULL buffer");
  if (!(tol >= 0.0)) return fail(GBMG_ERR_INVALID_ARG, "mg_solve_host_sequence: tol must be >= 0");
  if (count == 0) return GBMG_OK;
  if (ctx->o.op == GBMG_OP_CURV19 && !ctx->geom_ready)
    return fail(GBMG_ERR_STATE, "mg_solve_host_sequence: curvilinear solve before mg_set_geometry");
  DeviceGuard g(ctx->device);
  TRYS(seq_resources(ctx));
  const size_t bytes = (size_t)ncell(ctx->lv[0].d) * sizeof(double);
  // events: 0,1 source k landed; 2,3 source buffer k read by its solve; 4,5 phi buffer
  // k copied out; 6 solve done
  cudaEvent_t* ev = ctx->seq_ev;
  cudaStream_t cs = ctx->stream, h2d = ctx->seq_h2d, d2h = ctx->seq_d2h;
  // the compute stream's earlier work (and whatever wrote the host buffers' device
  // views) comes first
  // any exit from here on first drains the copy streams, which may still read or write
  // the caller's host buffers
  auto drain = [&]() {
    cudaStreamSynchronize(h2d);
    cudaStreamSynchronize(d2h);
  };
#define STRY(call)                     \
  do {                                 \
    cudaError_t e_ = (call);           \
    if (e_ != cudaSuccess) {           \
      drain();                         \
      return cuda_fail(e_, #call);     \
    }                                  \
  } while (0)
  STRY(cudaEventRecord(ev[6], cs));
  STRY(cudaStreamWaitEvent(h2d, ev[6], 0));
  STRY(cudaStreamWaitEvent(d2h, ev[6], 0));
  STRY(cudaMemcpyAsync(ctx->seq_F[0], sources_host[0], bytes, cudaMemcpyHostToDevice, h2d));
  STRY(cudaEventRecord(ev[0], h2d));
  if (phi0_host) {
    STRY(cudaMemcpyAsync(ctx->seq_phi[0], phi0_host, bytes, cudaMemcpyHostToDevice, h2d));
    STRY(cudaEventRecord(ev[0], h2d));
  } else {
    STRY(cudaMemsetAsync(ctx->seq_phi[0], 0, bytes, cs));
  }
  gbmg_status worst = GBMG_OK;
  for (int t = 0; t < count; ++t) {
    const int k = t & 1, o = k ^ 1;
    // prefetch the next source into the other buffer once the solve that read it is done
    if (t + 1 < count) {
      if (t >= 1) STRY(cudaStreamWaitEvent(h2d, ev[2 + o], 0));
      STRY(cudaMemcpyAsync(ctx->seq_F[o], sources_host[t + 1], bytes, cudaMemcpyHostToDevice, h2d));
      STRY(cudaEventRecord(ev[o], h2d));
    }
    // solve t: source k, initial guess phi k (phi_{t-1}), result into phi o, whose
    // previous content (phi_{t-2}) must have been copied out
    STRY(cudaStreamWaitEvent(cs, ev[k], 0));
    if (t >= 2) STRY(cudaStreamWaitEvent(cs, ev[4 + o], 0));
    gbmg_stats st;
    const gbmg_status s = solve_core(ctx, ctx->seq_F[k], ctx->seq_phi[k], ctx->seq_phi[o], tol, max_vcycles, st);
    if (s != GBMG_OK) {
      drain();
      return s;
    }
    STRY(cudaEventRecord(ev[2 + k], cs));
    STRY(cudaEventRecord(ev[6], cs));
    STRY(cudaStreamWaitEvent(d2h, ev[6], 0));
    STRY(cudaMemcpyAsync(phi_host[t], ctx->seq_phi[o], bytes, cudaMemcpyDeviceToHost, d2h));
    STRY(cudaEventRecord(ev[4 + o], d2h));
    ctx->last = st;
    if (stats) stats[t] = st;
    if (st.status != GBMG_OK && worst == GBMG_OK) worst = (gbmg_status)st.status;
  }
  STRY(cudaStreamSynchronize(ctx->seq_d2h));
  STRY(cudaStreamSynchronize(ctx->seq_h2d));
  STRY(cudaStreamSynchronize(cs));
#undef STRY
  if (worst != GBMG_OK) g_last_error = std::string("mg_solve_host_sequence: ") + mg_status_string(worst);
  return worst;
}

// ------------------------------------------------------------------ components

extern "C" gbmg_status mg_apply(gbmg_ctx* c, int level, int dtype, const void* u, void* out) {
  TRYS(check_level(c, level, dtype, "mg_apply"));
  if (!u || !out) return fail(GBMG_ERR_INVALID_ARG, "mg_apply: NULL buffer");
  DeviceGuard g(c->device);
  const Level& L = c->lv[level];
  const double ih2 = 1.0 / (L.h * L.h);
  if (dtype == GBMG_F64) TRY(launch_apply<double>(c->stream, L.d, (const double*)u, (double*)out, ih2));
  else TRY(launch_apply<float>(c->stream, L.d, (const float*)u, (float*)out, (float)ih2));
  return GBMG_OK;
}

extern "C" gbmg_status mg_residual(gbmg_ctx* c, int level, int dtype, const void* f, const void* u, void* out) {
  TRYS(check_level(c, level, dtype, "mg_residual"));
  if (!f || !u || !out) return fail(GBMG_ERR_INVALID_ARG, "mg_residual: NULL buffer");
  DeviceGuard g(c->device);
  const Level& L = c->lv[level];
  const double ih2 = 1.0 / (L.h * L.h);
  if (dtype == GBMG_F64)
    TRY(launch_residual<double>(c->stream, L.d, (const double*)f, (const double*)u, (double*)out, ih2, nullptr));
  else
    TRY(launch_residual<float>(c->stream, L.d, (const float*)f, (const float*)u, (float*)out, (float)ih2, nullptr));
  return GBMG_OK;
}

template <typename T>
static gbmg_status smooth_component(gbmg_ctx* c, int level, int dtype, T* e_io, const T* r) {
  void* s = nullptr;
  TRYS(comp_scratch(c, dtype, &s));
  T* eo = (T*)s;
  T* dv = eo + ncell(c->lv[0].d);
  T* e = e_io;
  TRYS(smooth_pass<T>(c, level, e, eo, r, dv, false));
  if (e != e_io)
    TRY(cudaMemcpyAsync(e_io, e, (size_t)ncell(c->lv[level].d) * sizeof(T), cudaMemcpyDeviceToDevice, c->stream));
  return GBMG_OK;
}

extern "C" gbmg_status mg_smooth(gbmg_ctx* c, int level, int dtype, void* e, const void* r) {
  TRYS(check_level(c, level, dtype, "mg_smooth"));
  if (!e || !r) return fail(GBMG_ERR_INVALID_ARG, "mg_smooth: NULL buffer");
  DeviceGuard g(c->device);
  if (dtype == GBMG_F64) return smooth_component<double>(c, level, dtype, (double*)e, (const double*)r);
  return smooth_component<float>(c, level, dtype, (float*)e, (const float*)r);
}

extern "C" gbmg_status mg_restrict(gbmg_ctx* c, int level, int dtype, const void* fine, void* coarse) {
  TRYS(check_level(c, level, dtype, "mg_restrict"));
  if (level + 1 >= c->L) return fail(GBMG_ERR_INVALID_ARG, "mg_restrict: level has no coarser level");
  if (!fine || !coarse) return fail(GBMG_ERR_INVALID_ARG, "mg_restrict: NULL buffer");
  DeviceGuard g(c->device);
  if (dtype == GBMG_F64) TRY(launch_restrict<double>(c->stream, c->lv[level].d, (const double*)fine, (double*)coarse));
  else TRY(launch_restrict<float>(c->stream, c->lv[level].d, (const float*)fine, (float*)coarse));
  return GBMG_OK;
}

extern "C" gbmg_status mg_prolong_add(gbmg_ctx* c, int level, int dtype, const void* coarse, void* fine) {
  TRYS(check_level(c, level, dtype, "mg_prolong_add"));
  if (level + 1 >= c->L) return fail(GBMG_ERR_INVALID_ARG, "mg_prolong_add: level has no coarser level");
  if (!fine || !coarse) return fail(GBMG_ERR_INVALID_ARG, "mg_prolong_add: NULL buffer");
  DeviceGuard g(c->device);
  const Dims dc = c->lv[level + 1].d;
  if (dtype == GBMG_F64) TRY(launch_prolong_add<double>(c->stream, dc, (const double*)coarse, (double*)fine));
  else TRY(launch_prolong_add<float>(c->stream, dc, (const float*)coarse, (float*)fine));
  return GBMG_OK;
}

extern "C" gbmg_status mg_coarse_solve(gbmg_ctx* c, int dtype, const void* r, void* e) {
  TRYS(check_level(c, 0, dtype, "mg_coarse_solve"));
  if (!r || !e) return fail(GBMG_ERR_INVALID_ARG, "mg_coarse_solve: NULL buffer");
  DeviceGuard g(c->device);
  if (dtype == GBMG_F64) TRY(launch_coarse_matvec<double>(c->stream, c->nc, c->G64, (const double*)r, (double*)e));
  else TRY(launch_coarse_matvec<float>(c->stream, c->nc, c->G32, (const float*)r, (float*)e));
  return GBMG_OK;
}

extern "C" gbmg_status mg_vcycle(gbmg_ctx* c, const void* r, void* e_out) {
  if (!c || !r || !e_out) return fail(GBMG_ERR_INVALID_ARG, "mg_vcycle: NULL argument");
  DeviceGuard g(c->device);
  const Level& L0 = c->lv[0];
  const long long n = ncell(L0.d);
  if (c->o.prec == GBMG_FP64) {
    double* e = (double*)L0.e;
    double* eo = (double*)L0.e2;
    TRY(cudaMemsetAsync(e, 0, (size_t)n * 8, c->stream));
    TRYS(vcycle_unfused<double>(c, 0, e, eo, (const double*)r));
    TRY(cudaMemcpyAsync(e_out, e, (size_t)n * 8, cudaMemcpyDeviceToDevice, c->stream));
  } else {
    float* e = (float*)L0.e;
    if (c->o.fused) {
      TRYS(vcycle_fused(c, 0, e, (const float*)r));
    } else {
      float* eo = (float*)L0.e2;
      TRY(cudaMemsetAsync(e, 0, (size_t)n * 4, c->stream));
      TRYS(vcycle_unfused<float>(c, 0, e, eo, (const float*)r));
    }
    TRY(cudaMemcpyAsync(e_out, e, (size_t)n * 4, cudaMemcpyDeviceToDevice, c->stream));
  }
  return GBMG_OK;
}

extern "C" gbmg_status mg_f64_to_df(gbmg_ctx* c, long long n, const double* x, float* df) {
  if (!c || !x || !df || n < 0) return fail(GBMG_ERR_INVALID_ARG, "mg_f64_to_df: bad argument");
  DeviceGuard g(c->device);
  TRY(launch_f64_to_df(c->stream, n, x, (float2*)df, nullptr));
  return GBMG_OK;
}

extern "C" gbmg_status mg_df_to_f64(gbmg_ctx* c, long long n, const float* df, double* x) {
  if (!c || !x || !df || n < 0) return fail(GBMG_ERR_INVALID_ARG, "mg_df_to_f64: bad argument");
  DeviceGuard g(c->device);
  TRY(launch_df_to_f64(c->stream, n, (const float2*)df, nullptr, x));
  return GBMG_OK;
}

extern "C" gbmg_status mg_df_residual(gbmg_ctx* c, const float* F, double m, const float* phi, float* r) {
  if (!c || !F || !phi || !r) return fail(GBMG_ERR_INVALID_ARG, "mg_df_residual: NULL argument");
  DeviceGuard g(c->device);
  double* slot = c->scal + S_USER;
  TRY(cudaStreamSynchronize(c->stream));
  TRY(cudaMemcpy(slot, &m, sizeof(double), cudaMemcpyHostToDevice));
  TRY(launch_df_residual(c->stream, c->lv[0].d, (const float2*)F, slot, (const float2*)phi, r, nullptr, nullptr));
  return GBMG_OK;
}
