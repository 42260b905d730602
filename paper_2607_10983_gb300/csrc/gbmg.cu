// Host side of the library: context and workspace, the multigrid hierarchy, the
// V-cycle level loop, the solve drivers and the C ABI declared in include/gbmg.h.
#include <cmath>
#include <cstdio>
#include <algorithm>
#include <atomic>
#include <cstring>
#include <string>
#include <vector>

#include "gbmg.h"
#include "kernels.h"
#include "solver.h"

namespace gbmg {

thread_local std::string g_last_error;

static std::atomic<long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void note_launches(long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

gbmg_status fail(gbmg_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

gbmg_status cuda_fail(cudaError_t e, const char* what) {
  if (e == cudaErrorMemoryAllocation) return fail(GBMG_ERR_OOM, std::string(what) + ": " + cudaGetErrorString(e));
  return fail(GBMG_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

}  // namespace gbmg

using namespace gbmg;

// ------------------------------------------------------------------ context

gbmg_ctx::~gbmg_ctx() {
  for (cudaGraphExec_t g : cyc_exec)
    if (g) cudaGraphExecDestroy(g);
  for (cudaGraphExec_t g : curv_exec)
    if (g) cudaGraphExecDestroy(g);
  for (auto& slot : gprof_ev)
    for (auto& fam : slot)
      for (auto& pr : fam)
        for (cudaEvent_t ev : pr)
          if (ev) cudaEventDestroy(ev);
  if (cap_stream) cudaStreamDestroy(cap_stream);
  for (auto& v : prof_ev)
    for (cudaEvent_t e : v) cudaEventDestroy(e);
  for (cudaStream_t s : {seq_h2d, seq_d2h})
    if (s) {
      cudaStreamSynchronize(s);
      cudaStreamDestroy(s);
    }
  for (cudaEvent_t e : seq_ev)
    if (e) cudaEventDestroy(e);
  if (arena) cudaFree(arena);
  if (host_scal) cudaFreeHost(host_scal);
  for (void* p : owned) cudaFree(p);
}

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

extern "C" void gbmg_default_opts(gbmg_opts* o) {
  if (!o) return;
  o->op = GBMG_OP_FLAT7;
  o->prec = GBMG_MIXED;
  o->smoother = GBMG_SMOOTH_CHEBYSHEV;
  o->degree = 3;
  o->alpha = 8.0;
  o->nu1 = 2;
  o->nu2 = 2;
  o->omega = 2.0 / 3.0;
  o->fused = 1;
  o->krylov = 0;
  o->curv_sym = 0;
  o->coarse_store = 0;
}

extern "C" const char* mg_status_string(gbmg_status s) {
  switch (s) {
    case GBMG_OK: return "ok";
    case GBMG_ERR_INVALID_ARG: return "invalid argument";
    case GBMG_ERR_CUDA: return "CUDA error";
    case GBMG_ERR_OOM: return "out of memory";
    case GBMG_ERR_NOT_CONVERGED: return "not converged";
    case GBMG_ERR_NONFINITE: return "non-finite residual";
    case GBMG_ERR_DIVERGED: return "diverged";
    case GBMG_ERR_STATE: return "invalid state";
  }
  return "unknown status";
}

extern "C" const char* mg_last_error(void) { return g_last_error.c_str(); }

extern "C" gbmg_status mg_setup(gbmg_ctx** out, int nx, int ny, int nz, int levels, int smoother_degree,
                                const gbmg_opts* opts, void* cuda_stream) {
  g_last_error.clear();
  if (!out) return fail(GBMG_ERR_INVALID_ARG, "mg_setup: out is NULL");
  if (nx < 4 || ny < 4 || nz < 4) return fail(GBMG_ERR_INVALID_ARG, "mg_setup: every side must be >= 4");
  if (levels < 0) return fail(GBMG_ERR_INVALID_ARG, "mg_setup: levels < 0");
  gbmg_opts o;
  gbmg_default_opts(&o);
  if (opts) o = *opts;
  if (smoother_degree > 0) o.degree = smoother_degree;
  if (o.op != GBMG_OP_FLAT7 && o.op != GBMG_OP_CURV19) return fail(GBMG_ERR_INVALID_ARG, "mg_setup: unsupported operator");
  if (o.op == GBMG_OP_CURV19 && o.smoother != GBMG_SMOOTH_JACOBI)
    return fail(GBMG_ERR_INVALID_ARG, "mg_setup: the curvilinear operator uses the weighted-Jacobi smoother");
  if (o.op == GBMG_OP_CURV19 && o.prec != GBMG_MIXED)
    return fail(GBMG_ERR_INVALID_ARG, "mg_setup: the curvilinear operator runs in mixed precision");
  if (o.prec != GBMG_FP64 && o.prec != GBMG_MIXED) return fail(GBMG_ERR_INVALID_ARG, "mg_setup: bad precision");
  if (o.smoother != GBMG_SMOOTH_CHEBYSHEV && o.smoother != GBMG_SMOOTH_JACOBI)
    return fail(GBMG_ERR_INVALID_ARG, "mg_setup: bad smoother");
  if (o.degree < 1 || o.degree > 16) return fail(GBMG_ERR_INVALID_ARG, "mg_setup: degree must be in [1, 16]");
  if (!(o.alpha > 1.0)) return fail(GBMG_ERR_INVALID_ARG, "mg_setup: alpha must be > 1");
  if (o.nu1 < 0 || o.nu2 < 0 || o.nu1 > 64 || o.nu2 > 64) return fail(GBMG_ERR_INVALID_ARG, "mg_setup: bad nu1/nu2");
  if (!(o.omega > 0.0 && o.omega < 2.0)) return fail(GBMG_ERR_INVALID_ARG, "mg_setup: omega must be in (0, 2)");
  if (o.fused && !(o.op == GBMG_OP_FLAT7 && o.prec == GBMG_MIXED && o.smoother == GBMG_SMOOTH_CHEBYSHEV &&
                   fused_degree_supported(o.degree)))
    o.fused = 0;
  if (o.fused && nx % 2 != 0) o.fused = 0;  // the fused kernels work on x-pairs
  if (o.krylov < 0 || o.krylov > 16) return fail(GBMG_ERR_INVALID_ARG, "mg_setup: krylov must be in [0, 16]");
  if (o.krylov && !(o.op == GBMG_OP_FLAT7 && o.prec == GBMG_MIXED && o.smoother == GBMG_SMOOTH_CHEBYSHEV))
    return fail(GBMG_ERR_INVALID_ARG, "mg_setup: krylov needs the flat operator, mixed precision and Chebyshev");
  if (o.curv_sym != 0 && o.curv_sym != 1) return fail(GBMG_ERR_INVALID_ARG, "mg_setup: curv_sym must be 0 or 1");
  if (o.curv_sym && o.op != GBMG_OP_CURV19)
    return fail(GBMG_ERR_INVALID_ARG, "mg_setup: curv_sym needs the curvilinear operator");
  if (o.coarse_store < 0 || o.coarse_store > 2)
    return fail(GBMG_ERR_INVALID_ARG, "mg_setup: coarse_store must be 0 (FP32), 1 (BF16) or 2 (FP16)");
  if (o.coarse_store && !(o.op == GBMG_OP_FLAT7 && o.prec == GBMG_MIXED))
    return fail(GBMG_ERR_INVALID_ARG, "mg_setup: coarse_store needs the flat operator in mixed precision");
  const bool curv = o.op == GBMG_OP_CURV19;

  std::vector<Dims> dims = level_dims(nx, ny, nz, levels);
  const Dims dc = dims.back();
  const long long nc = ncell(dc);
  if (nc > 512) return fail(GBMG_ERR_INVALID_ARG, "mg_setup: coarsest level has more than 512 cells");

  auto* c = new (std::nothrow) gbmg_ctx();
  if (!c) return fail(GBMG_ERR_OOM, "mg_setup: host allocation");
  cudaError_t e = cudaGetDevice(&c->device);
  if (e != cudaSuccess) {
    delete c;
    return cuda_fail(e, "cudaGetDevice");
  }
  c->stream = (cudaStream_t)cuda_stream;
  c->o = o;
  c->L = (int)dims.size();
  c->nc = (int)nc;
  c->fused_all = o.fused == 2;
  chebyshev_schedule(o.degree, o.alpha, c->cc1, c->cc2);

  const size_t esz = o.prec == GBMG_FP64 ? sizeof(double) : sizeof(float);
  const long long n0 = ncell(dims[0]);
  // workspace layout
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o0 = off;
    off += align256(bytes);
    return o0;
  };
  struct Offs {
    size_t r, e, e2, dv, t;
  };
  std::vector<Offs> lo(dims.size());
  std::vector<size_t> lpsi(dims.size()), lcoef(dims.size());
  for (size_t l = 0; l < dims.size(); ++l) {
    const size_t b = (size_t)ncell(dims[l]) * esz;
    lo[l] = Offs{take(b), take(b), take(b), take(b), take(b)};
    if (curv) {
      lpsi[l] = take((size_t)ncell(dims[l]) * sizeof(double));
      lcoef[l] = take((size_t)ncell(dims[l]) * 7 * sizeof(float));
    }
  }
  size_t oF = 0, oP = 0, oP2 = 0, oR = 0;
  if (o.prec == GBMG_MIXED) {
    oF = take((size_t)n0 * sizeof(float2));
    oP = take((size_t)n0 * sizeof(float2));
    if (o.fused) oP2 = take((size_t)n0 * sizeof(float2));
    oR = take((size_t)n0 * sizeof(float));
  }
  const long long np = std::max(std::max(partial_count(dims[0]), df_partial_count(n0)),
                                df_update_residual_partials(dims[0]));
  const size_t oPart = take((size_t)np * 4 * sizeof(double));
  const size_t oScal = take(64 * sizeof(double));
  const size_t oG64 = take((size_t)nc * nc * sizeof(double));
  const size_t oG32 = take((size_t)nc * nc * sizeof(float));
  size_t oG64T = 0, oG32T = 0, oDense = 0;
  if (curv) {
    oG64T = take((size_t)nc * nc * sizeof(double));
    oG32T = take((size_t)nc * nc * sizeof(float));
    oDense = take((size_t)nc * nc * sizeof(double));
  }
  c->arena_bytes = off;
  e = cudaMalloc((void**)&c->arena, off);
  if (e != cudaSuccess) {
    delete c;
    return cuda_fail(e, "mg_setup: workspace allocation");
  }
  e = cudaMallocHost((void**)&c->host_scal, 64 * sizeof(double));
  if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&c->host_scal_dev, c->host_scal, 0);
  if (e != cudaSuccess) {
    delete c;
    return cuda_fail(e, "mg_setup: pinned allocation");
  }
  char* a = c->arena;
  c->lv.resize(dims.size());
  for (size_t l = 0; l < dims.size(); ++l) {
    Level& L = c->lv[l];
    L.d = dims[l];
    L.h = std::ldexp(1.0, (int)l);
    L.r = a + lo[l].r;
    L.e = a + lo[l].e;
    L.e2 = a + lo[l].e2;
    L.dv = a + lo[l].dv;
    L.t = a + lo[l].t;
    if (curv) {
      L.psi = (double*)(a + lpsi[l]);
      float* cb = (float*)(a + lcoef[l]);
      const long long nl = ncell(dims[l]);
      L.cc.J = cb;
      for (int k = 0; k < 6; ++k) L.cc.B[k] = cb + (k + 1) * nl;
      L.cc.h2 = (float)(L.h * L.h);
    }
  }
  if (curv) {
    c->G64T = (double*)(a + oG64T);
    c->G32T = (float*)(a + oG32T);
    c->dense = (double*)(a + oDense);
  }
  if (o.prec == GBMG_MIXED) {
    c->F_df = (float2*)(a + oF);
    c->phi_df = (float2*)(a + oP);
    c->phi_df2 = o.fused ? (float2*)(a + oP2) : nullptr;
    c->r_alt = (float*)(a + oR);
  }
  c->npart = np;
  c->partials = (double*)(a + oPart);
  c->scal = (double*)(a + oScal);
  c->G64 = (double*)(a + oG64);
  c->G32 = (float*)(a + oG32);

  if (curv) {
    // the coarsest pseudo-inverse depends on the geometry: built by mg_set_geometry
    e = cudaMemset(c->scal, 0, 64 * sizeof(double));
    if (e != cudaSuccess) {
      delete c;
      return cuda_fail(e, "mg_setup: memset");
    }
    std::memset(&c->last, 0, sizeof(c->last));
    *out = c;
    return GBMG_OK;
  }
  // coarsest-level pseudo-inverse of the rediscretised 7-point operator
  std::vector<double> A = dense_flat(dc, c->lv.back().h), G;
  std::vector<double> w((size_t)nc, 1.0);
  if (!dense_pinv((int)nc, A, w, G)) {
    delete c;
    return fail(GBMG_ERR_INVALID_ARG, "mg_setup: coarsest operator is not invertible on the zero-mean subspace");
  }
  std::vector<float> G32(G.begin(), G.end());
  e = cudaMemcpy(c->G64, G.data(), G.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(c->G32, G32.data(), G32.size() * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(c->scal, 0, 64 * sizeof(double));
  if (e != cudaSuccess) {
    delete c;
    return cuda_fail(e, "mg_setup: upload");
  }
  std::memset(&c->last, 0, sizeof(c->last));
  *out = c;
  return GBMG_OK;
}

extern "C" void mg_destroy(gbmg_ctx* ctx) { delete ctx; }

extern "C" gbmg_status mg_set_stream(gbmg_ctx* ctx, void* s) {
  if (!ctx) return fail(GBMG_ERR_INVALID_ARG, "mg_set_stream: ctx is NULL");
  ctx->stream = (cudaStream_t)s;
  return GBMG_OK;
}

extern "C" gbmg_status mg_set_cycle_graphs(gbmg_ctx* ctx, int enable) {
  if (!ctx) return fail(GBMG_ERR_INVALID_ARG, "mg_set_cycle_graphs: ctx is NULL");
  DeviceGuard g(ctx->device);
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(e, "mg_set_cycle_graphs");
  ctx->cyc_off = enable == 0;
  ctx->graph_mask = -1;  // drop the graphs captured so far
  sync_graph_mask(ctx);
  return GBMG_OK;
}

extern "C" int mg_num_levels(const gbmg_ctx* ctx) { return ctx ? ctx->L : 0; }

extern "C" gbmg_status mg_level_dims(const gbmg_ctx* ctx, int level, int* nx, int* ny, int* nz) {
  if (!ctx || level < 0 || level >= ctx->L) return fail(GBMG_ERR_INVALID_ARG, "mg_level_dims: bad level");
  if (nx) *nx = ctx->lv[level].d.nx;
  if (ny) *ny = ctx->lv[level].d.ny;
  if (nz) *nz = ctx->lv[level].d.nz;
  return GBMG_OK;
}

extern "C" gbmg_status mg_last_stats(gbmg_ctx* ctx, gbmg_stats* stats) {
  if (!ctx || !stats) return fail(GBMG_ERR_INVALID_ARG, "mg_last_stats: NULL argument");
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(e, "mg_last_stats");
  *stats = ctx->last;
  return GBMG_OK;
}

extern "C" long long mg_launch_count(void) { return launch_count(); }

extern "C" gbmg_status mg_profile_begin(gbmg_ctx* ctx, int family_mask) {
  if (!ctx) return fail(GBMG_ERR_INVALID_ARG, "mg_profile_begin: ctx is NULL");
  if (family_mask < 0 || family_mask >= (1 << 8)) return fail(GBMG_ERR_INVALID_ARG, "mg_profile_begin: bad mask");
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(e, "mg_profile_begin");
  ctx->prof_mask = family_mask & ~1;
  for (int& n : ctx->prof_n) n = 0;
  for (int& n : ctx->prof_gn) n = 0;
  for (double& t : ctx->prof_gms) t = 0.0;
  // event pairs for the cycle graphs' timed launches (created here, outside any capture)
  for (auto& slot : ctx->gprof_ev)
    for (int f = 1; f < 8; ++f) {
      if (!(ctx->prof_mask >> f & 1)) continue;
      for (auto& pr : slot[f])
        for (cudaEvent_t& ev : pr)
          if (!ev) {
            e = cudaEventCreate(&ev);
            if (e != cudaSuccess) return cuda_fail(e, "mg_profile_begin: cudaEventCreate");
          }
    }
  return GBMG_OK;
}

extern "C" gbmg_status mg_profile_read(gbmg_ctx* ctx, int family, int* launches, double* total_ms) {
  if (!ctx || family < 1 || family > 7) return fail(GBMG_ERR_INVALID_ARG, "mg_profile_read: bad argument");
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(e, "mg_profile_read");
  double ms = 0.0;
  const std::vector<cudaEvent_t>& ev = ctx->prof_ev[family];
  for (int i = 0; i < ctx->prof_n[family]; ++i) {
    float t = 0.f;
    e = cudaEventElapsedTime(&t, ev[2 * i], ev[2 * i + 1]);
    if (e != cudaSuccess) return cuda_fail(e, "mg_profile_read: cudaEventElapsedTime");
    ms += t;
  }
  if (launches) *launches = ctx->prof_n[family] + ctx->prof_gn[family];
  if (total_ms) *total_ms = ms + ctx->prof_gms[family];
  return GBMG_OK;
}

extern "C" gbmg_status mg_profile_end(gbmg_ctx* ctx) {
  if (!ctx) return fail(GBMG_ERR_INVALID_ARG, "mg_profile_end: ctx is NULL");
  ctx->prof_mask = 0;
  for (int& n : ctx->prof_n) n = 0;
  for (int& n : ctx->prof_gn) n = 0;
  for (double& t : ctx->prof_gms) t = 0.0;
  return GBMG_OK;
}
