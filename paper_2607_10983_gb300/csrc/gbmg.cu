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
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

gbmg_status fail(gbmg_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

gbmg_status cuda_fail(cudaError_t e, const char* what) {
  if (e == cudaErrorMemoryAllocation) return fail(GBMG_ERR_OOM, std::string(what) + ": " + cudaGetErrorString(e));
  return fail(GBMG_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// ------------------------------------------------------------------ hierarchy

std::vector<Dims> level_dims(int nx, int ny, int nz, int levels) {
  std::vector<Dims> out{Dims{nx, ny, nz}};
  for (;;) {
    if (levels > 0 && (int)out.size() >= levels) break;
    const Dims d = out.back();
    if (d.nx % 2 == 0 && d.ny % 2 == 0 && d.nz % 2 == 0 && d.nx / 2 >= 4 && d.ny / 2 >= 4 && d.nz / 2 >= 4)
      out.push_back(Dims{d.nx / 2, d.ny / 2, d.nz / 2});
    else
      break;
  }
  return out;
}

// Minimum-norm least-squares inverse of a singular n x n operator L whose null space
// is span(1) and whose left null space is span(w): the bordered system
// [[L, 1], [1^T, 0]] is inverted by Gauss-Jordan with partial pivoting; its leading
// block X solves L x = r' with 1^T x = 0 for r' orthogonal to w, and
// G = X (I - w w^T / w^T w) projects r onto the range of L first.
bool dense_pinv(int n, const std::vector<double>& Lm, const std::vector<double>& w, std::vector<double>& G) {
  const int m = n + 1;
  std::vector<double> K((size_t)m * m, 0.0), I((size_t)m * m, 0.0);
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j < n; ++j) K[(size_t)i * m + j] = Lm[(size_t)i * n + j];
    K[(size_t)i * m + n] = 1.0;
    K[(size_t)n * m + i] = 1.0;
  }
  for (int i = 0; i < m; ++i) I[(size_t)i * m + i] = 1.0;
  for (int col = 0; col < m; ++col) {
    int piv = col;
    double best = std::fabs(K[(size_t)col * m + col]);
    for (int r = col + 1; r < m; ++r) {
      const double v = std::fabs(K[(size_t)r * m + col]);
      if (v > best) {
        best = v;
        piv = r;
      }
    }
    if (!(best > 1e-300)) return false;
    if (piv != col) {
      for (int j = 0; j < m; ++j) {
        std::swap(K[(size_t)piv * m + j], K[(size_t)col * m + j]);
        std::swap(I[(size_t)piv * m + j], I[(size_t)col * m + j]);
      }
    }
    const double inv = 1.0 / K[(size_t)col * m + col];
    for (int j = 0; j < m; ++j) {
      K[(size_t)col * m + j] *= inv;
      I[(size_t)col * m + j] *= inv;
    }
    for (int r = 0; r < m; ++r) {
      if (r == col) continue;
      const double f = K[(size_t)r * m + col];
      if (f == 0.0) continue;
      for (int j = 0; j < m; ++j) {
        K[(size_t)r * m + j] -= f * K[(size_t)col * m + j];
        I[(size_t)r * m + j] -= f * I[(size_t)col * m + j];
      }
    }
  }
  double ww = 0.0;
  for (int i = 0; i < n; ++i) ww += w[i] * w[i];
  std::vector<double> Xw(n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Xw[i] += I[(size_t)i * m + j] * w[j];
  G.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) G[(size_t)i * n + j] = I[(size_t)i * m + j] - Xw[i] * w[j] / ww;
  return true;
}

// Dense 7-point operator of a periodic level with spacing h (sides >= 3).
std::vector<double> dense_flat(Dims d, double h) {
  const int n = d.nx * d.ny * d.nz;
  std::vector<double> A((size_t)n * n, 0.0);
  const double s = 1.0 / (h * h);
  for (int z = 0; z < d.nz; ++z)
    for (int y = 0; y < d.ny; ++y)
      for (int x = 0; x < d.nx; ++x) {
        const int i = (z * d.ny + y) * d.nx + x;
        auto at = [&](int xx, int yy, int zz) {
          xx = (xx + d.nx) % d.nx;
          yy = (yy + d.ny) % d.ny;
          zz = (zz + d.nz) % d.nz;
          return (zz * d.ny + yy) * d.nx + xx;
        };
        A[(size_t)i * n + i] -= 6.0 * s;
        A[(size_t)i * n + at(x - 1, y, z)] += s;
        A[(size_t)i * n + at(x + 1, y, z)] += s;
        A[(size_t)i * n + at(x, y - 1, z)] += s;
        A[(size_t)i * n + at(x, y + 1, z)] += s;
        A[(size_t)i * n + at(x, y, z - 1)] += s;
        A[(size_t)i * n + at(x, y, z + 1)] += s;
      }
  return A;
}

// Chebyshev semi-iteration coefficients on [2/alpha, 2] (Sec. 2.3): step 0 has
// c1 = 0, c2 = 1/theta; step k >= 1 has rho' = 1/(2 sigma - rho),
// c1 = rho' rho, c2 = 2 rho' / delta.
void chebyshev_schedule(int degree, double alpha, std::vector<double>& c1, std::vector<double>& c2) {
  const double a = 2.0 / alpha, b = 2.0;
  const double theta = 0.5 * (a + b), delta = 0.5 * (b - a), sigma = theta / delta;
  c1.assign(degree, 0.0);
  c2.assign(degree, 0.0);
  c2[0] = 1.0 / theta;
  double rho = 1.0 / sigma;
  for (int k = 1; k < degree; ++k) {
    const double rn = 1.0 / (2.0 * sigma - rho);
    c1[k] = rn * rho;
    c2[k] = 2.0 * rn / delta;
    rho = rn;
  }
}

}  // namespace gbmg

using namespace gbmg;

// ------------------------------------------------------------------ context

gbmg_ctx::~gbmg_ctx() {
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
  if (launches) *launches = ctx->prof_n[family];
  if (total_ms) *total_ms = ms;
  return GBMG_OK;
}

extern "C" gbmg_status mg_profile_end(gbmg_ctx* ctx) {
  if (!ctx) return fail(GBMG_ERR_INVALID_ARG, "mg_profile_end: ctx is NULL");
  ctx->prof_mask = 0;
  for (int& n : ctx->prof_n) n = 0;
  return GBMG_OK;
}
