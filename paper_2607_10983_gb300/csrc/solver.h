// Internal definition of the solver context shared by the host translation units.
#pragma once
#include <cmath>
#include <string>
#include <vector>

#include "common.cuh"
#include "gbmg.h"
#include "kernels.h"

namespace gbmg {

struct Level {
  Dims d;
  double h;       // spacing 2^l in finest-level cells
  // element type = working precision (double for GBMG_FP64, float for GBMG_MIXED)
  void* r;        // right-hand side of the level's error equation
  void* e;        // error iterate (ping-pong with e2)
  void* e2;
  void* dv;       // Chebyshev direction
  void* t;        // residual scratch
  double* psi = nullptr;  // curvilinear: deformation potential restricted to this level (FP64)
  CurvCoef cc{};          // curvilinear: J and B of this level (FP32)
};

gbmg_status fail(gbmg_status s, const std::string& msg);
gbmg_status cuda_fail(cudaError_t e, const char* what);
extern thread_local std::string g_last_error;

// curvilinear / adjoint drivers (curv_solve.cu)
gbmg_status curv_solve(gbmg_ctx* c, const double* F, double* phi, double tol, int maxv, gbmg_stats& st);

// Parameters of the single-CTA bottom cycle from level l (false when it does not apply).
bool small_cycle_params(const gbmg_ctx* c, int l, SmallCycle* out);

// Slots of the device scalar area gbmg_ctx::scal.
enum Scal {
  S_SUM_F = 0,   // sum of F, then its mean
  S_MEAN_F = 1,
  S_F2 = 2,      // ||F - mean||^2
  S_R2 = 3,      // ||r||^2
  S_SUM_PHI = 4,
  S_MEAN_PHI = 5,
  S_USER = 8,    // component calls
};

}  // namespace gbmg

struct gbmg_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  gbmg_opts o{};
  int L = 0;
  std::vector<gbmg::Level> lv;
  char* arena = nullptr;
  size_t arena_bytes = 0;
  int nc = 0;                   // cells on the coarsest level
  double* G64 = nullptr;        // coarsest pseudo-inverse, row-major nc x nc
  float* G32 = nullptr;
  double* G64T = nullptr;       // curvilinear: pseudo-inverse of the transposed-solve operator
  float* G32T = nullptr;
  double* dense = nullptr;      // curvilinear: nc x nc scratch for the coarsest operator
  bool geom_ready = false;      // curvilinear: mg_set_geometry or mg_set_coefficients has run
  bool geom_from_psi = false;   // the coefficients were built from psi (psi_bar needs psi)
  bool fused_all = false;       // testing: blocked kernels on every level of at least 16^3
  double* adj_S = nullptr;      // adjoint scratch (6 finest fields), allocated on first use
  double* adj_lam = nullptr;    // adjoint scratch (1 finest field)
  double* motion = nullptr;     // mesh-motion scratch (2 finest fields), allocated on first use
  float* force_scratch = nullptr;  // FP32 potential and force grid (4 finest fields), first use of mg_force
  float* pcg = nullptr;         // conjugate-gradient vectors e, p, q (3 finest FP32 fields), first use
  float2* F_df = nullptr;       // mixed precision: source as double-float
  float2* phi_df = nullptr;     // mixed precision: potential as double-float
  float2* phi_df2 = nullptr;    // mixed precision: second potential buffer (fused update)
  float* r_alt = nullptr;       // mixed precision: second finest residual buffer
  double* partials = nullptr;   // 4 regions of npart block partial sums
  long long npart = 0;
  double* scal = nullptr;       // 64 device scalars (enum Scal)
  double* host_scal = nullptr;  // 64 pinned host scalars
  double* host_scal_dev = nullptr;  // its device address (the device writes it directly)
  std::vector<double> cc1, cc2; // Chebyshev schedule
  gbmg_stats last{};
  std::vector<void*> owned;     // lazily allocated buffers (component scratch, staging)
  void* comp_scratch[2] = {nullptr, nullptr};  // per dtype: 2 finest-level fields
  int prof_mask = 0;            // bit (1 << gbmg_prof_family) set = family timed
  int prof_n[8] = {0};          // timed launches per family
  std::vector<cudaEvent_t> prof_ev[8];  // start/stop event pairs per family
  double* stage_F = nullptr;    // mg_solve_host device staging
  double* stage_phi = nullptr;
  double* seq_F[2] = {nullptr, nullptr};    // mg_solve_host_sequence: sources in flight
  double* seq_phi[2] = {nullptr, nullptr};  // and the iterate, ping-pong
  cudaStream_t seq_h2d = nullptr, seq_d2h = nullptr;
  cudaEvent_t seq_ev[7] = {};
  // mixed fused solves: one cycle as a CUDA graph per parity of the potential buffers
  // (captured on a private stream on first use, launched on `stream`)
  cudaGraphExec_t cyc_exec[2] = {nullptr, nullptr};
  long long cyc_kernels[2] = {0, 0};
  cudaStream_t cap_stream = nullptr;
  bool cyc_off = false;   // a capture failed: this context launches its cycles one by one
  bool cyc_warm = false;  // a cycle has run eagerly (the kernels' one-time attributes are set)
  // curvilinear solves: one cycle as a CUDA graph per orientation (forward, transposed)
  cudaGraphExec_t curv_exec[2] = {nullptr, nullptr};
  long long curv_kernels[2] = {0, 0};
  bool curv_warm[2] = {false, false};
  // kernel timing inside the cycle graphs: per graph slot (flat parity 0 / 1, curvilinear
  // orientation 0 / 1), family and timed launch an event pair that the graph's nodes record
  // on every replay; read after each replay into the per-family totals
  static constexpr int GSLOTS = 4, GPAIRS = 8;
  cudaEvent_t gprof_ev[GSLOTS][8][GPAIRS][2] = {};
  int gprof_cnt[GSLOTS][8] = {};
  int cap_slot = -1;            // slot of the graph being captured (-1: none)
  int graph_mask = 0;           // prof_mask the cycle graphs were captured with
  double prof_gms[8] = {};      // graph-timed milliseconds and launches per family
  int prof_gn[8] = {};
  ~gbmg_ctx();
};

namespace gbmg {

#define TRY(call)                                  \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)
#define TRYS(call)                  \
  do {                              \
    gbmg_status s_ = (call);        \
    if (s_ != GBMG_OK) return s_;   \
  } while (0)

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

// Brackets one launch with CUDA events on the context's stream when its kernel
// family is being timed (mg_profile_begin); no effect otherwise.
struct ProfScope {
  gbmg_ctx* c;
  int f;
  bool on = false;
  int k = -1;  // pair of the cycle graph being captured (-1: eager)
  ProfScope(gbmg_ctx* ctx, int family) : c(ctx), f(family) {
    if (family <= GBMG_PROF_OFF || family > 7 || !(c->prof_mask >> family & 1)) return;
    if (c->cap_slot >= 0) {
      // inside a capture: the events were created by mg_profile_begin; launches of a
      // family beyond GPAIRS per cycle are not timed
      const int n = c->gprof_cnt[c->cap_slot][f];
      cudaEvent_t* p = c->gprof_ev[c->cap_slot][f][n < gbmg_ctx::GPAIRS ? n : 0];
      if (n >= gbmg_ctx::GPAIRS || !p[0] || !p[1]) return;
      // (external: an event-record node of the graph, not a capture dependency)
      on = cudaEventRecordWithFlags(p[0], c->stream, cudaEventRecordExternal) == cudaSuccess;
      k = n;
      return;
    }
    std::vector<cudaEvent_t>& ev = c->prof_ev[f];
    const size_t need = 2 * (size_t)c->prof_n[f] + 2;
    while (ev.size() < need) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return;
      ev.push_back(e);
    }
    on = cudaEventRecord(ev[2 * c->prof_n[f]], c->stream) == cudaSuccess;
  }
  ~ProfScope() {
    if (!on) return;
    if (k >= 0) {
      if (cudaEventRecordWithFlags(c->gprof_ev[c->cap_slot][f][k][1], c->stream, cudaEventRecordExternal) == cudaSuccess)
        c->gprof_cnt[c->cap_slot][f] = k + 1;
      return;
    }
    if (cudaEventRecord(c->prof_ev[f][2 * c->prof_n[f] + 1], c->stream) == cudaSuccess) c->prof_n[f] += 1;
  }
};

// Drops the cycle graphs when the set of timed families has changed since they were
// captured (they are captured again, with or without event nodes).
inline void sync_graph_mask(gbmg_ctx* c) {
  if (c->graph_mask == c->prof_mask) return;
  for (cudaGraphExec_t& g : c->cyc_exec)
    if (g) cudaGraphExecDestroy(g), g = nullptr;
  for (cudaGraphExec_t& g : c->curv_exec)
    if (g) cudaGraphExecDestroy(g), g = nullptr;
  for (auto& row : c->gprof_cnt)
    for (int& n : row) n = 0;
  c->graph_mask = c->prof_mask;
}

// After a replay of the graph in `slot` has finished: its timed launches into the totals.
inline void gprof_collect(gbmg_ctx* c, int slot) {
  for (int f = 1; f < 8; ++f)
    for (int k = 0; k < c->gprof_cnt[slot][f]; ++k) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, c->gprof_ev[slot][f][k][0], c->gprof_ev[slot][f][k][1]) == cudaSuccess) {
        c->prof_gms[f] += t;
        c->prof_gn[f] += 1;
      } else {
        (void)cudaGetLastError();  // not counted; leaves no error behind for later launches
      }
    }
}

// Captures the launches `body` makes on c->stream into a CUDA graph, on the context's
// private capture stream (the caller's may be the legacy default stream, which cannot be
// captured), and instantiates it into `exec`; nothing runs.  The recorded launches are
// taken off the launch count and their number goes to `kernels`.  If capturing or
// instantiating fails, `exec` stays null and the context is switched to eager launches.
template <class Body>
gbmg_status capture_graph(gbmg_ctx* c, int slot, Body body, cudaGraphExec_t& exec, long long& kernels) {
  if (!c->cap_stream) TRY(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
  cudaStream_t user = c->stream;
  const long long k0 = launch_count();
  cudaGraph_t g = nullptr;
  c->stream = c->cap_stream;
  for (int& n : c->gprof_cnt[slot]) n = 0;
  c->cap_slot = slot;
  cudaError_t e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
  gbmg_status s = GBMG_OK;
  if (e == cudaSuccess) {
    s = body();
    const cudaError_t e2 = cudaStreamEndCapture(c->cap_stream, &g);
    if (e2 != cudaSuccess) e = e2;
  }
  c->cap_slot = -1;
  c->stream = user;
  const long long nk = launch_count() - k0;
  note_launches(-nk);
  cudaGraphExec_t x = nullptr;
  if (e == cudaSuccess && s == GBMG_OK && g) e = cudaGraphInstantiate(&x, g, 0);
  if (g) cudaGraphDestroy(g);
  if (e != cudaSuccess || s != GBMG_OK || !x) {
    (void)cudaGetLastError();
    c->cyc_off = true;
    return GBMG_OK;
  }
  exec = x;
  kernels = nk;
  return GBMG_OK;
}

// The relative residual from the scalars a cycle copied to pinned host memory, after
// waiting for the stream.
inline gbmg_status rel_from_host(gbmg_ctx* c, double& rel) {
  TRY(cudaStreamSynchronize(c->stream));
  const double f2 = c->host_scal[S_F2], r2 = c->host_scal[S_R2];
  rel = f2 > 0.0 ? std::sqrt(r2 / f2) : std::sqrt(r2);
  return GBMG_OK;
}

// Reads ||F||^2 and ||r||^2 back and returns the relative residual.
inline gbmg_status read_rel(gbmg_ctx* c, double& rel) {
  TRY(launch_scalars_to_host(c->stream, c->scal, c->host_scal_dev, 8));
  TRY(cudaStreamSynchronize(c->stream));
  const double f2 = c->host_scal[S_F2], r2 = c->host_scal[S_R2];
  rel = f2 > 0.0 ? std::sqrt(r2 / f2) : std::sqrt(r2);
  return GBMG_OK;
}

}  // namespace gbmg
