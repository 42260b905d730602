// Internal definition of the solver context shared by the host translation units.
#pragma once
#include <string>
#include <vector>

#include "common.cuh"
#include "gbmg.h"

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
};

gbmg_status fail(gbmg_status s, const std::string& msg);
gbmg_status cuda_fail(cudaError_t e, const char* what);
extern thread_local std::string g_last_error;

std::vector<Dims> level_dims(int nx, int ny, int nz, int levels);
bool dense_pinv(int n, const std::vector<double>& Lm, const std::vector<double>& w, std::vector<double>& G);
std::vector<double> dense_flat(Dims d, double h);
void chebyshev_schedule(int degree, double alpha, std::vector<double>& c1, std::vector<double>& c2);

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
  float2* F_df = nullptr;       // mixed precision: source as double-float
  float2* phi_df = nullptr;     // mixed precision: potential as double-float
  float2* phi_df2 = nullptr;    // mixed precision: second potential buffer (fused update)
  float* r_alt = nullptr;       // mixed precision: second finest residual buffer
  double* partials = nullptr;   // 4 regions of npart block partial sums
  long long npart = 0;
  double* scal = nullptr;       // 64 device scalars (enum Scal)
  double* host_scal = nullptr;  // 64 pinned host scalars
  std::vector<double> cc1, cc2; // Chebyshev schedule
  gbmg_stats last{};
  std::vector<void*> owned;     // lazily allocated buffers (component scratch, staging)
  void* comp_scratch[2] = {nullptr, nullptr};  // per dtype: 2 finest-level fields
  int prof_mask = 0;            // bit (1 << gbmg_prof_family) set = family timed
  int prof_n[8] = {0};          // timed launches per family
  std::vector<cudaEvent_t> prof_ev[8];  // start/stop event pairs per family
  double* stage_F = nullptr;    // mg_solve_host device staging
  double* stage_phi = nullptr;
  ~gbmg_ctx();
};
