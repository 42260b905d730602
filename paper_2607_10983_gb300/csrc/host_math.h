// Host-side numerics of the hierarchy set-up, in plain C++ (no CUDA): the mesh
// dimensions type, the level ladder, the dense operator of a coarsest level and its
// minimum-norm inverse, the Chebyshev coefficient schedule, and the convergence
// monitor of the solve loops.  Compiled into the library and, by the CPU tests, on
// its own.
#pragma once
#include <cmath>
#include <vector>

#include "gbmg.h"

namespace gbmg {

struct Dims {
  int nx, ny, nz;
};

// Finest level first; each next level halves every side while all sides are even and
// the halves are >= 4 (Sec. 4.3.3), at most `levels` levels (0: no limit).
std::vector<Dims> level_dims(int nx, int ny, int nz, int levels);
// Minimum-norm inverse G (n x n, row-major) of a singular operator L with null space
// span(1) and left null space span(w): L G r = r - w (w.r) / (w.w), 1^T G r = 0.
// False when the bordered system is singular.
bool dense_pinv(int n, const std::vector<double>& Lm, const std::vector<double>& w, std::vector<double>& G);
// Dense periodic 7-point operator (row-major, x fastest) of a level with spacing h.
std::vector<double> dense_flat(Dims d, double h);
// Coefficients of the Chebyshev semi-iteration on [2/alpha, 2] (Sec. 2.3), degree steps.
void chebyshev_schedule(int degree, double alpha, std::vector<double>& c1, std::vector<double>& c2);

// Convergence bookkeeping shared by the solve drivers: stop at tol, at max_vcycles,
// on a non-finite residual, or when the residual grew tenfold over two cycles.
struct Monitor {
  gbmg_stats& st;
  double tol;
  int maxv;
  std::vector<double> hist;  // hist[k] = relative residual after k cycles
  Monitor(gbmg_stats& s, double t, int m) : st(s), tol(t), maxv(m) {}
  void start(double rel) {
    st.rel_res0 = rel;
    st.rel_res = rel;
    st.cycles = 0;
    st.status = GBMG_OK;
    hist.assign(1, rel);
  }
  bool done() {
    if (!std::isfinite(st.rel_res)) {
      st.status = GBMG_ERR_NONFINITE;
      return true;
    }
    if (st.rel_res <= tol) return true;
    if (st.cycles >= maxv) {
      st.status = GBMG_ERR_NOT_CONVERGED;
      return true;
    }
    return false;
  }
  // record the residual after one more cycle; true if the solve must stop (diverged)
  bool record(double rel) {
    if (st.cycles < 64) st.res_hist[st.cycles] = rel;
    st.cycles += 1;
    st.rel_res = rel;
    hist.push_back(rel);
    const size_t k = hist.size() - 1;
    if (k >= 2 && std::isfinite(rel) && rel > 10.0 * hist[k - 2]) {
      st.status = GBMG_ERR_DIVERGED;
      return true;
    }
    return false;
  }
};

}  // namespace gbmg
