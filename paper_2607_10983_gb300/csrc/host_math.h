// Host-side numerics of the hierarchy set-up, in plain C++ (no CUDA): the mesh
// dimensions type, the level ladder, the dense operator of a coarsest level and its
// minimum-norm inverse, and the Chebyshev coefficient schedule.  Compiled into the
// library and, by the CPU tests, on its own.
#pragma once
#include <vector>

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

}  // namespace gbmg
