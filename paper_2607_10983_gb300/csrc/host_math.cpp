// Host-side numerics of the hierarchy set-up (declared in host_math.h).
#include "host_math.h"

#include <cmath>
#include <utility>

namespace gbmg {

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
