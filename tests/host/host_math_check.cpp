// CPU check driver for the library's host-side numerics (host_math.cpp), built with a
// plain C++ compiler by tests/test_host_math.py.  Reads commands on stdin and writes
// one line of numbers per command on stdout:
//   levels nx ny nz L              -> nx ny nz of every level, finest first
//   cheb degree alpha              -> c1[0..degree-1] then c2[0..degree-1]
//   flat nx ny nz h                -> the dense operator, row-major
//   pinv n w[0..n-1] L[0..n*n-1]   -> 1 and G row-major, or 0 when singular
#include <cstdio>
#include <iostream>
#include <string>
#include <vector>

#include "host_math.h"

static void put(const std::vector<double>& v) {
  for (double x : v) std::printf("%.17g ", x);
}

int main() {
  std::string cmd;
  while (std::cin >> cmd) {
    if (cmd == "levels") {
      int nx, ny, nz, L;
      std::cin >> nx >> ny >> nz >> L;
      for (const gbmg::Dims& d : gbmg::level_dims(nx, ny, nz, L)) std::printf("%d %d %d ", d.nx, d.ny, d.nz);
    } else if (cmd == "cheb") {
      int degree;
      double alpha;
      std::cin >> degree >> alpha;
      std::vector<double> c1, c2;
      gbmg::chebyshev_schedule(degree, alpha, c1, c2);
      put(c1);
      put(c2);
    } else if (cmd == "flat") {
      int nx, ny, nz;
      double h;
      std::cin >> nx >> ny >> nz >> h;
      put(gbmg::dense_flat(gbmg::Dims{nx, ny, nz}, h));
    } else if (cmd == "pinv") {
      int n;
      std::cin >> n;
      std::vector<double> w(n), L((size_t)n * n), G;
      for (double& x : w) std::cin >> x;
      for (double& x : L) std::cin >> x;
      const bool ok = gbmg::dense_pinv(n, L, w, G);
      std::printf("%d ", ok ? 1 : 0);
      if (ok) put(G);
    } else {
      std::fprintf(stderr, "unknown command %s\n", cmd.c_str());
      return 2;
    }
    std::printf("\n");
  }
  return 0;
}
