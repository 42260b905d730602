// CPU check driver for the library's host-side numerics (host_math.cpp), built with a
// plain C++ compiler by tests/test_host_math.py.  Reads commands on stdin and writes
// one line of numbers per command on stdout:
//   levels nx ny nz L              -> nx ny nz of every level, finest first
//   cheb degree alpha              -> c1[0..degree-1] then c2[0..degree-1]
//   flat nx ny nz h                -> the dense operator, row-major
//   pinv n w[0..n-1] L[0..n*n-1]   -> 1 and G row-major, or 0 when singular
//   monitor tol maxv k r[0..k-1]   -> status cycles rel_res0 rel_res res_hist[0..cycles-1] of
//                                     the solve loop's bookkeeping fed the residuals r[0], r[1], ...
#include <cstdio>
#include <cstdlib>
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
    } else if (cmd == "monitor") {
      double tol;
      int maxv, k;
      std::cin >> tol >> maxv >> k;
      std::vector<double> r(k);
      for (double& x : r) {
        std::string t;
        std::cin >> t;
        x = std::strtod(t.c_str(), nullptr);  // accepts nan and inf
      }
      gbmg_stats st{};
      gbmg::Monitor mon(st, tol, maxv);
      mon.start(r[0]);
      // the solve loops: one V-cycle per pass, then the residual it left
      for (int i = 1; !mon.done() && i < k; ++i)
        if (mon.record(r[i])) break;
      std::printf("%d %d %.17g %.17g ", (int)st.status, st.cycles, st.rel_res0, st.rel_res);
      for (int i = 0; i < st.cycles && i < 64; ++i) std::printf("%.17g ", st.res_hist[i]);
    } else {
      std::fprintf(stderr, "unknown command %s\n", cmd.c_str());
      return 2;
    }
    std::printf("\n");
  }
  return 0;
}
