/* Plain FP64 geometric-multigrid solve of the periodic 7-point Poisson problem, in C.
 *
 * TEST INFRASTRUCTURE (the CPU oracle, timed as the CPU baseline).  Only tests/,
 * __graft_entry__.smoke() and bench.py's CPU legs may load it; it shares no code with
 * the CUDA library.  It restates oracle/flat.py's V-cycle in C so that the oracle can
 * run a full 512^3 solve on a machine's host cores in seconds:
 *
 *   Sec. 2.1, Eq. (linsys): A u = (sum of the 6 face neighbours - 6 u) / h^2, periodic;
 *     F mean-projected, the solution fixed to zero mean (gauge).
 *   Sec. 2.3, Eq. (flat_chebyshev): Chebyshev semi-iteration on D^-1 A, D = -6/h^2, over
 *     [2/alpha, 2], `degree` operator applications per smoothing pass (the reading of the
 *     degree taken by the oracle: v applications, error factor T_v((theta-mu)/delta) /
 *     T_v(theta/delta)).
 *   Sec. 2.3 + Appendix B: residual, full-weighting restriction ([1/4, 1/2, 1/4] per
 *     axis, coarse node I on fine node 2I), V-cycle recursion on rediscretised levels
 *     (h_l = 2^l), trilinear prolongation and correction, post-smoothing.
 *   Sec. 2.3 "directly on the coarsest level": the exact minimum-norm solve, written as
 *     the periodic convolution e = G * (r - mean r) with
 *     G(d) = (1/n) sum_{k != 0} cos(k . d) / lambda(k),
 *     lambda(k) = (2 cos kx + 2 cos ky + 2 cos kz - 6) / h^2 (Eq. fftsolve's symbol).
 *   Levels: halve while every side is even and its half is >= 4.
 *
 * Every operation is its own loop over the mesh in the order of the algorithm, no
 * fusion or blocking; loops over z planes run in parallel with OpenMP (each cell is
 * computed the same way whatever the thread count) and every norm or mean is the
 * plane sums added in plane order, so results do not depend on the thread count.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define MAXLEV 24

typedef struct {
  int nx, ny, nz;
} dims_t;

typedef struct {
  dims_t d;
  double h;
  double *r, *e, *z, *dv, *t; /* right-hand side, iterate, Jacobi residual, direction, scratch */
} level_t;

typedef struct {
  int nlev, degree;
  double alpha;
  level_t lv[MAXLEV];
  double* G;      /* coarsest Green's function, n values */
  double* plane;  /* per-plane partial sums (finest nz) */
  double norm_f;  /* ||F - m|| of the solve in progress */
} ora_ctx;

static long long ncell(dims_t d) { return (long long)d.nx * d.ny * d.nz; }
static int wrap(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }
static long long at(dims_t d, int x, int y, int z) {
  return ((long long)wrap(z, d.nz) * d.ny + wrap(y, d.ny)) * d.nx + wrap(x, d.nx);
}

int ora_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* out = A u (7-point, spacing h) */
static void apply_A(dims_t d, double h, const double* u, double* out) {
  const double ih2 = 1.0 / (h * h);
  const long long sy = d.nx, sz = (long long)d.nx * d.ny;
#pragma omp parallel for schedule(static)
  for (int z = 0; z < d.nz; ++z) {
    const long long zo = z * sz, zm = wrap(z - 1, d.nz) * sz, zp = wrap(z + 1, d.nz) * sz;
    for (int y = 0; y < d.ny; ++y) {
      const long long yo = y * sy, ym = wrap(y - 1, d.ny) * sy, yp = wrap(y + 1, d.ny) * sy;
      for (int x = 0; x < d.nx; ++x) {
        const int xm = wrap(x - 1, d.nx), xp = wrap(x + 1, d.nx);
        const double c = u[zo + yo + x];
        const double s = u[zo + yo + xm] + u[zo + yo + xp] + u[zo + ym + x] + u[zo + yp + x] + u[zm + yo + x] +
                         u[zp + yo + x];
        out[zo + yo + x] = (s - 6.0 * c) * ih2;
      }
    }
  }
}

/* out = f - A u */
static void residual(dims_t d, double h, const double* f, const double* u, double* out) {
  apply_A(d, h, u, out);
  const long long n = ncell(d);
#pragma omp parallel for schedule(static)
  for (long long i = 0; i < n; ++i) out[i] = f[i] - out[i];
}

/* sum of u (or of u^2) over the mesh: plane sums, added in plane order */
static double mesh_sum(dims_t d, const double* u, int squares, double* plane) {
  const long long np = (long long)d.nx * d.ny;
#pragma omp parallel for schedule(static)
  for (int z = 0; z < d.nz; ++z) {
    double s = 0.0;
    const double* p = u + (long long)z * np;
    for (long long i = 0; i < np; ++i) s += squares ? p[i] * p[i] : p[i];
    plane[z] = s;
  }
  double s = 0.0;
  for (int z = 0; z < d.nz; ++z) s += plane[z];
  return s;
}

/* coarse rc = full weighting of fine r: weights w(a) w(b) w(c), w(0) = 1/2, w(+-1) = 1/4 */
static void restrict_fw(dims_t d, const double* r, double* rc) {
  const dims_t c = {d.nx / 2, d.ny / 2, d.nz / 2};
  static const double w[3] = {0.25, 0.5, 0.25};
#pragma omp parallel for schedule(static)
  for (int Z = 0; Z < c.nz; ++Z)
    for (int Y = 0; Y < c.ny; ++Y)
      for (int X = 0; X < c.nx; ++X) {
        double s = 0.0;
        for (int k = -1; k <= 1; ++k)
          for (int j = -1; j <= 1; ++j)
            for (int i = -1; i <= 1; ++i)
              s += w[k + 1] * w[j + 1] * w[i + 1] * r[at(d, 2 * X + i, 2 * Y + j, 2 * Z + k)];
        rc[at(c, X, Y, Z)] = s;
      }
}

/* e += P ec: fine node 2I + s (s in {0,1}^3) takes the mean of the coarse nodes I + s'
 * with s' <= s componentwise (trilinear, vertex-centred) */
static void prolong_add(dims_t d, const double* ec, double* e) {
  const dims_t c = {d.nx / 2, d.ny / 2, d.nz / 2};
#pragma omp parallel for schedule(static)
  for (int z = 0; z < d.nz; ++z)
    for (int y = 0; y < d.ny; ++y)
      for (int x = 0; x < d.nx; ++x) {
        const int X = x / 2, Y = y / 2, Z = z / 2, sx = x % 2, sy = y % 2, sz = z % 2;
        double s = 0.0;
        int cnt = 0;
        for (int k = 0; k <= sz; ++k)
          for (int j = 0; j <= sy; ++j)
            for (int i = 0; i <= sx; ++i) {
              s += ec[at(c, X + i, Y + j, Z + k)];
              ++cnt;
            }
        e[at(d, x, y, z)] += s / cnt;
      }
}

/* Chebyshev smoothing of A e = r (Eq. flat_chebyshev; Saad, Iterative Methods for
 * Sparse Linear Systems, 2nd ed., Alg. 12.1, on D^-1 A) */
static void smooth_cheb(level_t* L, int degree, double alpha) {
  const dims_t d = L->d;
  const long long n = ncell(d);
  const double a = 2.0 / alpha, b = 2.0, theta = 0.5 * (a + b), delta = 0.5 * (b - a), sigma = theta / delta;
  const double Dinv = -(L->h * L->h) / 6.0;
  residual(d, L->h, L->r, L->e, L->z);
#pragma omp parallel for schedule(static)
  for (long long i = 0; i < n; ++i) L->dv[i] = (Dinv * L->z[i]) / theta;
  double rho = 1.0 / sigma;
  for (int it = 1; it <= degree; ++it) {
#pragma omp parallel for schedule(static)
    for (long long i = 0; i < n; ++i) L->e[i] += L->dv[i];
    if (it < degree) {
      residual(d, L->h, L->r, L->e, L->z);
      const double rho_new = 1.0 / (2.0 * sigma - rho);
      const double c1 = rho_new * rho, c2 = 2.0 * rho_new / delta;
#pragma omp parallel for schedule(static)
      for (long long i = 0; i < n; ++i) L->dv[i] = c1 * L->dv[i] + c2 * (Dinv * L->z[i]);
      rho = rho_new;
    }
  }
}

/* coarsest level: e = G * (r - mean r) */
static void coarse_solve(ora_ctx* C, level_t* L) {
  const dims_t d = L->d;
  const long long n = ncell(d);
  double m = 0.0;
  for (long long i = 0; i < n; ++i) m += L->r[i];
  m /= (double)n;
  for (int z = 0; z < d.nz; ++z)
    for (int y = 0; y < d.ny; ++y)
      for (int x = 0; x < d.nx; ++x) {
        double s = 0.0;
        for (int zz = 0; zz < d.nz; ++zz)
          for (int yy = 0; yy < d.ny; ++yy)
            for (int xx = 0; xx < d.nx; ++xx)
              s += C->G[at(d, x - xx, y - yy, z - zz)] * (L->r[at(d, xx, yy, zz)] - m);
        L->e[at(d, x, y, z)] = s;
      }
}

/* V-cycle for A_l e = r on level l, e holding the initial iterate */
static void vcycle(ora_ctx* C, int l) {
  level_t* L = &C->lv[l];
  if (l == C->nlev - 1) {
    coarse_solve(C, L);
    return;
  }
  level_t* Lc = &C->lv[l + 1];
  smooth_cheb(L, C->degree, C->alpha);
  residual(L->d, L->h, L->r, L->e, L->t);
  restrict_fw(L->d, L->t, Lc->r);
  memset(Lc->e, 0, (size_t)ncell(Lc->d) * sizeof(double));
  vcycle(C, l + 1);
  prolong_add(L->d, Lc->e, L->e);
  smooth_cheb(L, C->degree, C->alpha);
}

void ora_destroy(ora_ctx* C) {
  if (!C) return;
  for (int l = 0; l < C->nlev; ++l) {
    free(C->lv[l].r);
    free(C->lv[l].e);
    free(C->lv[l].z);
    free(C->lv[l].dv);
    free(C->lv[l].t);
  }
  free(C->G);
  free(C->plane);
  free(C);
}

/* Set up the hierarchy of an nx x ny x nz mesh (levels: 0 = as many as the ladder allows).
 * Returns NULL on invalid sizes or when the coarsest level exceeds 4096 cells. */
ora_ctx* ora_create(int nx, int ny, int nz, int levels, int degree, double alpha) {
  if (nx < 3 || ny < 3 || nz < 3 || degree < 1 || !(alpha > 1.0)) return NULL;
  ora_ctx* C = (ora_ctx*)calloc(1, sizeof(ora_ctx));
  if (!C) return NULL;
  C->degree = degree;
  C->alpha = alpha;
  dims_t d = {nx, ny, nz};
  for (;;) {
    level_t* L = &C->lv[C->nlev];
    L->d = d;
    L->h = ldexp(1.0, C->nlev);
    const size_t b = (size_t)ncell(d) * sizeof(double);
    L->r = (double*)calloc(1, b);
    L->e = (double*)calloc(1, b);
    L->z = (double*)calloc(1, b);
    L->dv = (double*)calloc(1, b);
    L->t = (double*)calloc(1, b);
    C->nlev++;
    if (!L->r || !L->e || !L->z || !L->dv || !L->t) {
      ora_destroy(C);
      return NULL;
    }
    if ((levels > 0 && C->nlev >= levels) || C->nlev >= MAXLEV) break;
    if (d.nx % 2 || d.ny % 2 || d.nz % 2 || d.nx / 2 < 4 || d.ny / 2 < 4 || d.nz / 2 < 4) break;
    d.nx /= 2;
    d.ny /= 2;
    d.nz /= 2;
  }
  const level_t* Lc = &C->lv[C->nlev - 1];
  const long long nc = ncell(Lc->d);
  C->plane = (double*)calloc((size_t)nz, sizeof(double));
  if (nc > 4096 || !C->plane) {
    ora_destroy(C);
    return NULL;
  }
  /* G(d) = (1/n) sum_{k != 0} cos(k . d) / lambda(k) */
  C->G = (double*)calloc((size_t)nc, sizeof(double));
  if (!C->G) {
    ora_destroy(C);
    return NULL;
  }
  const dims_t c = Lc->d;
  const double pi = acos(-1.0), ih2 = 1.0 / (Lc->h * Lc->h);
  for (int dz = 0; dz < c.nz; ++dz)
    for (int dy = 0; dy < c.ny; ++dy)
      for (int dx = 0; dx < c.nx; ++dx) {
        double s = 0.0;
        for (int kz = 0; kz < c.nz; ++kz)
          for (int ky = 0; ky < c.ny; ++ky)
            for (int kx = 0; kx < c.nx; ++kx) {
              if (kx == 0 && ky == 0 && kz == 0) continue;
              const double ax = 2.0 * pi * kx / c.nx, ay = 2.0 * pi * ky / c.ny, az = 2.0 * pi * kz / c.nz;
              const double lam = (2.0 * cos(ax) + 2.0 * cos(ay) + 2.0 * cos(az) - 6.0) * ih2;
              s += cos(ax * dx + ay * dy + az * dz) / lam;
            }
        C->G[at(c, dx, dy, dz)] = s / (double)nc;
      }
  return C;
}

int ora_levels(const ora_ctx* C) { return C ? C->nlev : 0; }

/* One V-cycle on the error equation A e = r of the finest level from e = 0. */
void ora_vcycle(ora_ctx* C, const double* r, double* e_out) {
  level_t* L = &C->lv[0];
  const size_t b = (size_t)ncell(L->d) * sizeof(double);
  memcpy(L->r, r, b);
  memset(L->e, 0, b);
  vcycle(C, 0);
  memcpy(e_out, L->e, b);
}

/* The solve of A phi = F - mean(F) from a warm start, in three calls, each V-cycle applied
 * to the iterate itself (e = phi, r = F - m):
 *   ora_begin: r = F - m, e = phi_in; returns ||r - A e|| / ||r||;
 *   ora_cycle: one V-cycle on e; returns the new relative residual;
 *   ora_end:   phi_out = e - mean(e) (the gauge). */
double ora_begin(ora_ctx* C, const double* F, const double* phi_in) {
  level_t* L = &C->lv[0];
  const dims_t d = L->d;
  const long long n = ncell(d);
  const double m = mesh_sum(d, F, 0, C->plane) / (double)n;
#pragma omp parallel for schedule(static)
  for (long long i = 0; i < n; ++i) {
    L->r[i] = F[i] - m;
    L->e[i] = phi_in[i];
  }
  C->norm_f = sqrt(mesh_sum(d, L->r, 1, C->plane));
  residual(d, L->h, L->r, L->e, L->t);
  return sqrt(mesh_sum(d, L->t, 1, C->plane)) / C->norm_f;
}

double ora_cycle(ora_ctx* C) {
  level_t* L = &C->lv[0];
  vcycle(C, 0);
  residual(L->d, L->h, L->r, L->e, L->t);
  return sqrt(mesh_sum(L->d, L->t, 1, C->plane)) / C->norm_f;
}

void ora_end(ora_ctx* C, double* phi_out) {
  level_t* L = &C->lv[0];
  const long long n = ncell(L->d);
  const double pm = mesh_sum(L->d, L->e, 0, C->plane) / (double)n;
#pragma omp parallel for schedule(static)
  for (long long i = 0; i < n; ++i) phi_out[i] = L->e[i] - pm;
}

/* Until ||F - m - A phi|| / ||F - m|| <= tol or max_cycles V-cycles.  hist (max_cycles + 1
 * doubles, nullable) receives the relative residual before the first and after every
 * cycle.  phi_inout: the warm start in, the solution (mean removed) out.  Returns the
 * number of cycles run. */
int ora_solve(ora_ctx* C, const double* F, double* phi_inout, double tol, int max_cycles, double* hist) {
  double rel = ora_begin(C, F, phi_inout);
  if (hist) hist[0] = rel;
  int cycles = 0;
  while (cycles < max_cycles && !(rel <= tol)) {
    rel = ora_cycle(C);
    ++cycles;
    if (hist) hist[cycles] = rel;
  }
  ora_end(C, phi_inout);
  return cycles;
}

/* Component entry points for the pins: out = A u at spacing h; one Chebyshev smoothing
 * pass of A e = r in place on e. */
void ora_apply(int nx, int ny, int nz, double h, const double* u, double* out) {
  const dims_t d = {nx, ny, nz};
  apply_A(d, h, u, out);
}

int ora_smooth_cheb(int nx, int ny, int nz, double h, int degree, double alpha, double* e, const double* r) {
  level_t L;
  L.d.nx = nx;
  L.d.ny = ny;
  L.d.nz = nz;
  L.h = h;
  const size_t b = (size_t)ncell(L.d) * sizeof(double);
  L.r = (double*)r;
  L.e = e;
  L.z = (double*)malloc(b);
  L.dv = (double*)malloc(b);
  L.t = NULL;
  if (!L.z || !L.dv) {
    free(L.z);
    free(L.dv);
    return 1;
  }
  smooth_cheb(&L, degree, alpha);
  free(L.z);
  free(L.dv);
  return 0;
}

/* Thread count of the OpenMP loops (results do not depend on it). */
void ora_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}
