// Moving-mesh (curvilinear) operator kernels (Sec. 4.2-4.3, Appendix B).
//
// Geometry per level (Sec. 4.2, Eq. triad and Eq. metric): A = I + Hess psi with
// second-order central differences (mixed terms by the four-point 1/(4h^2)
// stencil), J = sqrt(g) = det A and B = sqrt(g) g^-1 = J A^-2 = adj(A)^2 / J.
// Built in double-float arithmetic (about 48 bits) from the FP64 psi of the level,
// stored as FP32 (J and the six components of the symmetric B).
//
// Operator (Sec. 4.3.1): (M u)_i = sum_a (F^a_{i+1/2} - F^a_{i-1/2}) / h with face
// fluxes F^a = sum_b B^{ab}_face G_b, B_face the mean of the two adjacent cells,
// G_a the two-point normal difference and G_b (b != a) the central differences of
// the two adjacent cells averaged onto the face.  L = M / J is the operator the
// V-cycle solves (Eq. curv_linsys); the transposed solve of the adjoint uses the
// exact transpose M^T (by summation by parts) with the same 1/J.
//
// Symmetric variant S (an option; not the paper's scheme): the same B^{aa} face terms,
// the cross terms on the cell edges, -sum_{a != b} E_a^T C_ab E_b, C_ab the mean of B^{ab}
// over the edge's four cells and E_a the a-difference averaged over the edge's two
// b-positions.  S = S^T; it is its own transpose in the adjoint.
//
// Operator form of a launch: 0 = M, 1 = M^T, 2 = S.
#include <cmath>

#include "kernels.h"
#include "stencil.cuh"

namespace gbmg {

namespace {

constexpr int BX = 32, BY = 8;
inline dim3 cell_grid(Dims d) { return dim3((d.nx + BX - 1) / BX, (d.ny + BY - 1) / BY, d.nz); }

// component index of B^{ab} in the packed symmetric layout xx, yy, zz, xy, xz, yz
__host__ __device__ constexpr int bidx(int a, int b) {
  return a == b ? a : (a + b == 1 ? 3 : (a + b == 2 ? 4 : 5));
}

// 3x3x3 neighbourhood of a cell with periodic wrap: idx(dx, dy, dz), d* in {-1, 0, 1}.
struct Nbhd {
  long long zo[3];
  int yo[3];
  int xo[3];
  __device__ __forceinline__ Nbhd(Dims d, int x, int y, int z) {
    const long long pst = (long long)d.nx * d.ny;
    xo[0] = wrapi(x - 1, d.nx);
    xo[1] = x;
    xo[2] = wrapi(x + 1, d.nx);
    yo[0] = wrapi(y - 1, d.ny) * d.nx;
    yo[1] = y * d.nx;
    yo[2] = wrapi(y + 1, d.ny) * d.nx;
    zo[0] = (long long)wrapi(z - 1, d.nz) * pst;
    zo[1] = (long long)z * pst;
    zo[2] = (long long)wrapi(z + 1, d.nz) * pst;
  }
  // offset of the cell displaced by (dx, dy, dz)
  __device__ __forceinline__ long long operator()(int dx, int dy, int dz) const {
    return zo[dz + 1] + yo[dy + 1] + xo[dx + 1];
  }
};

// displacement of unit vector a (0 = x, 1 = y, 2 = z) scaled by s, added to (dx, dy, dz)
__device__ __forceinline__ void shift(int a, int s, int& dx, int& dy, int& dz) {
  if (a == 0) dx += s;
  else if (a == 1) dy += s;
  else dz += s;
}

// Face coefficient B^{ab} on the a-face between the cell at offset c and c + e_a.
template <typename T, typename BF>
__device__ __forceinline__ T face_B(const BF& Bc, int a, int b, int cx, int cy, int cz) {
  int px = cx, py = cy, pz = cz;
  shift(a, 1, px, py, pz);
  return T(0.5) * (T(Bc(bidx(a, b), cx, cy, cz)) + T(Bc(bidx(a, b), px, py, pz)));
}

// h * (flux F^a on the face between offset c and c + e_a), plain arithmetic in T.
template <typename T, typename UF, typename BF>
__device__ __forceinline__ T face_flux(const UF& u, const BF& Bc, int a, int cx, int cy, int cz) {
  int px = cx, py = cy, pz = cz;
  shift(a, 1, px, py, pz);
  T f = face_B<T>(Bc, a, a, cx, cy, cz) * (u(px, py, pz) - u(cx, cy, cz));
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    if (b == a) continue;
    int c1x = cx, c1y = cy, c1z = cz, c2x = cx, c2y = cy, c2z = cz;
    shift(b, 1, c1x, c1y, c1z);
    shift(b, -1, c2x, c2y, c2z);
    int d1x = px, d1y = py, d1z = pz, d2x = px, d2y = py, d2z = pz;
    shift(b, 1, d1x, d1y, d1z);
    shift(b, -1, d2x, d2y, d2z);
    const T tang = T(0.25) * ((u(c1x, c1y, c1z) - u(c2x, c2y, c2z)) + (u(d1x, d1y, d1z) - u(d2x, d2y, d2z)));
    f += face_B<T>(Bc, a, b, cx, cy, cz) * tang;
  }
  return f;
}

// h^2 (M u) at the centre cell.
template <typename T, typename UF, typename BF>
__device__ __forceinline__ T apply_M_h2(const UF& u, const BF& Bc) {
  T out = T(0);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    int mx = 0, my = 0, mz = 0;
    shift(a, -1, mx, my, mz);
    out += face_flux<T>(u, Bc, a, 0, 0, 0) - face_flux<T>(u, Bc, a, mx, my, mz);
  }
  return out;
}

// h^2 (M^T y) at the centre cell j, from <y, M x> = sum_a sum_i h F^a[x]_i (y_i - y_{i+a}) / h^2:
// q_ab(c) = B^{ab}_face(c) (y_c - y_{c+a});  M^T y = sum_a [q_aa(j-a) - q_aa(j)]
//   + sum_{b != a} [(q_ab(j-b) - q_ab(j+b)) + (q_ab(j-a-b) - q_ab(j-a+b))] / 4.
template <typename T, typename UF, typename BF>
__device__ __forceinline__ T apply_MT_h2(const UF& y, const BF& Bc) {
  auto q = [&](int a, int b, int cx, int cy, int cz) -> T {
    int px = cx, py = cy, pz = cz;
    shift(a, 1, px, py, pz);
    return face_B<T>(Bc, a, b, cx, cy, cz) * (y(cx, cy, cz) - y(px, py, pz));
  };
  T out = T(0);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    int ax = 0, ay = 0, az = 0;
    shift(a, -1, ax, ay, az);  // j - a
    out += q(a, a, ax, ay, az) - q(a, a, 0, 0, 0);
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      if (b == a) continue;
      int m1x = 0, m1y = 0, m1z = 0, p1x = 0, p1y = 0, p1z = 0;
      shift(b, -1, m1x, m1y, m1z);
      shift(b, 1, p1x, p1y, p1z);
      int m2x = ax, m2y = ay, m2z = az, p2x = ax, p2y = ay, p2z = az;
      shift(b, -1, m2x, m2y, m2z);
      shift(b, 1, p2x, p2y, p2z);
      out += T(0.25) * ((q(a, b, m1x, m1y, m1z) - q(a, b, p1x, p1y, p1z)) +
                        (q(a, b, m2x, m2y, m2z) - q(a, b, p2x, p2y, p2z)));
    }
  }
  return out;
}

// h^2 times the diagonal of M (and of M^T): -sum_a (B^{aa}_{+face} + B^{aa}_{-face}) (Appendix B).
template <typename T, typename BF>
__device__ __forceinline__ T diag_M_h2(const BF& Bc) {
  T d = T(0);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    int mx = 0, my = 0, mz = 0;
    shift(a, -1, mx, my, mz);
    d -= face_B<T>(Bc, a, a, 0, 0, 0) + face_B<T>(Bc, a, a, mx, my, mz);
  }
  return d;
}

// Edge coefficient C_ab of the ab-edge at c + (e_a + e_b)/2: mean of B^{ab} over its four cells.
template <typename T, typename BF>
__device__ __forceinline__ T edge_B(const BF& Bc, int a, int b, int cx, int cy, int cz) {
  int ax = cx, ay = cy, az = cz, bx = cx, by = cy, bz = cz;
  shift(a, 1, ax, ay, az);
  shift(b, 1, bx, by, bz);
  int px = ax, py = ay, pz = az;
  shift(b, 1, px, py, pz);
  const int k = bidx(a, b);
  return T(0.25) * ((T(Bc(k, cx, cy, cz)) + T(Bc(k, ax, ay, az))) + (T(Bc(k, bx, by, bz)) + T(Bc(k, px, py, pz))));
}

// Offsets of the four edges around the centre cell in the ab-plane and of the edge
// neighbour each couples to: edge k has its base at -a (k & 1), -b (k & 2); the
// neighbour is at (k & 1 ? -a : +a) + (k & 2 ? -b : +b).  -(E_a^T C E_b + E_b^T C E_a) u
// at the centre is (1/2) sum_k sgn_k C(edge k) (u(nbr k) - u_0), sgn = +1 for k = 0, 3
// and -1 for k = 1, 2 (written out from the two transposed edge differences).
__device__ __forceinline__ void edge_k(int a, int b, int k, int& ex, int& ey, int& ez, int& nx, int& ny, int& nz) {
  ex = ey = ez = 0;
  if (k & 1) shift(a, -1, ex, ey, ez);
  if (k & 2) shift(b, -1, ex, ey, ez);
  nx = ny = nz = 0;
  shift(a, (k & 1) ? -1 : 1, nx, ny, nz);
  shift(b, (k & 2) ? -1 : 1, nx, ny, nz);
}

// h^2 (S u) at the centre cell (symmetric variant).
template <typename T, typename UF, typename BF>
__device__ __forceinline__ T apply_S_h2(const UF& u, const BF& Bc) {
  const T u0 = u(0, 0, 0);
  T out = T(0);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    int px = 0, py = 0, pz = 0, mx = 0, my = 0, mz = 0;
    shift(a, 1, px, py, pz);
    shift(a, -1, mx, my, mz);
    out += face_B<T>(Bc, a, a, 0, 0, 0) * (u(px, py, pz) - u0) - face_B<T>(Bc, a, a, mx, my, mz) * (u0 - u(mx, my, mz));
  }
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = a + 1; b < 3; ++b) {
      T c = T(0);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        int ex, ey, ez, nx, ny, nz;
        edge_k(a, b, k, ex, ey, ez, nx, ny, nz);
        const T t = edge_B<T>(Bc, a, b, ex, ey, ez) * (u(nx, ny, nz) - u0);
        c += (k == 1 || k == 2) ? -t : t;
      }
      out += T(0.5) * c;
    }
  return out;
}

// h^2 times the diagonal of S: the face part of diag_M_h2 and, per pair a < b,
// (1/2) (-C(edge 0) + C(edge 1) + C(edge 2) - C(edge 3)).
template <typename T, typename BF>
__device__ __forceinline__ T diag_S_h2(const BF& Bc) {
  T d = diag_M_h2<T>(Bc);
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = a + 1; b < 3; ++b) {
      T c = T(0);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        int ex, ey, ez, nx, ny, nz;
        edge_k(a, b, k, ex, ey, ez, nx, ny, nz);
        const T t = edge_B<T>(Bc, a, b, ex, ey, ez);
        c += (k == 1 || k == 2) ? t : -t;
      }
      d += T(0.5) * c;
    }
  return d;
}

// operator of form 0 / 1 / 2 (M, M^T, S) and its diagonal
template <typename T, typename UF, typename BF>
__device__ __forceinline__ T op_form_h2(const UF& u, const BF& Bc, int form) {
  return form == 2 ? apply_S_h2<T>(u, Bc) : (form == 1 ? apply_MT_h2<T>(u, Bc) : apply_M_h2<T>(u, Bc));
}
template <typename T, typename BF>
__device__ __forceinline__ T diag_form_h2(const BF& Bc, int form) {
  return form == 2 ? diag_S_h2<T>(Bc) : diag_M_h2<T>(Bc);
}

template <typename V>
struct FieldAt {
  const V* __restrict__ p;
  const Nbhd* nb;
  __device__ __forceinline__ V operator()(int dx, int dy, int dz) const { return p[(*nb)(dx, dy, dz)]; }
};

struct CoefAt {
  CurvCoef c;
  const Nbhd* nb;
  __device__ __forceinline__ float operator()(int comp, int dx, int dy, int dz) const {
    return c.B[comp][(*nb)(dx, dy, dz)];
  }
};

template <typename T>
__device__ __forceinline__ T op_h2(const FieldAt<T>& u, const CoefAt& B, int form) {
  return op_form_h2<T>(u, B, form);
}

// ------------------------------------------------------------------ kernels

// out = op(u) / J (divide_J) or op(u), op of the given form
template <typename T>
__global__ void k_curv_apply(Dims d, CurvCoef cf, const T* __restrict__ u, T* __restrict__ out, T inv_h2,
                             int form, int divide_J) {
  const int x = blockIdx.x * BX + threadIdx.x, y = blockIdx.y * BY + threadIdx.y, z = blockIdx.z;
  if (x >= d.nx || y >= d.ny) return;
  const Nbhd nb(d, x, y, z);
  const FieldAt<T> U{u, &nb};
  const CoefAt Bc{cf, &nb};
  const long long i = nb(0, 0, 0);
  T v = op_h2<T>(U, Bc, form) * inv_h2;
  if (divide_J) v /= T(cf.J[i]);
  out[i] = v;
}

// out = r - op(u) / J, with optional block partial sums of out^2
template <typename T>
__global__ void k_curv_residual(Dims d, CurvCoef cf, const T* __restrict__ r, const T* __restrict__ u,
                                T* __restrict__ out, T inv_h2, int form, double* __restrict__ partials) {
  __shared__ double sh[32];
  const int x = blockIdx.x * BX + threadIdx.x, y = blockIdx.y * BY + threadIdx.y, z = blockIdx.z;
  T res = T(0);
  if (x < d.nx && y < d.ny) {
    const Nbhd nb(d, x, y, z);
    const FieldAt<T> U{u, &nb};
    const CoefAt Bc{cf, &nb};
    const long long i = nb(0, 0, 0);
    res = r[i] - op_h2<T>(U, Bc, form) * inv_h2 / T(cf.J[i]);
    out[i] = res;
  }
  if (partials) {
    double s;
    if constexpr (sizeof(T) == 8) s = block_sum((double)res * (double)res, sh);
    else s = block_sum_f(res * res, sh);
    if (is_thread0()) partials[block_linear_id()] = s;
  }
}

// Weighted Jacobi (Appendix B, Eq. jacobi): e' = e + omega (r - L e) / D_L, D_L = diag(M) / J,
// written as e + omega (J r - M e) / diag(M).
template <typename T>
__global__ void k_curv_jacobi(Dims d, CurvCoef cf, const T* __restrict__ r, const T* __restrict__ e_in,
                              T* __restrict__ e_out, int form, T omega) {
  const int x = blockIdx.x * BX + threadIdx.x, y = blockIdx.y * BY + threadIdx.y, z = blockIdx.z;
  if (x >= d.nx || y >= d.ny) return;
  const Nbhd nb(d, x, y, z);
  const FieldAt<T> U{e_in, &nb};
  const CoefAt Bc{cf, &nb};
  const long long i = nb(0, 0, 0);
  const T Mh2 = op_h2<T>(U, Bc, form);
  const T Dh2 = diag_form_h2<T>(Bc, form);
  // (J r - M e) / diag(M) with h^2 scalings cancelling: (J r h^2 - M e h^2) / (diag h^2)
  e_out[i] = e_in[i] + omega * ((T(cf.J[i]) * r[i] * cf.h2 - Mh2) / Dh2);
}

// The first weighted-Jacobi sweep of a smoothing pass that starts from e = 0: op(0) = 0,
// so the sweep is pointwise, e' = omega (J r h^2 - 0) / diag h^2, and reads only r, J and
// the coefficients of the diagonal.  Written with the sweep's own expression, an explicit
// zero iterate and operator value, so that it rounds exactly like k_curv_tiled<CM_JACOBI>
// on a zero input (whose operator sum is +0).
template <int FORM>
__global__ void k_curv_jacobi_zero(Dims d, CurvCoef cf, const float* __restrict__ r, float* __restrict__ e_out,
                                   float omega) {
  const int x = blockIdx.x * BX + threadIdx.x, y = blockIdx.y * BY + threadIdx.y, z = blockIdx.z;
  if (x >= d.nx || y >= d.ny) return;
  const Nbhd nb(d, x, y, z);
  const CoefAt Bc{cf, &nb};
  const long long i = nb(0, 0, 0);
  const float Dh2 = FORM == 2 ? diag_S_h2<float>(Bc) : diag_M_h2<float>(Bc);
  const float Jc = cf.J[i], rc = r[i];
  const float u0 = 0.f, Mh2 = 0.f;
  e_out[i] = u0 + omega * ((Jc * rc * cf.h2 - Mh2) / Dh2);
}

// Dense matrix of the level operator (row-major n x n, FP64): entry (i, j) = (op(e_j) / J)_i.
struct UnitAt {
  const Nbhd* nb;
  long long j;
  __device__ __forceinline__ double operator()(int dx, int dy, int dz) const { return (*nb)(dx, dy, dz) == j ? 1.0 : 0.0; }
};

__global__ void k_curv_dense(Dims d, CurvCoef cf, int form, double* __restrict__ out) {
  const long long n = ncell(d);
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= n * n) return;
  const long long i = idx / n, j = idx % n;
  const int x = (int)(i % d.nx), y = (int)((i / d.nx) % d.ny), z = (int)(i / ((long long)d.nx * d.ny));
  const Nbhd nb(d, x, y, z);
  const UnitAt U{&nb, j};
  const CoefAt Bc{cf, &nb};
  const double v = op_form_h2<double>(U, Bc, form);
  out[idx] = v / ((double)cf.h2 * (double)cf.J[i]);
}

// ---- double-float residual of the outer defect correction on the finest level ----

// DF difference a - b of two double-float values, as an unnormalised pair (s, e):
// s = RN(a.hi - b.hi) with its exact error, plus the low parts' difference in e.  Its
// only use is the product with an FP32 weight in df_acc_prod, where e enters one FP32
// multiply, so the pair is not renormalised.
__device__ __forceinline__ float2 df_sub(float2 a, float2 b) {
  float s, e;
  two_sum(a.x, -b.x, s, e);
  e += a.y - b.y;
  return make_float2(s, e);
}

// acc += w * v exactly up to the rounding of the small terms (w float, v double-float).
__device__ __forceinline__ void df_acc_prod(DfAcc& acc, float w, float2 v) {
  const float p = w * v.x;
  const float pe = __fmaf_rn(w, v.x, -p);
  acc.add(p);
  acc.c += pe + w * v.y;
}

// h * (flux F^a on the face between offset c and c + e_a) of a double-float u, as a
// compensated pair (s, c): the five products of face_flux, each difference in
// double-float, summed as in df_acc_prod.
template <typename UF, typename BF>
__device__ __forceinline__ float2 df_face_flux(const UF& u, const BF& Bc, int a, int cx, int cy, int cz) {
  int px = cx, py = cy, pz = cz;
  shift(a, 1, px, py, pz);
  const float wa = face_B<float>(Bc, a, a, cx, cy, cz);
  const float2 v = df_sub(u(px, py, pz), u(cx, cy, cz));
  DfAcc f;
  f.s = wa * v.x;
  f.c = __fmaf_rn(wa, v.x, -f.s) + wa * v.y;
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    if (b == a) continue;
    const float w = 0.25f * face_B<float>(Bc, a, b, cx, cy, cz);
    int c1x = cx, c1y = cy, c1z = cz, c2x = cx, c2y = cy, c2z = cz;
    shift(b, 1, c1x, c1y, c1z);
    shift(b, -1, c2x, c2y, c2z);
    int d1x = px, d1y = py, d1z = pz, d2x = px, d2y = py, d2z = pz;
    shift(b, 1, d1x, d1y, d1z);
    shift(b, -1, d2x, d2y, d2z);
    df_acc_prod(f, w, df_sub(u(c1x, c1y, c1z), u(c2x, c2y, c2z)));
    df_acc_prod(f, w, df_sub(u(d1x, d1y, d1z), u(d2x, d2y, d2z)));
  }
  return make_float2(f.s, f.c);
}

// acc += sign * (s + c) of a face flux pair (sign +-1: exact).
__device__ __forceinline__ void df_acc_face(DfAcc& acc, float2 f, float sign) {
  acc.add(sign * f.x);
  acc.c += sign * f.y;
}

// acc += sign * h^2 (M^T y) with y double-float.
template <typename UF, typename BF>
__device__ __forceinline__ void df_apply_MT(DfAcc& acc, const UF& y, const BF& Bc, float sign) {
  auto q = [&](float w, int a, int b, int cx, int cy, int cz) {
    int px = cx, py = cy, pz = cz;
    shift(a, 1, px, py, pz);
    df_acc_prod(acc, w * face_B<float>(Bc, a, b, cx, cy, cz), df_sub(y(cx, cy, cz), y(px, py, pz)));
  };
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    int ax = 0, ay = 0, az = 0;
    shift(a, -1, ax, ay, az);
    q(sign, a, a, ax, ay, az);
    q(-sign, a, a, 0, 0, 0);
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      if (b == a) continue;
      int m1x = 0, m1y = 0, m1z = 0, p1x = 0, p1y = 0, p1z = 0;
      shift(b, -1, m1x, m1y, m1z);
      shift(b, 1, p1x, p1y, p1z);
      int m2x = ax, m2y = ay, m2z = az, p2x = ax, p2y = ay, p2z = az;
      shift(b, -1, m2x, m2y, m2z);
      shift(b, 1, p2x, p2y, p2z);
      const float w = 0.25f * sign;
      q(w, a, b, m1x, m1y, m1z);
      q(-w, a, b, p1x, p1y, p1z);
      q(w, a, b, m2x, m2y, m2z);
      q(-w, a, b, p2x, p2y, p2z);
    }
  }
}

// acc += sign * h^2 (S u) (symmetric variant) with u double-float, every difference in double-float.
template <typename UF, typename BF>
__device__ __forceinline__ void df_apply_S(DfAcc& acc, const UF& u, const BF& Bc, float sign) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    int px = 0, py = 0, pz = 0, mx = 0, my = 0, mz = 0;
    shift(a, 1, px, py, pz);
    shift(a, -1, mx, my, mz);
    df_acc_prod(acc, sign * face_B<float>(Bc, a, a, 0, 0, 0), df_sub(u(px, py, pz), u(0, 0, 0)));
    df_acc_prod(acc, -sign * face_B<float>(Bc, a, a, mx, my, mz), df_sub(u(0, 0, 0), u(mx, my, mz)));
  }
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = a + 1; b < 3; ++b)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        int ex, ey, ez, nx, ny, nz;
        edge_k(a, b, k, ex, ey, ez, nx, ny, nz);
        const float w = ((k == 1 || k == 2) ? -0.5f : 0.5f) * sign * edge_B<float>(Bc, a, b, ex, ey, ez);
        df_acc_prod(acc, w, df_sub(u(nx, ny, nz), u(0, 0, 0)));
      }
}

// partial sums of x * J and of J (volume-weighted mean, Eq. solvability)
__global__ void k_wsum(long long n, const double* __restrict__ x, const float* __restrict__ J,
                       double* __restrict__ pxj, double* __restrict__ pj) {
  __shared__ double sh[32];
  DfAcc s{0.f, 0.f}, w{0.f, 0.f};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float2 v = f64_to_df(x[i]);
    const float j = J[i];
    const float p = v.x * j;
    s.add(p);
    s.c += __fmaf_rn(v.x, j, -p) + v.y * j;
    w.add(j);
  }
  const double bs = block_sum_acc(s, sh);
  const double bw = block_sum_acc(w, sh);
  if (threadIdx.x == 0) {
    pxj[blockIdx.x] = bs;
    pj[blockIdx.x] = bw;
  }
}

__global__ void k_ratio(const double* a, const double* b, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) out[0] = b[0] != 0.0 ? a[0] / b[0] : 0.0;
}


// psi_bar = sum_a D_aa(S_aa) + sum_{a<b} D_ab(S_ab): the transpose of psi -> Hess psi,
// each second-difference stencil being self-adjoint on the periodic mesh.  S holds
// double-float pairs (exact sums of FP32 values); the 21 weighted terms are accumulated
// in a compensated pair (the weights 1/h^2, 1/(4h^2) are powers of two) and the sum is
// written in FP64.
__global__ void k_psibar_H(Dims d, const float2* __restrict__ S, float ih2, double* __restrict__ out) {
  const int x = blockIdx.x * BX + threadIdx.x, y = blockIdx.y * BY + threadIdx.y, z = blockIdx.z;
  if (x >= d.nx || y >= d.ny) return;
  const long long n = ncell(d);
  const Nbhd nb(d, x, y, z);
  auto C = [&](int k, int dx, int dy, int dz) { return S[k * n + nb(dx, dy, dz)]; };
  const float iq = 0.25f * ih2;
  DfAcc acc{0.f, 0.f};
  auto add = [&](float2 v, float w) {
    acc.add(w * v.x);
    acc.c += w * v.y;
  };
  add(C(0, 1, 0, 0), ih2);
  add(C(0, 0, 0, 0), -2.f * ih2);
  add(C(0, -1, 0, 0), ih2);
  add(C(1, 0, 1, 0), ih2);
  add(C(1, 0, 0, 0), -2.f * ih2);
  add(C(1, 0, -1, 0), ih2);
  add(C(2, 0, 0, 1), ih2);
  add(C(2, 0, 0, 0), -2.f * ih2);
  add(C(2, 0, 0, -1), ih2);
  add(C(3, 1, 1, 0), iq);
  add(C(3, 1, -1, 0), -iq);
  add(C(3, -1, 1, 0), -iq);
  add(C(3, -1, -1, 0), iq);
  add(C(4, 1, 0, 1), iq);
  add(C(4, 1, 0, -1), -iq);
  add(C(4, -1, 0, 1), -iq);
  add(C(4, -1, 0, -1), iq);
  add(C(5, 0, 1, 1), iq);
  add(C(5, 0, 1, -1), -iq);
  add(C(5, 0, -1, 1), -iq);
  add(C(5, 0, -1, -1), iq);
  out[nb(0, 0, 0)] = (double)acc.s + (double)acc.c;
}

// out = J (lam - s) in FP64 from a double-float lam (delta_bar of the curvilinear adjoint).
__global__ void k_jscale(long long n, const float2* __restrict__ lam, const float* __restrict__ J,
                         const double* __restrict__ s_dev, double* __restrict__ out, double* __restrict__ lam64) {
  const double s = s_dev ? s_dev[0] : 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double l = df_to_f64(lam[i]);
    if (lam64) lam64[i] = l;
    if (out) out[i] = (double)J[i] * (l - s);
  }
}

// ------------------------------------------------------------------ tiled, z-streaming forms
//
// The FP32 sweep and residual and the double-float residual of the finest level run
// as z-streaming tile kernels: a CTA owns a CTX x CTY tile of cells (one per thread)
// and a chunk of z planes; the haloed planes (one cell of halo) of u and of the six
// B components pass through a four-slot shared-memory ring, so every neighbour read
// of the 19-point operator is a shared-memory load at a constant offset.  The
// operator is the same template (face_flux / apply_MT_h2 / apply_S_h2 / diag_M_h2)
// read through shared-memory accessors.  For M (form 0) each face flux is formed once
// per plane and shared through shared memory (x and y faces) or carried in a register
// (z faces), instead of once by each of the face's two cells.  Loads of the plane two
// ahead (and of the cell's own J and right-hand side one plane ahead) are issued
// before the current plane is computed; one barrier per plane, two for form 0.
constexpr int CTX = 32, CTY = 8, CNT = CTX * CTY;
constexpr int CSW = CTX + 2, CSH = CTY + 2, CSN = CSW * CSH;  // haloed plane
constexpr int CQ = (CSN + CNT - 1) / CNT;                      // haloed cells per thread

template <typename V>
struct RingU {
  const V* pl[3];  // planes t - 1, t, t + 1
  int c;           // haloed index of the thread's cell
  __device__ __forceinline__ V operator()(int dx, int dy, int dz) const { return pl[dz + 1][c + dy * CSW + dx]; }
};
struct RingB {
  const float* pl[3];
  int c;
  __device__ __forceinline__ float operator()(int comp, int dx, int dy, int dz) const {
    return pl[dz + 1][comp * CSN + c + dy * CSW + dx];
  }
};

// One ring slot: the haloed plane of u (V = float or float2) followed by B (6 x CSN floats).
template <typename V>
constexpr size_t ring_slot_bytes() {
  return ((CSN * sizeof(V) + 15) / 16 * 16) + 6 * CSN * sizeof(float);
}

template <typename V>
struct Ring {
  char* base;
  __device__ __forceinline__ V* u(int slot) const { return reinterpret_cast<V*>(base + slot * ring_slot_bytes<V>()); }
  __device__ __forceinline__ float* b(int slot) const {
    return reinterpret_cast<float*>(base + slot * ring_slot_bytes<V>() + (CSN * sizeof(V) + 15) / 16 * 16);
  }
};

// Prefetch registers of one haloed plane: each thread loads CQ haloed cells.
template <typename V>
struct PlaneRegs {
  V u[CQ];
  float b[CQ][6];
};

// In-plane offsets of the thread's CQ haloed cells (periodic wrap in x and y), the same
// for every plane of the chunk: computed once per CTA, before the z loop.
struct PlaneIdx {
  int off[CQ];
};
__device__ __forceinline__ PlaneIdx plane_idx(Dims d, int x0, int y0) {
  PlaneIdx P;
#pragma unroll
  for (int k = 0; k < CQ; ++k) {
    const int q = min((int)threadIdx.x + k * CNT, CSN - 1);
    // full modulo: a tile may be wider than a coarse level
    const int gx = ((x0 - 1 + q % CSW) % d.nx + d.nx) % d.nx, gy = ((y0 - 1 + q / CSW) % d.ny + d.ny) % d.ny;
    P.off[k] = gy * d.nx + gx;
  }
  return P;
}

// Plane z in [-1, nz] (the chunk's planes and one on each side) wrapped onto the mesh.
template <typename V>
__device__ __forceinline__ void load_plane(Dims d, const V* __restrict__ u, const CurvCoef& cf, const PlaneIdx& P,
                                           int z, PlaneRegs<V>& R) {
  const int zw = z < 0 ? z + d.nz : (z >= d.nz ? z - d.nz : z);
  const long long zo = (long long)zw * d.nx * d.ny;
#pragma unroll
  for (int k = 0; k < CQ; ++k) {
    const int q = threadIdx.x + k * CNT;
    if (q < CSN) {
      const long long gi = zo + P.off[k];
      R.u[k] = u[gi];
#pragma unroll
      for (int m = 0; m < 6; ++m) R.b[k][m] = __ldg(cf.B[m] + gi);
    }
  }
}

template <typename V>
__device__ __forceinline__ void store_plane(const Ring<V>& ring, int slot, const PlaneRegs<V>& R) {
  V* su = ring.u(slot);
  float* sb = ring.b(slot);
#pragma unroll
  for (int k = 0; k < CQ; ++k) {
    const int q = threadIdx.x + k * CNT;
    if (q < CSN) {
      su[q] = R.u[k];
#pragma unroll
      for (int m = 0; m < 6; ++m) sb[m * CSN + q] = R.b[k][m];
    }
  }
}

// ---- geometry of a level in double-float arithmetic ----

// (hi, lo) products and the reciprocal: Dekker's product with the error of a.hi b.hi
// from one FMA, the cross terms added to it, renormalised.
__device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
  const float p = a.x * b.x;
  float e = __fmaf_rn(a.x, b.x, -p);
  e = __fmaf_rn(a.x, b.y, e);
  e = __fmaf_rn(a.y, b.x, e);
  float h, l;
  quick_two_sum(p, e, h, l);
  return make_float2(h, l);
}
__device__ __forceinline__ float2 df_scale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// 1 / a: q0 = RN(1 / a.hi), one Newton correction q0 (1 - a q0) with the residual in
// double-float (1 - a.hi q0 is exact by Sterbenz's lemma once its rounding error is split off).
__device__ __forceinline__ float2 df_recip(float2 a) {
  const float q0 = 1.0f / a.x;
  const float p = a.x * q0;
  const float pe = __fmaf_rn(a.x, q0, -p);
  const float r = ((1.0f - p) - pe) - a.y * q0;
  float h, l;
  quick_two_sum(q0, q0 * r, h, l);
  return make_float2(h, l);
}
// a b + c d + e f
__device__ __forceinline__ float2 df_dot3(float2 a, float2 b, float2 c, float2 d, float2 e, float2 f) {
  return df_add(df_add(df_mul(a, b), df_mul(c, d)), df_mul(e, f));
}

// Geometry of one level (Sec. 4.2, Eq. triad and Eq. metric): A = I + Hess psi with the
// central second differences, J = det A = a . adj(A) row 0, B = adj(A)^2 / J, every
// step in double-float from the FP64 psi (each value converted once, in a z-streaming
// tile with a three-plane ring) and rounded to FP32 at the end.  ih2 = 1 / h^2 and
// iq = 1 / (4 h^2) are powers of two (h = 2^l), so the scalings are exact.
__global__ void __launch_bounds__(CNT) k_geom_tiled(Dims d, const double* __restrict__ psi, float ih2,
                                                    CurvCoefOut out, int zc) {
  __shared__ float2 ring[4][CSN];
  const int tx = threadIdx.x % CTX, ty = threadIdx.x / CTX;
  const int x0 = blockIdx.x * CTX, y0 = blockIdx.y * CTY, z0 = blockIdx.z * zc;
  const int zend = min(z0 + zc, d.nz);
  const int x = x0 + tx, y = y0 + ty;
  const bool own = x < d.nx && y < d.ny;
  const long long pst = (long long)d.nx * d.ny;
  const int c = (ty + 1) * CSW + tx + 1;
  const PlaneIdx PI = plane_idx(d, x0, y0);
  double pre[CQ];
  auto load = [&](int z) {
    const int zw = z < 0 ? z + d.nz : (z >= d.nz ? z - d.nz : z);
#pragma unroll
    for (int k = 0; k < CQ; ++k)
      if (threadIdx.x + k * CNT < CSN) pre[k] = psi[(long long)zw * pst + PI.off[k]];
  };
  auto store = [&](int slot) {
#pragma unroll
    for (int k = 0; k < CQ; ++k) {
      const int q = threadIdx.x + k * CNT;
      if (q < CSN) ring[slot][q] = f64_to_df(pre[k]);
    }
  };
  auto slot = [&](int p) { return (p - (z0 - 1)) & 3; };
  load(z0 - 1);
  store(slot(z0 - 1));
  load(z0);
  store(slot(z0));
  load(z0 + 1);
  const float iq = 0.25f * ih2;
  for (int t = z0; t < zend; ++t) {
    store(slot(t + 1));
    __syncthreads();
    if (t + 1 < zend) load(t + 2);
    if (own) {
      const float2* pl[3] = {ring[slot(t - 1)], ring[slot(t)], ring[slot(t + 1)]};
      auto P = [&](int dx, int dy, int dz) { return pl[dz + 1][c + dy * CSW + dx]; };
      const float2 c2 = df_scale(P(0, 0, 0), -2.0f);
      auto second = [&](float2 p, float2 m) { return df_add_f(df_scale(df_add(df_add(p, m), c2), ih2), 1.0f); };
      auto mixed = [&](float2 pp, float2 pm, float2 mp, float2 mm) {
        return df_scale(df_add(df_add(pp, make_float2(-pm.x, -pm.y)), df_add(mm, make_float2(-mp.x, -mp.y))), iq);
      };
      const float2 a = second(P(1, 0, 0), P(-1, 0, 0));
      const float2 b = second(P(0, 1, 0), P(0, -1, 0));
      const float2 cc = second(P(0, 0, 1), P(0, 0, -1));
      const float2 dxy = mixed(P(1, 1, 0), P(1, -1, 0), P(-1, 1, 0), P(-1, -1, 0));
      const float2 dxz = mixed(P(1, 0, 1), P(1, 0, -1), P(-1, 0, 1), P(-1, 0, -1));
      const float2 dyz = mixed(P(0, 1, 1), P(0, 1, -1), P(0, -1, 1), P(0, -1, -1));
      auto neg = [](float2 v) { return make_float2(-v.x, -v.y); };
      // adjugate of the symmetric triad [[a, dxy, dxz], [dxy, b, dyz], [dxz, dyz, c]]
      const float2 j00 = df_add(df_mul(b, cc), neg(df_mul(dyz, dyz)));
      const float2 j11 = df_add(df_mul(a, cc), neg(df_mul(dxz, dxz)));
      const float2 j22 = df_add(df_mul(a, b), neg(df_mul(dxy, dxy)));
      const float2 j01 = df_add(df_mul(dxz, dyz), neg(df_mul(dxy, cc)));
      const float2 j02 = df_add(df_mul(dxy, dyz), neg(df_mul(b, dxz)));
      const float2 j12 = df_add(df_mul(dxy, dxz), neg(df_mul(a, dyz)));
      const float2 J = df_dot3(a, j00, dxy, j01, dxz, j02);
      const float2 iJ = df_recip(J);
      const long long i = (long long)t * pst + (long long)y * d.nx + x;
      out.J[i] = J.x;
      out.B[0][i] = df_mul(df_dot3(j00, j00, j01, j01, j02, j02), iJ).x;
      out.B[1][i] = df_mul(df_dot3(j01, j01, j11, j11, j12, j12), iJ).x;
      out.B[2][i] = df_mul(df_dot3(j02, j02, j12, j12, j22, j22), iJ).x;
      out.B[3][i] = df_mul(df_dot3(j00, j01, j01, j11, j02, j12), iJ).x;
      out.B[4][i] = df_mul(df_dot3(j00, j02, j01, j12, j02, j22), iJ).x;
      out.B[5][i] = df_mul(df_dot3(j01, j02, j11, j12, j12, j22), iJ).x;
    }
  }
}

// ---- adjoint of the geometry (Sec. 4.8, Eq. adj_op) ----

// Per cell of the finest level: the cotangent of the triad A for the scalar
//   <lam, b(J)> - <lam, M(B) phi>,  b = J (delta - m_w),
// where Jbar = (delta - m_w)(lam - s_lam), s_lam = sum(J lam)/sum(J), and Bbar
// comes from <lam, M phi> = sum_a sum_i sum_b B^{ab}_face(i) G^a_b[phi](i) (lam_i - lam_{i+a})/h,
// B^{ab}_face(i) = (B^{ab}_i + B^{ab}_{i+a})/2.  With B = J A^-2 and J = det A:
//   Abar_J = Jbar J A^-1,  Abar_B = J <Bbar, A^-2> A^-1 - J (A^-1 Bbar A^-2 + A^-2 Bbar A^-1).
// Writes S = Abar_J - Abar_B symmetrised for the Hessian stencils:
// S_aa = Abar_aa, S_ab = Abar_ab + Abar_ba (a < b), packed xx, yy, zz, xy, xz, yz.
// Precision: the differences that cancel (second differences of psi, differences of phi
// and lam across faces and edges) are formed in double-float from psi, phi (FP64,
// converted once per cell in a z-streaming three-plane ring) and lam (double-float) and
// rounded to FP32; the pointwise algebra of the 3 x 3 triad (adjugate, J, A^-1, A^-2 and
// the cotangent products) runs in FP32, A having its eigenvalues in [1/2, 3/2] (FP64
// arithmetic runs at a small fraction of the FP32 rate).  S is written as double-float
// pairs: the diagonal entries exactly, the off-diagonal sums by an error-free addition.
__global__ void __launch_bounds__(CNT) k_psibar_tiled(Dims d, const double* __restrict__ psi,
                                                      const double* __restrict__ phi, const float2* __restrict__ lam,
                                                      const double* __restrict__ delta,
                                                      const double* __restrict__ mw_dev,
                                                      const double* __restrict__ slam_dev, float ih, int sym,
                                                      float2* __restrict__ S, int zc) {
  __shared__ float2 rps[4][CSN], rph[4][CSN], rla[4][CSN];  // psi, phi, lam rings
  const int tx = threadIdx.x % CTX, ty = threadIdx.x / CTX;
  const int x0 = blockIdx.x * CTX, y0 = blockIdx.y * CTY, z0 = blockIdx.z * zc;
  const int zend = min(z0 + zc, d.nz);
  const int x = x0 + tx, y = y0 + ty;
  const bool own = x < d.nx && y < d.ny;
  const long long n = ncell(d);
  const long long pst = (long long)d.nx * d.ny;
  const int c = (ty + 1) * CSW + tx + 1;
  const PlaneIdx PI = plane_idx(d, x0, y0);
  double qps[CQ], qph[CQ];
  float2 qla[CQ];
  auto load = [&](int z) {
    const int zw = z < 0 ? z + d.nz : (z >= d.nz ? z - d.nz : z);
#pragma unroll
    for (int k = 0; k < CQ; ++k)
      if (threadIdx.x + k * CNT < CSN) {
        const long long gi = (long long)zw * pst + PI.off[k];
        qps[k] = psi[gi];
        qph[k] = phi[gi];
        qla[k] = lam[gi];
      }
  };
  auto store = [&](int slot) {
#pragma unroll
    for (int k = 0; k < CQ; ++k) {
      const int q = threadIdx.x + k * CNT;
      if (q < CSN) {
        rps[slot][q] = f64_to_df(qps[k]);
        rph[slot][q] = f64_to_df(qph[k]);
        rla[slot][q] = qla[k];
      }
    }
  };
  auto slot = [&](int p) { return (p - (z0 - 1)) & 3; };
  load(z0 - 1);
  store(slot(z0 - 1));
  load(z0);
  store(slot(z0));
  load(z0 + 1);
  const float ih2 = ih * ih, iq = 0.25f * ih2;  // powers of two
  const double mw = mw_dev[0], sl = slam_dev[0];
  for (int t = z0; t < zend; ++t) {
    store(slot(t + 1));
    __syncthreads();
    if (t + 1 < zend) load(t + 2);
    if (!own) continue;
    const int s0 = slot(t - 1), s1 = slot(t), s2 = slot(t + 1);
    auto at = [&](const float2 (*r)[CSN], int dx, int dy, int dz) {
      return r[dz < 0 ? s0 : (dz > 0 ? s2 : s1)][c + dy * CSW + dx];
    };
    auto PS = [&](int dx, int dy, int dz) { return at(rps, dx, dy, dz); };
    auto PH = [&](int dx, int dy, int dz) { return at(rph, dx, dy, dz); };
    auto LA = [&](int dx, int dy, int dz) { return at(rla, dx, dy, dz); };
    auto neg = [](float2 v) { return make_float2(-v.x, -v.y); };
    // a - b of two double-float values, rounded to FP32
    auto dd = [](float2 a, float2 b) {
      float s, e;
      two_sum(a.x, -b.x, s, e);
      return s + (e + (a.y - b.y));
    };
    // triad at this cell: double-float second differences, then FP32
    const float2 c2 = df_scale(PS(0, 0, 0), -2.0f);
    auto second = [&](float2 p, float2 m) { return 1.0f + df_add(df_add(p, m), c2).x * ih2; };
    auto mixed = [&](float2 pp, float2 pm, float2 mp, float2 mm) {
      return df_add(df_add(pp, neg(pm)), df_add(mm, neg(mp))).x * iq;
    };
    float A[3][3];
    A[0][0] = second(PS(1, 0, 0), PS(-1, 0, 0));
    A[1][1] = second(PS(0, 1, 0), PS(0, -1, 0));
    A[2][2] = second(PS(0, 0, 1), PS(0, 0, -1));
    A[0][1] = A[1][0] = mixed(PS(1, 1, 0), PS(1, -1, 0), PS(-1, 1, 0), PS(-1, -1, 0));
    A[0][2] = A[2][0] = mixed(PS(1, 0, 1), PS(1, 0, -1), PS(-1, 0, 1), PS(-1, 0, -1));
    A[1][2] = A[2][1] = mixed(PS(0, 1, 1), PS(0, 1, -1), PS(0, -1, 1), PS(0, -1, -1));
    float adj[3][3];
    adj[0][0] = A[1][1] * A[2][2] - A[1][2] * A[1][2];
    adj[1][1] = A[0][0] * A[2][2] - A[0][2] * A[0][2];
    adj[2][2] = A[0][0] * A[1][1] - A[0][1] * A[0][1];
    adj[0][1] = adj[1][0] = A[0][2] * A[1][2] - A[0][1] * A[2][2];
    adj[0][2] = adj[2][0] = A[0][1] * A[1][2] - A[1][1] * A[0][2];
    adj[1][2] = adj[2][1] = A[0][1] * A[0][2] - A[0][0] * A[1][2];
    const float J = A[0][0] * adj[0][0] + A[0][1] * adj[0][1] + A[0][2] * adj[0][2];
    const float iJ = 1.0f / J;
    float Ai[3][3], Ai2[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) Ai[a][b] = adj[a][b] * iJ;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) Ai2[a][b] = Ai[a][0] * Ai[0][b] + Ai[a][1] * Ai[1][b] + Ai[a][2] * Ai[2][b];
    // Bbar at this cell: faces a at i (own) and i - a (left neighbour's face); each face
    // value G^a_b[phi] (lam_c - lam_{c+a}) / h from differences rounded to FP32 (ih = 1/h)
    auto fbar = [&](int a, int b, int cx, int cy, int cz) -> float {
      int px = cx, py = cy, pz = cz;
      shift(a, 1, px, py, pz);
      const float Lam = dd(LA(cx, cy, cz), LA(px, py, pz)) * ih;
      float G;
      if (a == b) {
        G = dd(PH(px, py, pz), PH(cx, cy, cz)) * ih;
      } else {
        int c1x = cx, c1y = cy, c1z = cz, c2x = cx, c2y = cy, c2z = cz;
        shift(b, 1, c1x, c1y, c1z);
        shift(b, -1, c2x, c2y, c2z);
        int d1x = px, d1y = py, d1z = pz, d2x = px, d2y = py, d2z = pz;
        shift(b, 1, d1x, d1y, d1z);
        shift(b, -1, d2x, d2y, d2z);
        G = 0.25f * (dd(PH(c1x, c1y, c1z), PH(c2x, c2y, c2z)) + dd(PH(d1x, d1y, d1z), PH(d2x, d2y, d2z))) * ih;
      }
      return G * Lam;
    };
    float Bb[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      int mx = 0, my = 0, mz = 0;
      shift(a, -1, mx, my, mz);
#pragma unroll
      for (int b = 0; b < 3; ++b)
        Bb[a][b] = (sym && b != a) ? 0.f : 0.5f * (fbar(a, b, 0, 0, 0) + fbar(a, b, mx, my, mz));
    }
    if (sym) {
      // symmetric variant: d<lam, S phi>/dC on the ab-edge at base e is
      //   (1/2h^2) [(lam_e - lam_{e+a+b}) (phi_{e+a+b} - phi_e) + (lam_{e+a} - lam_{e+b}) (phi_{e+a} - phi_{e+b})],
      // and each of the four edges around this cell takes a quarter of its B^{ab} (a < b).
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = a + 1; b < 3; ++b) {
          float acc = 0.f;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            int ex = 0, ey = 0, ez = 0;
            if (k & 1) shift(a, -1, ex, ey, ez);
            if (k & 2) shift(b, -1, ex, ey, ez);
            int ax = ex, ay = ey, az = ez, bx = ex, by = ey, bz = ez;
            shift(a, 1, ax, ay, az);
            shift(b, 1, bx, by, bz);
            int px = ax, py = ay, pz = az;
            shift(b, 1, px, py, pz);
            acc += dd(LA(ex, ey, ez), LA(px, py, pz)) * dd(PH(px, py, pz), PH(ex, ey, ez)) +
                   dd(LA(ax, ay, az), LA(bx, by, bz)) * dd(PH(ax, ay, az), PH(bx, by, bz));
          }
          Bb[a][b] = 0.125f * acc * ih2;
        }
    }
    // Abar_B = J <Bbar, A^-2> A^-1 - J (A^-1 Bbar A^-2 + A^-2 Bbar A^-1)   (A symmetric)
    float inner = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) inner += Bb[a][b] * Ai2[a][b];
    float T1[3][3], T2[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        T1[a][b] = Bb[a][0] * Ai2[0][b] + Bb[a][1] * Ai2[1][b] + Bb[a][2] * Ai2[2][b];  // Bbar A^-2
        T2[a][b] = Bb[a][0] * Ai[0][b] + Bb[a][1] * Ai[1][b] + Bb[a][2] * Ai[2][b];     // Bbar A^-1
      }
    const long long i = (long long)t * pst + (long long)y * d.nx + x;
    const float Jbar = (float)((delta[i] - mw) * (df_to_f64(LA(0, 0, 0)) - sl));
    float Ab[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const float t = Ai[a][0] * T1[0][b] + Ai[a][1] * T1[1][b] + Ai[a][2] * T1[2][b] +
                        Ai2[a][0] * T2[0][b] + Ai2[a][1] * T2[1][b] + Ai2[a][2] * T2[2][b];
        const float AbB = J * inner * Ai[a][b] - J * t;
        Ab[a][b] = Jbar * J * Ai[a][b] - AbB;
      }
    S[i] = make_float2(Ab[0][0], 0.f);
    S[n + i] = make_float2(Ab[1][1], 0.f);
    S[2 * n + i] = make_float2(Ab[2][2], 0.f);
    auto pair = [](float u, float v) {
      float s, e;
      two_sum(u, v, s, e);
      return make_float2(s, e);
    };
    S[3 * n + i] = pair(Ab[0][1], Ab[1][0]);
    S[4 * n + i] = pair(Ab[0][2], Ab[2][0]);
    S[5 * n + i] = pair(Ab[1][2], Ab[2][1]);
  }
}

// z chunk: halved until there are four waves of four CTAs per SM, down to 4 planes (on
// small levels a CTA's planes are a chain of dependent load rounds: 8-plane chunks made
// the 256^3 moving-mesh solve 2% slower); the outputs do not depend on it.
int curv_zchunk(Dims d) {
  const long long tiles = (long long)((d.nx + CTX - 1) / CTX) * ((d.ny + CTY - 1) / CTY);
  int zc = d.nz;
  while (zc > 4 && tiles * ((d.nz + zc - 1) / zc) < 4 * 4 * 152) zc = (zc + 1) / 2;
  return zc;
}
dim3 curv_tiled_grid(Dims d) {
  const int zc = curv_zchunk(d);
  return dim3((d.nx + CTX - 1) / CTX, (d.ny + CTY - 1) / CTY, (d.nz + zc - 1) / zc);
}

enum CurvMode { CM_JACOBI = 0, CM_RESID = 1 };

// FP32 forms.  CM_JACOBI: out = e + omega (J r h^2 - op(e) h^2) / diag h^2 (Appendix B);
// CM_RESID: out = r - op(u) / (h^2 J) with block partial sums of out^2 (partials nullable).
template <int MODE, int TR>
__global__ void __launch_bounds__(CNT) k_curv_tiled(Dims d, CurvCoef cf, const float* __restrict__ r,
                                                      const float* __restrict__ u, float* __restrict__ out,
                                                      float omega, float inv_h2, double* __restrict__ partials, int zc) {
  extern __shared__ __align__(16) char smc[];
  __shared__ double shr[32];
  const Ring<float> ring{smc};
  const int tx = threadIdx.x % CTX, ty = threadIdx.x / CTX;
  const int x0 = blockIdx.x * CTX, y0 = blockIdx.y * CTY, z0 = blockIdx.z * zc;
  const int zend = min(z0 + zc, d.nz);
  const int x = x0 + tx, y = y0 + ty;
  const bool own = x < d.nx && y < d.ny;
  const long long pst = (long long)d.nx * d.ny;
  const int c = (ty + 1) * CSW + tx + 1;
  float rr = 0.f;
  __shared__ float sfx[CTY][CTX + 1], sfy[CTY + 1][CTX];  // x- and y-face fluxes of M (form 0)
  float fzm = 0.f;                                         // -z face flux of M (form 0)
  PlaneRegs<float> R;
  const PlaneIdx PI = plane_idx(d, x0, y0);
  auto slot = [&](int p) { return (p - (z0 - 1)) & 3; };
  load_plane(d, u, cf, PI, z0 - 1, R);
  store_plane(ring, slot(z0 - 1), R);
  load_plane(d, u, cf, PI, z0, R);
  store_plane(ring, slot(z0), R);
  load_plane(d, u, cf, PI, z0 + 1, R);
  // J and r of the thread's cell, one plane ahead
  const long long i0 = (long long)y * d.nx + x;
  float Jn = 0.f, rn = 0.f;
  if (own) {
    Jn = cf.J[(long long)z0 * pst + i0];
    rn = r[(long long)z0 * pst + i0];
  }
  for (int t = z0; t < zend; ++t) {
    store_plane(ring, slot(t + 1), R);
    __syncthreads();
    if (t + 1 < zend) load_plane(d, u, cf, PI, t + 2, R);
    const float Jc = Jn, rc = rn;
    if (own && t + 1 < zend) {
      Jn = cf.J[(long long)(t + 1) * pst + i0];
      rn = r[(long long)(t + 1) * pst + i0];
    }
    const RingU<float> U{{ring.u(slot(t - 1)), ring.u(slot(t)), ring.u(slot(t + 1))}, c};
    const RingB Bc{{ring.b(slot(t - 1)), ring.b(slot(t)), ring.b(slot(t + 1))}, c};
    float Mh2 = 0.f;
    if constexpr (TR == 0) {
      // Each face flux of M once: the thread's -x, -y and +z faces, the tile's last
      // column and row of +x / +y faces by warp 0 (8 lanes) and warp CTY - 1, the -z
      // face carried from the plane below.  Threads outside the mesh hold periodic
      // images of its cells, so their fluxes are the wrapped ones.
      if (t == z0) fzm = face_flux<float>(U, Bc, 2, 0, 0, -1);
      sfx[ty][tx] = face_flux<float>(U, Bc, 0, -1, 0, 0);
      sfy[ty][tx] = face_flux<float>(U, Bc, 1, 0, -1, 0);
      const float fzp = face_flux<float>(U, Bc, 2, 0, 0, 0);
      if (ty == CTY - 1) sfy[CTY][tx] = face_flux<float>(U, Bc, 1, 0, 0, 0);
      if (ty == 0 && tx < CTY) {
        const int ce = (tx + 1) * CSW + CTX;  // haloed index of the cell (CTX - 1, tx)
        const RingU<float> Ue{{U.pl[0], U.pl[1], U.pl[2]}, ce};
        const RingB Be{{Bc.pl[0], Bc.pl[1], Bc.pl[2]}, ce};
        sfx[tx][CTX] = face_flux<float>(Ue, Be, 0, 0, 0, 0);
      }
      __syncthreads();
      // same association as apply_M_h2: ((0 + x) + y) + z
      Mh2 = ((0.f + (sfx[ty][tx + 1] - sfx[ty][tx])) + (sfy[ty + 1][tx] - sfy[ty][tx])) + (fzp - fzm);
      fzm = fzp;
    }
    if (own) {
      const long long i = (long long)t * pst + i0;
      if constexpr (TR != 0) Mh2 = TR == 2 ? apply_S_h2<float>(U, Bc) : apply_MT_h2<float>(U, Bc);
      if (MODE == CM_JACOBI) {
        const float Dh2 = TR == 2 ? diag_S_h2<float>(Bc) : diag_M_h2<float>(Bc);
        out[i] = U(0, 0, 0) + omega * ((Jc * rc * cf.h2 - Mh2) / Dh2);
      } else {
        const float res = rc - Mh2 * inv_h2 / Jc;
        out[i] = res;
        rr += res * res;
      }
    }
  }
  if (MODE == CM_RESID && partials) {
    const double s = block_sum_f(rr, shr);
    if (is_thread0()) partials[block_linear_id()] = s;
  }
}

struct DfRingAt {
  const float2* pl[3];
  int c;
  __device__ __forceinline__ float2 operator()(int dx, int dy, int dz) const { return pl[dz + 1][c + dy * CSW + dx]; }
};

// r = (b - op(u) / h^2) / J rounded to float, with b = J (src - m) when scale_J (forward
// source in L-form) or b = src (transposed solve, M-form right-hand side).  Partial sums
// of r^2 and of (b / J)^2.  Three CTAs per SM (80 registers, no spill): the kernel is
// bound by instruction issue, and 24 warps per SM run it 6% faster than 16.
__global__ void __launch_bounds__(CNT, 3) k_curv_df_residual_tiled(Dims d, CurvCoef cf, const float2* __restrict__ src,
                                                                 const double* __restrict__ m_dev, int scale_J,
                                                                 const float2* __restrict__ u, int form,
                                                                 float* __restrict__ r, double* __restrict__ pr2,
                                                                 double* __restrict__ pf2, int zc) {
  extern __shared__ __align__(16) char smc[];
  __shared__ double shr[32];
  const Ring<float2> ring{smc};
  const int tx = threadIdx.x % CTX, ty = threadIdx.x / CTX;
  const int x0 = blockIdx.x * CTX, y0 = blockIdx.y * CTY, z0 = blockIdx.z * zc;
  const int zend = min(z0 + zc, d.nz);
  const int x = x0 + tx, y = y0 + ty;
  const bool own = x < d.nx && y < d.ny;
  const long long pst = (long long)d.nx * d.ny;
  const int c = (ty + 1) * CSW + tx + 1;
  float2 m = make_float2(0.f, 0.f);
  if (m_dev) m = f64_to_df(m_dev[0]);
  float r2 = 0.f, f2 = 0.f;
  __shared__ float2 sfx[CTY][CTX + 1], sfy[CTY + 1][CTX];  // x- and y-face fluxes of M (form 0), (s, c)
  float2 fzm = make_float2(0.f, 0.f);                      // -z face flux of M (form 0)
  PlaneRegs<float2> R;
  const PlaneIdx PI = plane_idx(d, x0, y0);
  auto slot = [&](int p) { return (p - (z0 - 1)) & 3; };
  load_plane(d, u, cf, PI, z0 - 1, R);
  store_plane(ring, slot(z0 - 1), R);
  load_plane(d, u, cf, PI, z0, R);
  store_plane(ring, slot(z0), R);
  load_plane(d, u, cf, PI, z0 + 1, R);
  // J and the source of the thread's cell, one plane ahead
  const long long i0 = (long long)y * d.nx + x;
  float Jn = 0.f;
  float2 bn = make_float2(0.f, 0.f);
  if (own) {
    Jn = cf.J[(long long)z0 * pst + i0];
    bn = src[(long long)z0 * pst + i0];
  }
  for (int t = z0; t < zend; ++t) {
    store_plane(ring, slot(t + 1), R);
    __syncthreads();
    if (t + 1 < zend) load_plane(d, u, cf, PI, t + 2, R);
    const float J = Jn;
    float2 b = bn;
    if (own && t + 1 < zend) {
      Jn = cf.J[(long long)(t + 1) * pst + i0];
      bn = src[(long long)(t + 1) * pst + i0];
    }
    const DfRingAt U{{ring.u(slot(t - 1)), ring.u(slot(t)), ring.u(slot(t + 1))}, c};
    const RingB Bc{{ring.b(slot(t - 1)), ring.b(slot(t)), ring.b(slot(t + 1))}, c};
    float2 fzp = make_float2(0.f, 0.f);
    if (form == 0) {
      // each face flux of M once, as in the FP32 sweep (the -x, -y, +z faces of every
      // thread, the tile's last column / row of +x / +y faces, the -z face carried)
      if (t == z0) fzm = df_face_flux(U, Bc, 2, 0, 0, -1);
      sfx[ty][tx] = df_face_flux(U, Bc, 0, -1, 0, 0);
      sfy[ty][tx] = df_face_flux(U, Bc, 1, 0, -1, 0);
      fzp = df_face_flux(U, Bc, 2, 0, 0, 0);
      if (ty == CTY - 1) sfy[CTY][tx] = df_face_flux(U, Bc, 1, 0, 0, 0);
      if (ty == 0 && tx < CTY) {
        const int ce = (tx + 1) * CSW + CTX;  // haloed index of the cell (CTX - 1, tx)
        const DfRingAt Ue{{U.pl[0], U.pl[1], U.pl[2]}, ce};
        const RingB Be{{Bc.pl[0], Bc.pl[1], Bc.pl[2]}, ce};
        sfx[tx][CTX] = df_face_flux(Ue, Be, 0, 0, 0, 0);
      }
      __syncthreads();
    }
    if (own) {
      const long long i = (long long)t * pst + i0;
      if (m_dev) b = df_add(b, make_float2(-m.x, -m.y));
      DfAcc acc{0.f, 0.f};
      const float wb = scale_J ? J * cf.h2 : cf.h2;
      df_acc_prod(acc, wb, b);
      if (form == 0) {
        // acc -= sum_a (F_a(+) - F_a(-)), every face flux a compensated pair
        df_acc_face(acc, sfx[ty][tx + 1], -1.f);
        df_acc_face(acc, sfx[ty][tx], 1.f);
        df_acc_face(acc, sfy[ty + 1][tx], -1.f);
        df_acc_face(acc, sfy[ty][tx], 1.f);
        df_acc_face(acc, fzp, -1.f);
        df_acc_face(acc, fzm, 1.f);
      } else if (form == 2) {
        df_apply_S(acc, U, Bc, -1.f);
      } else {
        df_apply_MT(acc, U, Bc, -1.f);
      }
      const float rv = (acc.s + acc.c) / (J * cf.h2);
      r[i] = rv;
      r2 += rv * rv;
      const float fv = scale_J ? (b.x + b.y) : (b.x + b.y) / J;
      f2 += fv * fv;
    }
    fzm = fzp;
  }
  if (pr2) {
    const double s = block_sum_f(r2, shr);
    if (is_thread0()) pr2[block_linear_id()] = s;
  }
  if (pf2) {
    const double s = block_sum_f(f2, shr);
    if (is_thread0()) pf2[block_linear_id()] = s;
  }
}

}  // namespace

cudaError_t launch_psibar(cudaStream_t st, Dims d, const double* psi, const double* phi, const float2* lam,
                          const double* delta, const double* mw_dev, const double* slam_dev, double h, int sym,
                          float2* S, double* out) {
  int ex;
  if (!(h > 0.0) || std::frexp(h, &ex) != 0.5 || ex < -20 || ex > 20) return cudaErrorInvalidValue;  // h = 2^l
  k_psibar_tiled<<<curv_tiled_grid(d), CNT, 0, st>>>(d, psi, phi, lam, delta, mw_dev, slam_dev, (float)(1.0 / h), sym,
                                                    S, curv_zchunk(d));
  note_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_psibar_H<<<cell_grid(d), dim3(BX, BY), 0, st>>>(d, S, (float)(1.0 / (h * h)), out);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_jscale(cudaStream_t st, long long n, const float2* lam, const float* J, const double* s_dev,
                          double* out, double* lam64) {
  k_jscale<<<(int)df_partial_count(n), 256, 0, st>>>(n, lam, J, s_dev, out, lam64);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_geom(cudaStream_t st, Dims d, const double* psi, double h, CurvCoefOut out) {
  int ex;
  if (!(h > 0.0) || std::frexp(h, &ex) != 0.5 || ex < -20 || ex > 20) return cudaErrorInvalidValue;  // h = 2^l
  k_geom_tiled<<<curv_tiled_grid(d), CNT, 0, st>>>(d, psi, (float)(1.0 / (h * h)), out, curv_zchunk(d));
  note_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_curv_apply(cudaStream_t st, Dims d, CurvCoef cf, const T* u, T* out, int form, int divide_J) {
  k_curv_apply<T><<<cell_grid(d), dim3(BX, BY), 0, st>>>(d, cf, u, out, (T)(1.0 / cf.h2), form, divide_J);
  note_launch();
  return cudaGetLastError();
}

long long curv_partial_count(Dims d) {
  const dim3 g = curv_tiled_grid(d);
  return (long long)g.x * g.y * g.z;
}

// FP32 sweeps and residuals of levels of at most 32^3 cells run one thread per cell
// (k_curv_jacobi / k_curv_residual: every load of a cell in one round) instead of the
// z-streaming tiles, whose few CTAs there take one dependent round of loads per plane.
// Both evaluate the same operator templates in the same order, so the results are the
// same bits (the moving-mesh solve's phi, delta-bar and psi-bar were compared).
static bool curv_cellwise(Dims d) { return (long long)d.nx * d.ny * d.nz <= 32 * 32 * 32; }

template <typename T>
cudaError_t launch_curv_residual(cudaStream_t st, Dims d, CurvCoef cf, const T* r, const T* u, T* out, int form,
                                 double* partials) {
  if (form < 0 || form > 2) return cudaErrorInvalidValue;
  if (sizeof(T) == 4 && !partials && curv_cellwise(d)) {
    k_curv_residual<T><<<cell_grid(d), dim3(BX, BY), 0, st>>>(d, cf, r, u, out, (T)(1.0 / cf.h2), form, partials);
  } else if constexpr (sizeof(T) == 4) {
    const size_t sm = 4 * ring_slot_bytes<float>();
    const float ih2 = (float)(1.0 / cf.h2);
    const dim3 g = curv_tiled_grid(d);
    const int zc = curv_zchunk(d);
    if (form == 2) k_curv_tiled<CM_RESID, 2><<<g, CNT, sm, st>>>(d, cf, r, u, out, 0.f, ih2, partials, zc);
    else if (form == 1) k_curv_tiled<CM_RESID, 1><<<g, CNT, sm, st>>>(d, cf, r, u, out, 0.f, ih2, partials, zc);
    else k_curv_tiled<CM_RESID, 0><<<g, CNT, sm, st>>>(d, cf, r, u, out, 0.f, ih2, partials, zc);
  } else {
    k_curv_residual<T><<<cell_grid(d), dim3(BX, BY), 0, st>>>(d, cf, r, u, out, (T)(1.0 / cf.h2), form, partials);
  }
  note_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_curv_jacobi(cudaStream_t st, Dims d, CurvCoef cf, const T* r, const T* e_in, T* e_out, int form,
                               T omega) {
  if (form < 0 || form > 2) return cudaErrorInvalidValue;
  if (sizeof(T) == 4 && curv_cellwise(d)) {
    k_curv_jacobi<T><<<cell_grid(d), dim3(BX, BY), 0, st>>>(d, cf, r, e_in, e_out, form, omega);
  } else if constexpr (sizeof(T) == 4) {
    const size_t sm = 4 * ring_slot_bytes<float>();
    const dim3 g = curv_tiled_grid(d);
    const int zc = curv_zchunk(d);
    if (form == 2) k_curv_tiled<CM_JACOBI, 2><<<g, CNT, sm, st>>>(d, cf, r, e_in, e_out, omega, 0.f, nullptr, zc);
    else if (form == 1) k_curv_tiled<CM_JACOBI, 1><<<g, CNT, sm, st>>>(d, cf, r, e_in, e_out, omega, 0.f, nullptr, zc);
    else k_curv_tiled<CM_JACOBI, 0><<<g, CNT, sm, st>>>(d, cf, r, e_in, e_out, omega, 0.f, nullptr, zc);
  } else {
    k_curv_jacobi<T><<<cell_grid(d), dim3(BX, BY), 0, st>>>(d, cf, r, e_in, e_out, form, omega);
  }
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_curv_jacobi_zero(cudaStream_t st, Dims d, CurvCoef cf, const float* r, float* e_out, int form,
                                    float omega) {
  if (form < 0 || form > 2) return cudaErrorInvalidValue;
  if (form == 2) k_curv_jacobi_zero<2><<<cell_grid(d), dim3(BX, BY), 0, st>>>(d, cf, r, e_out, omega);
  else k_curv_jacobi_zero<0><<<cell_grid(d), dim3(BX, BY), 0, st>>>(d, cf, r, e_out, omega);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_curv_dense(cudaStream_t st, Dims d, CurvCoef cf, int form, double* out) {
  const long long n = ncell(d);
  k_curv_dense<<<(unsigned)((n * n + 255) / 256), 256, 0, st>>>(d, cf, form, out);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_curv_df_residual(cudaStream_t st, Dims d, CurvCoef cf, const float2* src, const double* m_dev,
                                    int scale_J, const float2* u, int form, float* r, double* pr2, double* pf2) {
  if (form < 0 || form > 2) return cudaErrorInvalidValue;
  k_curv_df_residual_tiled<<<curv_tiled_grid(d), CNT, 4 * ring_slot_bytes<float2>(), st>>>(
      d, cf, src, m_dev, scale_J, u, form, r, pr2, pf2, curv_zchunk(d));
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_wsum(cudaStream_t st, long long n, const double* x, const float* J, double* pxj, double* pj) {
  k_wsum<<<(int)df_partial_count(n), 256, 0, st>>>(n, x, J, pxj, pj);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_ratio(cudaStream_t st, const double* a, const double* b, double* out) {
  k_ratio<<<1, 32, 0, st>>>(a, b, out);
  note_launch();
  return cudaGetLastError();
}

template cudaError_t launch_curv_apply<float>(cudaStream_t, Dims, CurvCoef, const float*, float*, int, int);
template cudaError_t launch_curv_apply<double>(cudaStream_t, Dims, CurvCoef, const double*, double*, int, int);
template cudaError_t launch_curv_residual<float>(cudaStream_t, Dims, CurvCoef, const float*, const float*, float*, int, double*);
template cudaError_t launch_curv_residual<double>(cudaStream_t, Dims, CurvCoef, const double*, const double*, double*, int, double*);
template cudaError_t launch_curv_jacobi<float>(cudaStream_t, Dims, CurvCoef, const float*, const float*, float*, int, float);
template cudaError_t launch_curv_jacobi<double>(cudaStream_t, Dims, CurvCoef, const double*, const double*, double*, int, double);

}  // namespace gbmg
