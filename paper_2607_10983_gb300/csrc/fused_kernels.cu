// Fused double-float kernel of the finest level: phi' = phi + e in double-float and
// the next defect-correction residual r' = F - m - A phi' (Sec. 3.2) in one pass.
//
// A CTA owns an output tile of TX x TY cells in (x, y) and a chunk of z planes; it
// updates phi on the tile plus a one-cell halo, keeps the current plane in a padded,
// double-buffered shared-memory plane (x/y neighbours) and the two older z planes in
// registers, and forms the residual one plane behind.  One barrier per plane.
#include <cstdio>

#include "kernels.h"
#include "stencil.cuh"

namespace gbmg {

namespace {

__device__ __forceinline__ int wrapmod(int i, int n) {
  const int r = i % n;
  return r < 0 ? r + n : r;
}

template <int TX, int TY, int H, int NT>
struct Tile {
  static constexpr int WX = TX + 2 * H;
  static constexpr int WY = TY + 2 * H;
  static constexpr int NPOS = WX * WY;
  static constexpr int K = (NPOS + NT - 1) / NT;  // positions per thread
  static constexpr int PAD = WX + 1;              // padding so p +- 1, p +- WX stay in bounds
  // every thread slot (valid or not) owns a plane entry, so no slot needs a guard
  static constexpr int PLANE = K * NT + 2 * PAD;
};

// Per-thread position bookkeeping: plane offset of each owned position in the
// (wrapped) global mesh, and bit masks of valid / in-tile positions.
template <int TX, int TY, int H, int NT>
struct Positions {
  using TL = Tile<TX, TY, H, NT>;
  int goff[TL::K];
  unsigned vmask = 0, tmask = 0;
  __device__ __forceinline__ void init(Dims d, int x0, int y0) {
#pragma unroll
    for (int k = 0; k < TL::K; ++k) {
      const int p = threadIdx.x + k * NT;
      goff[k] = 0;
      if (p < TL::NPOS) {
        const int px = p % TL::WX, py = p / TL::WX;
        const int ux = x0 - H + px, uy = y0 - H + py;
        goff[k] = wrapmod(ux, d.nx) + wrapmod(uy, d.ny) * d.nx;
        vmask |= 1u << k;
        if (px >= H && px < H + TX && py >= H && py < H + TY && ux < d.nx && uy < d.ny) tmask |= 1u << k;
      }
    }
  }
};

// ------------------------------------------------------------------ finest level, double-float

// phi' = phi + e (double-float) on the tile plus a one-cell halo, then
// r' = F - m - A phi' on the tile; block partial sums of r'^2 and of phi'.
// Loads of the next plane are issued before the current plane is processed.
template <int TX, int TY, int NT>
__global__ void __launch_bounds__(NT)
k_df_update_residual(Dims d, const float2* __restrict__ phi_in, const float* __restrict__ e,
                     const float2* __restrict__ F, const double* __restrict__ m_dev, float2* __restrict__ phi_out,
                     float* __restrict__ r_out, double* __restrict__ pr2, double* __restrict__ psum,
                     double* __restrict__ pf2, int zc) {
  constexpr int H = 1;
  using TL = Tile<TX, TY, H, NT>;
  constexpr int WX = TL::WX, K = TL::K, PLANE = TL::PLANE, PAD = TL::PAD;
  __shared__ float2 sp[2][PLANE];
  __shared__ double shr[32];
  const int tid = threadIdx.x;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * zc;
  const int zend = min(z0 + zc, d.nz);
  const long long pst = (long long)d.nx * d.ny;
  Positions<TX, TY, H, NT> P;
  P.init(d, x0, y0);
  const float2 m = f64_to_df(m_dev[0]);
  float2 wp[K], wc[K];
  float2 nphi[K], fq[K];
  float ne[K];
  float r2 = 0.f, f2 = 0.f;
  DfAcc ps{0.f, 0.f};
#pragma unroll
  for (int k = 0; k < K; ++k) wp[k] = wc[k] = fq[k] = make_float2(0.f, 0.f);
#pragma unroll
  for (int k = 0; k < K; ++k) ne[k] = 0.f;
  const int tb = z0 - 1, te = zend;
  auto load = [&](int t) {
    const long long base = (long long)wrapmod(t, d.nz) * pst;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const bool v = P.vmask >> k & 1u;
      nphi[k] = v ? phi_in[base + P.goff[k]] : make_float2(0.f, 0.f);
      if (e) ne[k] = v ? __ldg(e + base + P.goff[k]) : 0.f;
    }
  };
  load(tb);
  for (int t = tb; t <= te; ++t) {
    const int cur = (t - tb) & 1, prv = cur ^ 1;
    const long long base = (long long)wrapmod(t, d.nz) * pst;
    float2 pn[K];
    float2 fcur[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      pn[k] = e ? df_add_f(nphi[k], ne[k]) : nphi[k];
      fcur[k] = fq[k];
    }
    if (t < te) {
      load(t + 1);
      // F of the plane whose residual the next iteration computes (plane t)
      if (t >= z0 && t < zend) {
#pragma unroll
        for (int k = 0; k < K; ++k) fq[k] = (P.tmask >> k & 1u) ? F[base + P.goff[k]] : make_float2(0.f, 0.f);
      }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if (P.vmask >> k & 1u) {
        sp[cur][PAD + tid + k * NT] = pn[k];
        if ((P.tmask >> k & 1u) && t >= z0 && t < zend) {
          if (phi_out) phi_out[base + P.goff[k]] = pn[k];
          ps.add(pn[k].x);
          ps.c += pn[k].y;
        }
      }
    }
    const int zp = t - 1;
    if (zp >= z0 && zp < zend) {
      const float2* src = sp[prv] + PAD;
      const long long pbase = (long long)zp * pst;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        if (P.tmask >> k & 1u) {
          const int p = tid + k * NT;
          const long long gi = pbase + P.goff[k];
          const float rv = df_resid(wc[k], src[p - 1], src[p + 1], src[p - WX], src[p + WX], wp[k], pn[k], fcur[k], m);
          r_out[gi] = rv;
          r2 += rv * rv;
          const float fv = __fadd_rn(__fsub_rn(fcur[k].x, m.x), __fsub_rn(fcur[k].y, m.y));
          f2 += fv * fv;
        }
      }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
      wp[k] = wc[k];
      wc[k] = pn[k];
    }
    __syncthreads();
  }
  const double b2 = block_sum_f(r2, shr);
  const double bs = block_sum_acc(ps, shr);
  const double bf = pf2 ? block_sum_f(f2, shr) : 0.0;
  if (tid == 0) {
    const int bid = block_linear_id();
    pr2[bid] = b2;
    psum[bid] = bs;
    if (pf2) pf2[bid] = bf;
  }
}

constexpr int FTX = 64, FTY = 16, FNT = 256;   // double-float update tile

}  // namespace

// ---- double-float update

// z chunk of the double-float update: at least four waves of three CTAs per SM, so
// that enough loads are in flight; the warm-up costs one plane per chunk.
int df_zchunk(Dims d) {
  const long long tiles = (long long)((d.nx + FTX - 1) / FTX) * ((d.ny + FTY - 1) / FTY);
  int zc = d.nz;
  while (zc > 16 && tiles * ((d.nz + zc - 1) / zc) < 4 * 3 * 152) zc = (zc + 1) / 2;
  return zc;
}

long long df_update_residual_partials(Dims d) {
  const int zc = df_zchunk(d);
  return (long long)((d.nx + FTX - 1) / FTX) * ((d.ny + FTY - 1) / FTY) * ((d.nz + zc - 1) / zc);
}

cudaError_t launch_df_update_residual(cudaStream_t st, Dims d, const float2* phi_in, const float* e, const float2* F,
                                      const double* m_dev, float2* phi_out, float* r_out, double* pr2, double* psum,
                                      double* pf2) {
  const int zc = df_zchunk(d);
  const dim3 grid((d.nx + FTX - 1) / FTX, (d.ny + FTY - 1) / FTY, (d.nz + zc - 1) / zc);
  k_df_update_residual<FTX, FTY, FNT><<<grid, FNT, 0, st>>>(d, phi_in, e, F, m_dev, phi_out, r_out, pr2, psum, pf2, zc);
  note_launch();
  return cudaGetLastError();
}

}  // namespace gbmg
