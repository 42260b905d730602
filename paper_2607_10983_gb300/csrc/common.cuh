// Shared device helpers for the multigrid kernels: periodic indexing, double-float
// (two-FP32) arithmetic, FP64 <-> double-float conversion by integer bit operations,
// and deterministic block reductions.
//
// Why double-float: on this GPU the FP64 pipe (FMA and conversions alike) issues
// about 1.6 operations per clock per SM against about 117 for FP32, so every
// per-cell operation of the hot path is FP32 or integer.  The outer residual of
// the defect correction (Sec. 3.2) needs more than FP32 because the potential of
// a k^-2 source is dominated by long waves and A phi cancels by a factor
// |phi|/|A phi| ~ (N/2pi)^2; a pair (hi, lo) of floats carries ~48 bits.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "host_math.h"

namespace gbmg {

__host__ __device__ __forceinline__ long long ncell(Dims d) { return (long long)d.nx * d.ny * d.nz; }

__device__ __forceinline__ int wrap_lo(int i, int n) { return i < 0 ? i + n : i; }
__device__ __forceinline__ int wrap_hi(int i, int n) { return i >= n ? i - n : i; }
__device__ __forceinline__ int wrapi(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }
__device__ __forceinline__ long long lin(Dims d, int x, int y, int z) {
  return ((long long)z * d.ny + y) * d.nx + x;
}

// ------------------------------------------------------------------ double-float

// Error-free sum: s + e == a + b exactly (Knuth).  No multiplications, so no FMA
// contraction can alter it; the build never uses fast-math.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// Error-free sum when |a| >= |b| (Dekker).
__device__ __forceinline__ void quick_two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  e = b - (s - a);
}

// (hi, lo) + f, renormalised.
__device__ __forceinline__ float2 df_add_f(float2 a, float b) {
  float s, e;
  two_sum(a.x, b, s, e);
  e += a.y;
  float h, l;
  quick_two_sum(s, e, h, l);
  return make_float2(h, l);
}

// (hi, lo) + (hi, lo), renormalised.
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
  float s, e;
  two_sum(a.x, b.x, s, e);
  e += a.y + b.y;
  float h, l;
  quick_two_sum(s, e, h, l);
  return make_float2(h, l);
}

// Compensated accumulator: value = s + c.  add() keeps s exact up to the
// rounding of c, which only ever sums tiny error terms.
struct DfAcc {
  float s, c;
  __device__ __forceinline__ void add(float t) {
    float ns, e;
    two_sum(s, t, ns, e);
    s = ns;
    c += e;
  }
};

// FP64 -> (hi, lo) with hi = RN24(x), lo = RN24(x - hi), by integer operations.
// |x| below 2^-126 flushes to zero; |x| at or above 2^128 gives +-inf; NaN stays NaN.
__device__ __forceinline__ float2 f64_to_df(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hw = (unsigned)(b >> 32), lw = (unsigned)b;
  const unsigned sign = hw & 0x80000000u;
  const int e = (int)((hw >> 20) & 0x7ffu);
  if (e == 0) return make_float2(__uint_as_float(sign), 0.0f);
  if (e == 0x7ff) {
    const bool nan = ((hw & 0xfffffu) | lw) != 0u;
    return make_float2(__uint_as_float(sign | (nan ? 0x7fc00000u : 0x7f800000u)), 0.0f);
  }
  const int E0 = e - 1023;
  unsigned mh = ((hw & 0xfffffu) << 3) | (lw >> 29);   // top 23 fraction bits
  const unsigned rem = lw & 0x1fffffffu;                // remaining 29 bits
  int rem_s = (int)rem;
  if (rem > 0x10000000u || (rem == 0x10000000u && (mh & 1u))) {
    mh += 1u;
    rem_s = (int)rem - 0x20000000;
  }
  int E = E0;
  if (mh == 0x800000u) {
    mh = 0u;
    E += 1;
  }
  if (E > 127) return make_float2(__uint_as_float(sign | 0x7f800000u), 0.0f);
  if (E < -126) return make_float2(__uint_as_float(sign), 0.0f);
  const float hi = __uint_as_float(sign | ((unsigned)(E + 127) << 23) | mh);
  // lo = sign * |rem_s| * 2^k, k = E0 - 52, rounded once to float.
  const unsigned a = (unsigned)(rem_s < 0 ? -rem_s : rem_s);   // < 2^29
  const int k = E0 - 52;
  float lo;
  if (k >= -126) {
    lo = (float)a * __uint_as_float((unsigned)(k + 127) << 23);   // exact scaling of RN(a)
  } else {
    const int j = -126 - k;                                          // normal iff a >= 2^j
    if (j < 29 && a >= (1u << j)) {
      lo = (float)a * __uint_as_float((unsigned)(k + 64 + 127) << 23) * 5.421010862427522e-20f;  // * 2^-64
    } else {
      // subnormal result: keep a * 2^(k + 149) rounded half-to-even as the bit pattern
      const int s = j - 23;
      unsigned m;
      if (s <= 0) {
        m = a << (-s);
      } else if (s >= 30) {
        m = 0u;
      } else {
        m = a >> s;
        const unsigned rest = a & ((1u << s) - 1u), half = 1u << (s - 1);
        if (rest > half || (rest == half && (m & 1u))) m += 1u;
      }
      lo = __uint_as_float(m);
    }
  }
  // the remainder is negative when hi was rounded up
  return make_float2(hi, ((sign != 0u) != (rem_s < 0)) ? -lo : lo);
}

// (hi, lo) -> FP64 by integer operations, for a normalised pair (|lo| <= ulp(hi)).
// Rounds the low part's bits below 2^-53 of hi toward zero (error < 2^-52 relative).
__device__ __forceinline__ double df_to_f64(float2 v) {
  const unsigned hb = __float_as_uint(v.x), lb = __float_as_uint(v.y);
  const unsigned eh = (hb >> 23) & 0xffu;
  const unsigned long long sgn = (unsigned long long)(hb >> 31) << 63;
  if (eh == 0u) return __longlong_as_double((long long)sgn);
  if (eh == 0xffu) {
    const bool nan = (hb & 0x7fffffu) != 0u;
    return __longlong_as_double((long long)(sgn | (nan ? 0x7ff8000000000000ull : 0x7ff0000000000000ull)));
  }
  long long S = (long long)(((unsigned long long)((hb & 0x7fffffu) | 0x800000u)) << 29);
  const int Eh = (int)eh - 127;
  const unsigned el = (lb >> 23) & 0xffu;
  if (el != 0xffu && (lb & 0x7fffffffu) != 0u) {
    // a subnormal low part has no implicit bit and the exponent of 2^-126
    const long long Lm = (long long)(el ? ((lb & 0x7fffffu) | 0x800000u) : (lb & 0x7fffffu));
    const int sh = (int)(el ? el : 1u) - 127 - Eh + 29;
    long long L = 0;
    if (sh >= 0) {
      L = sh <= 38 ? (Lm << sh) : 0;   // unnormalised pairs beyond this are not produced
    } else if (sh > -40) {
      L = Lm >> (-sh);
    }
    if ((lb ^ hb) & 0x80000000u) S -= L; else S += L;
  }
  int adj = 0;
  if (S >= (1ll << 53)) {
    S >>= 1;
    adj = 1;
  } else if (S < (1ll << 52)) {
    if (S <= 0) return 0.0;   // only reachable for unnormalised input
    S <<= 1;
    adj = -1;
  }
  const unsigned long long bits =
      sgn | ((unsigned long long)(Eh + adj + 1023) << 52) | ((unsigned long long)S & 0xfffffffffffffull);
  return __longlong_as_double((long long)bits);
}

// ------------------------------------------------------------------ reductions

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the block (any blockDim up to 1024, multiple of 32); result valid in thread 0.
// `sh` needs 32 doubles.  Fixed order: deterministic run to run.
__device__ __forceinline__ double block_sum(double v, double* sh) {
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int nt = blockDim.x * blockDim.y * blockDim.z;
  v = warp_sum(v);
  __syncthreads();
  if ((tid & 31) == 0) sh[tid >> 5] = v;
  __syncthreads();
  double r = 0.0;
  if (tid < 32) {
    r = tid < (nt + 31) / 32 ? sh[tid] : 0.0;
    r = warp_sum(r);
  }
  return r;
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block sum of one float per thread: warp sums in FP32, then FP64 across warps
// (one FP64 operation per warp, not per cell).  Result valid in thread 0.
__device__ __forceinline__ double block_sum_f(float v, double* sh) {
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int nt = blockDim.x * blockDim.y * blockDim.z;
  v = warp_sum_f(v);
  __syncthreads();
  if ((tid & 31) == 0) sh[tid >> 5] = (double)v;
  __syncthreads();
  double r = 0.0;
  if (tid < 32) {
    r = tid < (nt + 31) / 32 ? sh[tid] : 0.0;
    r = warp_sum(r);
  }
  return r;
}

// Block sum of per-thread compensated sums (s + c): each thread's pair goes to FP64
// once, then a deterministic FP64 block reduction.  Result valid in thread 0.
__device__ __forceinline__ double block_sum_acc(const DfAcc& a, double* sh) {
  return block_sum((double)a.s + (double)a.c, sh);
}

__device__ __forceinline__ int block_linear_id() {
  return blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
}

__device__ __forceinline__ bool is_thread0() {
  return threadIdx.x == 0 && threadIdx.y == 0 && threadIdx.z == 0;
}

}  // namespace gbmg
