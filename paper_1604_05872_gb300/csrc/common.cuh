// Shared device-side building blocks of the assembly kernels: per-request
// parameters, FP64 geometry, conversions, tile input loads and the coalesced
// output epilogue.  Every tile function runs with NT threads per CTA.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "layout.h"

namespace fea {

// ----------------------------------------------------------------------------
// Conversions written from the IEEE-754 binary32/binary64 encodings with
// integer operations.  On GB300 the F2F conversion instructions issue on the
// FP64 pipe (about 2 lane-operations per SM per clock), so converting every
// output entry with them would cost more than the HBM traffic; these run on the
// 32-bit integer pipe instead.
// ----------------------------------------------------------------------------

// Widening float -> double, exact for every normal float; zero and subnormal
// inputs give a signed zero (FP32 arithmetic here runs with flush-to-zero, so
// subnormals do not arise), inf and NaN stay inf and NaN.  Integer operations
// only: a data-dependent fallback to the hardware conversion would be
// if-converted into a predicated FP64-pipe instruction on every call.
__device__ __forceinline__ double f2d(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t a = u & 0x7fffffffu;
  uint32_t hi = (a >> 3) + 0x38000000u;  // exponent rebias by 1023 - 127
  uint32_t lo = a << 29;
  const bool small = a < 0x00800000u;
  const bool big = a >= 0x7f800000u;
  hi = small ? 0u : hi;
  lo = small ? 0u : lo;
  hi = big ? (0x7ff00000u | ((a & 0x007fffffu) ? 0x00080000u : 0u)) : hi;
  return __hiloint2double((int)(hi | (u & 0x80000000u)), (int)lo);
}

// double -> float, round to nearest even.  Results below the smallest normal
// float flush to signed zero; overflow gives inf; NaN stays NaN.
__device__ __forceinline__ float d2f(double x) {
  const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
  const uint32_t sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7ff);
  const uint32_t mant = ((hi & 0xfffffu) << 3) | (lo >> 29);
  const uint32_t rest = lo & 0x1fffffffu;
  const uint32_t up = (rest > 0x10000000u) | ((rest == 0x10000000u) & (mant & 1u));
  const int fe = e - 896;
  uint32_t f = ((uint32_t)fe << 23) + mant + up;
  if (fe <= 0) f = 0u;
  if (fe >= 255) f = (e == 0x7ff && ((hi & 0xfffffu) | lo)) ? 0x7fc00000u : 0x7f800000u;
  return __uint_as_float(sign | f);
}

// Cheaper conversions for values known to be finite and well scaled (the
// Neo-Hookean kinematics), where the exact special cases of f2d/d2f do not
// matter: f2d_normal widens exactly every normal float and zero (FP32 math here
// flushes subnormals); d2f_rz rounds toward zero, gives a signed zero below the
// float range and NaN above it (callers mark such points degenerate anyway).
__device__ __forceinline__ double f2d_normal(float f) {
  const uint32_t u = __float_as_uint(f), a = u & 0x7fffffffu;
  const uint32_t hi = a == 0u ? 0u : (a >> 3) + 0x38000000u;
  return __hiloint2double((int)(hi | (u & 0x80000000u)), (int)(u << 29));
}
__device__ __forceinline__ float d2f_rz(double x) {
  const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
  // hi << 3 | lo >> 29: the exponent's low 8 bits land on 23..30, the top 23 mantissa bits below;
  // for exponents 897..1150 the float exponent is those 8 bits with the top one flipped
  const uint32_t t = __funnelshift_l(lo, hi, 3);
  const uint32_t e = (hi >> 20) & 0x7ffu, sign = hi & 0x80000000u;
  const uint32_t f = ((t & 0x7fffffffu) ^ 0x40000000u) | sign;
  return __uint_as_float(e - 897u < 254u ? f : (e < 897u ? sign : 0x7fc00000u));
}

// Widening for values that come out of FTZ FP32 arithmetic (no subnormals):
// exact for normal floats, zeros, infinities and NaN.  One 32 x 32 -> 64-bit
// multiply-add places |x| << 29 across the two words with the exponent
// rebias (1023 - 127) << 52 added; zero and inf/NaN are then patched.
__device__ __forceinline__ double f2d_ftz(float f) {
  const uint32_t u = __float_as_uint(f), a = u & 0x7fffffffu;
  const uint64_t w = (uint64_t)a * (1ull << 29) + 0x3800000000000000ull;
  uint32_t hi = (uint32_t)(w >> 32);
  hi = a >= 0x7f800000u ? (hi | 0x7ff00000u) : hi;
  hi = a == 0u ? 0u : hi;
  return __hiloint2double((int)(hi | (u & 0x80000000u)), (int)(uint32_t)w);
}

template <typename T> __device__ __forceinline__ T from_double(double x);
template <> __device__ __forceinline__ double from_double<double>(double x) { return x; }
template <> __device__ __forceinline__ float from_double<float>(double x) { return d2f(x); }

// ----------------------------------------------------------------------------
// Geometry (Section 2.2: the change of variables x = x0 + J X).
// FP64: J (9 subtractions), the adjugate adj = det(J) J^-1 (nine 2x2 minors)
// and det J.  These are the steps where a badly shaped element loses digits to
// cancellation; everything downstream divides or multiplies them only.
// adj[a*3+b] = det(J) * dX_a/dx_b.
// ----------------------------------------------------------------------------
__device__ __forceinline__ double geometry_fp64(const double* x, double adj[9]) {
  double J[3][3];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) J[r][c] = x[3 * (c + 1) + r] - x[r];
  adj[0] = fma(J[1][1], J[2][2], -J[1][2] * J[2][1]);
  adj[1] = fma(J[0][2], J[2][1], -J[0][1] * J[2][2]);
  adj[2] = fma(J[0][1], J[1][2], -J[0][2] * J[1][1]);
  adj[3] = fma(J[1][2], J[2][0], -J[1][0] * J[2][2]);
  adj[4] = fma(J[0][0], J[2][2], -J[0][2] * J[2][0]);
  adj[5] = fma(J[0][2], J[1][0], -J[0][0] * J[1][2]);
  adj[6] = fma(J[1][0], J[2][1], -J[1][1] * J[2][0]);
  adj[7] = fma(J[0][1], J[2][0], -J[0][0] * J[2][1]);
  adj[8] = fma(J[0][0], J[1][1], -J[0][1] * J[1][0]);
  return fma(J[0][0], adj[0], fma(J[0][1], adj[3], J[0][2] * adj[6]));
}

__device__ __forceinline__ void flag_error(unsigned* err, unsigned code) {
  if (err) atomicOr(err, code);
}
constexpr unsigned ERR_DEGENERATE = 1u;
constexpr unsigned ERR_PATTERN = 8u;  // a global-assembly position outside the CSR pattern

// ----------------------------------------------------------------------------
// Tile input: copy `n` doubles from global (8-byte aligned start) to shared
// (16-byte aligned destination) with 16-byte loads where the source allows.
// ----------------------------------------------------------------------------
template <int NTH>
__device__ __forceinline__ void load_doubles(double* dst, const double* __restrict__ src, int n) {
  if ((reinterpret_cast<uintptr_t>(src) & 15) == 0) {
    const int n2 = n >> 1;
    const double2* s2 = reinterpret_cast<const double2*>(src);
    double2* d2 = reinterpret_cast<double2*>(dst);
    for (int k = threadIdx.x; k < n2; k += NTH) d2[k] = __ldg(s2 + k);
    if ((n & 1) && threadIdx.x == 0) dst[n - 1] = __ldg(src + n - 1);
  } else {
    for (int k = threadIdx.x; k < n; k += NTH) dst[k] = __ldg(src + k);
  }
}

// ----------------------------------------------------------------------------
// Epilogue: stage[0 .. cnt) (shared, type T) -> out + out_off (global, double
// or float), coalesced 16-byte (double) / 8-byte (float) stores.  An odd
// starting offset is handled by one scalar head store.
// ----------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ double widen(T v) {
  if constexpr (sizeof(T) == 4) return f2d(v);
  else return (double)v;
}

template <int NTH, typename T>
__device__ __forceinline__ void store_tile(void* out, int64_t out_off, const T* stage, int cnt, int out_f32) {
  const int head = (int)(out_off & 1);
  if (head && threadIdx.x == 0 && cnt > 0) {
    if (out_f32) reinterpret_cast<float*>(out)[out_off] = (float)stage[0];
    else reinterpret_cast<double*>(out)[out_off] = widen<T>(stage[0]);
  }
  const int rest = cnt - head;
  const int n2 = rest >> 1;
  const T* st = stage + head;
  if (out_f32) {
    float2* o = reinterpret_cast<float2*>(reinterpret_cast<float*>(out) + out_off + head);
    for (int k = threadIdx.x; k < n2; k += NTH) {
      float2 v;
      v.x = (float)st[2 * k];
      v.y = (float)st[2 * k + 1];
      __stcs(o + k, v);
    }
  } else {
    double2* o = reinterpret_cast<double2*>(reinterpret_cast<double*>(out) + out_off + head);
    for (int k = threadIdx.x; k < n2; k += NTH) {
      double2 v;
      v.x = widen<T>(st[2 * k]);
      v.y = widen<T>(st[2 * k + 1]);
      __stcs(o + k, v);
    }
  }
  if ((rest & 1) && threadIdx.x == 0) {
    if (out_f32) reinterpret_cast<float*>(out)[out_off + cnt - 1] = (float)stage[cnt - 1];
    else reinterpret_cast<double*>(out)[out_off + cnt - 1] = widen<T>(stage[cnt - 1]);
  }
}

}  // namespace fea
