// Building blocks of the symmetric vector kernels: packed two-lane arithmetic
// and the tables that split the upper triangle of an element matrix's blocks
// among threads.
//
// Both vector tangents (linear elasticity, Neo-Hookean) are symmetric:
// A_e[(a,c)][(b,d)] = A_e[(b,d)][(a,c)], the Hessian of an energy.  The kernels
// evaluate the 3x3 blocks (a, b) with a <= b only and write each one twice,
// as itself and transposed at (b, a).
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace fea {

// Two-lane arithmetic: float2 maps to the packed FP32x2 FMA (one instruction
// for two lanes; same FMA-pipe rate as two scalar FMAs, half the issue slots);
// double2 falls back to two scalar FP64 FMAs.
template <typename T> struct Vec2Of;
template <> struct Vec2Of<float> { using type = float2; };
template <> struct Vec2Of<double> { using type = double2; };

__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ double2 vfma(double2 a, double2 b, double2 c) {
  return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
}
__device__ __forceinline__ float2 vmk(float x, float y) { return make_float2(x, y); }
__device__ __forceinline__ double2 vmk(double x, double y) { return make_double2(x, y); }

// Four consecutive T from 16-byte aligned shared memory.
template <typename T>
__device__ __forceinline__ void ld4(const T* p, T& x, T& y, T& z, T& w) {
  if constexpr (sizeof(T) == 4) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    x = v.x; y = v.y; z = v.z; w = v.w;
  } else {
    const double2 u = *reinterpret_cast<const double2*>(p);
    const double2 v = *reinterpret_cast<const double2*>(p + 2);
    x = u.x; y = u.y; z = v.x; w = v.y;
  }
}

// Runs of trial functions b >= a of one test function a ("chunks"), at most
// BB long; each row of the upper triangle is cut into runs of near-equal
// length and the runs are listed longest first, so that the threads of a warp
// hold runs of the same length.  Entry: a | b0 << 8 | nb << 16.
template <int NS, int BB>
struct SymChunks {
  static constexpr int count() {
    int n = 0;
    for (int a = 0; a < NS; ++a) n += (NS - a + BB - 1) / BB;
    return n;
  }
  static constexpr int NCH = count();
  unsigned c[NCH];
  constexpr SymChunks() : c() {
    int k = 0;
    for (int s = BB; s >= 1; --s)
      for (int a = 0; a < NS; ++a) {
        const int m = NS - a, cnt = (m + BB - 1) / BB, q = m / cnt, r = m % cnt;
        int b = a;
        for (int j = 0; j < cnt; ++j) {
          const int sz = j < r ? q + 1 : q;
          if (sz == s) c[k++] = (unsigned)a | ((unsigned)b << 8) | ((unsigned)sz << 16);
          b += sz;
        }
      }
  }
};
template <int NS, int BB>
__constant__ SymChunks<NS, BB> kSymChunks{};

// Blocks (a, b) with a <= b in row-major order.  Entry: a | b << 8.
template <int NS>
struct SymPairs {
  static constexpr int NP = NS * (NS + 1) / 2;
  unsigned c[NP];
  constexpr SymPairs() : c() {
    int k = 0;
    for (int a = 0; a < NS; ++a)
      for (int b = a; b < NS; ++b) c[k++] = (unsigned)a | ((unsigned)b << 8);
  }
};
template <int NS>
__constant__ SymPairs<NS> kSymPairs{};

// Write the 3x3 block v[c][d] of the pair (a, b) into the staged element
// matrix (row length N), and its transpose at (b, a) when a != b.
template <int N, typename T>
__device__ __forceinline__ void put_sym_block(T* st, int a, int b, const T (&v)[9]) {
  T* o = st + (3 * a) * N + 3 * b;
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int d = 0; d < 3; ++d) o[c * N + d] = v[3 * c + d];
  if (a != b) {
    T* m = st + (3 * b) * N + 3 * a;
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int c = 0; c < 3; ++c) m[d * N + c] = v[3 * c + d];
  }
}

}  // namespace fea
