// Streaming form of the pre-evaluated elasticity kernel (P1-P3, FP32
// contraction): same arithmetic as PreVecTile (Algorithm 2 with the
// factorised block tr(M X) I + adj^T (X^T + L) adj, blocks a <= b mirrored),
// run by the batched streaming schedule (stream_batched.cuh).  Every compute
// thread owns one pair (a, b) of one element slot for the whole launch and
// keeps its 36 reference values in registers; the producer warp turns each
// element's coordinates and P1 coefficients into the FP64-derived record
// (adj, M = adj adj^T, mu, lam, 1/|det J|).
#pragma once
#include "common.cuh"
#include "pre_vec.cuh"
#include "stream_batched.cuh"
#include "sym.cuh"

namespace fea {

template <int P>
struct VecStreamPolicy {
  static constexpr int NS = nbasis_c(P);
  static constexpr int N = 3 * NS;
  static constexpr int NN = N * N;
  static constexpr int S = NS * NS;
  static constexpr int NP = NS * (NS + 1) / 2;
  static constexpr int TE = kStreamCompute / NP;  // element slots per tile
  static_assert(TE >= 1, "one element's pairs must fit the compute warps");
  static constexpr int GEO = 32;
  static constexpr int MINB = 3;

  __device__ static void record(const Req& q, int64_t e, float* g, unsigned* err) {
    double x[12], c[8];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      const double2 v = __ldg(reinterpret_cast<const double2*>(q.coords + e * 12) + i);
      x[2 * i] = v.x;
      x[2 * i + 1] = v.y;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const double2 v = __ldg(reinterpret_cast<const double2*>(q.coeffs + e * 8) + i);
      c[2 * i] = v.x;
      c[2 * i + 1] = v.y;
    }
    pre_vec_record<float>(x, c, g, err);
  }

  struct Thread {
    bool comp;
    int slot, a, b;
    float R[36];
    __device__ Thread(const Req& q, int t) : comp(t < TE * NP), slot(t / NP), a(0), b(0) {
      if (!comp) return;
      const unsigned ab = kSymPairs<NS>.c[t - slot * NP];
      a = (int)(ab & 0xffu);
      b = (int)(ab >> 8);
      const TabLayout L = tab_layout(q.Q, NS, 36);
      const float* Rg = reinterpret_cast<const float*>(q.tab) + L.offR;  // [(k,al,be)][a][b]
#pragma unroll
      for (int r = 0; r < 36; ++r) R[r] = __ldg(Rg + (size_t)r * S + a * NS + b);
    }
    // this thread's block (and its mirror) of element `slot` of the tile; false if it has none
    __device__ bool tile(const float* geo, int ne, char* stage, int out_f32) {
      if (!(comp && slot < ne)) return false;
      const float* g = geo + (size_t)slot * GEO;
      float v[9];
      pre_vec_block<float>(g, R, v);
      if (out_f32) {
        put_sym_block<N, float>(reinterpret_cast<float*>(stage) + (size_t)slot * NN, a, b, v);
      } else {
        const bool bad = g[26] != g[26];
        double d[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) d[i] = bad ? __longlong_as_double(0x7ff8000000000000ll) : f2d_finite(v[i]);
        put_sym_block<N, double>(reinterpret_cast<double*>(stage) + (size_t)slot * NN, a, b, d);
      }
      return true;
    }
  };
};

}  // namespace fea
