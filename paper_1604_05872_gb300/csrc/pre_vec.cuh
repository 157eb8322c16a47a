// Pre-evaluated variant for elasticity (Algorithm 2), followed by sharing
// elimination on the pre-evaluated expression (Algorithm 3, step 5).
//
// With pre-evaluated tables R_(k,al,be)[a][b] = int Phi1_k dPhi_a/dX_al dPhi_b/dX_be
// (36 per (a, b)) and the adjugate adj = det(J) J^-1:
//
//   A_e[(a,c)][(b,d)] = sum_(k,al,be) R_(k,al,be)[a][b] H_e[(k,al,be)][c][d]
//   H = (mu_k (d_cd M_al,be + adj_al,d adj_be,c) + lam_k adj_al,c adj_be,d) / |det J|,   M = adj adj^T
//
// Factorising the sums over k and (al, be) out of the (c, d) block gives
//
//   X = sum_k mu_k R_k,  L = sum_k lam_k R_k                     (3x3 each, per a, b)
//   A_e[(a,.)][(b,.)] = ( tr(M X) I + adj^T (X^T + L) adj ) / |det J|
//
// 144 FMA per (a, b) block instead of 324 for the plain geometry-tensor GEMV.
// The tangent is symmetric (block (b, a) is the transpose of block (a, b)), so
// only blocks a <= b are evaluated and each is written twice (sym.cuh).
// Each thread owns one (a, b) pair, keeps its 36 R values in registers and
// sweeps the tile's elements, reading the element's adjugate, M and
// coefficients with broadcast shared loads; results are staged in shared memory
// and written with coalesced 16-byte stores.
#pragma once
#include "common.cuh"
#include "sym.cuh"

namespace fea {

// Per-element record of the pre-evaluated elasticity kernels, from the FP64
// geometry: adj[9], M = adj adj^T [9], mu[4], lam[4], 1/|det J| (NaN for a
// degenerate element), pad to 32.
template <typename T>
__device__ __forceinline__ void pre_vec_record(const double* x, const double* c, T* g, unsigned* err) {
  double adj[9];
  const double det = geometry_fp64(x, adj);
  const bool bad = !(fabs(det) > 0.0) || !isfinite(det);
  if (bad) flag_error(err, ERR_DEGENERATE);
  T a[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) g[k] = a[k] = from_double<T>(adj[k]);
#pragma unroll
  for (int al = 0; al < 3; ++al)
#pragma unroll
    for (int be = 0; be < 3; ++be)
      g[9 + 3 * al + be] = a[3 * al] * a[3 * be] + a[3 * al + 1] * a[3 * be + 1] + a[3 * al + 2] * a[3 * be + 2];
#pragma unroll
  for (int k = 0; k < 8; ++k) g[18 + k] = from_double<T>(c[k]);
  const T nan = T(__int_as_float(0x7fc00000));
  g[26] = bad ? nan : T(1) / from_double<T>(fabs(det));
}

// One 3x3 block (a, b) from the pair's 36 reference values R_(k,al,be) and the
// element record g: v = (tr(M X) I + adj^T (X^T + L) adj) / |det J|.
template <typename T>
__device__ __forceinline__ void pre_vec_block(const T* g, const T (&R)[36], T (&v)[9]) {
  T X[9], Lm[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    X[k] = g[18] * R[k] + g[19] * R[9 + k] + g[20] * R[18 + k] + g[21] * R[27 + k];
    Lm[k] = g[22] * R[k] + g[23] * R[9 + k] + g[24] * R[18 + k] + g[25] * R[27 + k];
  }
  T tr = T(0);
#pragma unroll
  for (int k = 0; k < 9; ++k) tr = fma(g[9 + k], X[k], tr);
  // Z = X^T + L;  P = Z adj;  A = adj^T P
  T Pm[9];
#pragma unroll
  for (int al = 0; al < 3; ++al)
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      T x = T(0);
#pragma unroll
      for (int be = 0; be < 3; ++be) x = fma(X[3 * be + al] + Lm[3 * al + be], g[3 * be + d], x);
      Pm[3 * al + d] = x;
    }
  const T inv = g[26];
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      T x = c == d ? tr : T(0);
#pragma unroll
      for (int al = 0; al < 3; ++al) x = fma(g[3 * al + c], Pm[3 * al + d], x);
      v[3 * c + d] = x * inv;
    }
}

template <int P, typename T>
struct PreVecTile {
  static constexpr int MINB = sizeof(T) == 4 && P == 4 ? 3 : 1;  // resident CTAs per SM
  static constexpr int FORM = 2;
  static constexpr int NS = nbasis_c(P);
  static constexpr int N = 3 * NS;
  static constexpr int NN = N * N;
  static constexpr int S = NS * NS;              // (a, b) slots of the table
  static constexpr int NP = NS * (NS + 1) / 2;   // evaluated pairs a <= b
  static constexpr int CLEN = 8;
  static constexpr int GEO = 32;                 // adj[9], M[9], mu[4], lam[4], 1/|det|, pad

  FEA_HD static int max_tile() { return 64; }
  FEA_HD static size_t off_c(int TE) { return round_up_sz((size_t)TE * 12 * 8, 16); }
  FEA_HD static size_t off_geo(int TE) { return off_c(TE) + round_up_sz((size_t)TE * CLEN * 8, 16); }
  FEA_HD static size_t off_stage(int TE) { return off_geo(TE) + round_up_sz((size_t)TE * GEO * sizeof(T), 16); }
  FEA_HD static size_t smem(int TE, int Q) { (void)Q; return off_stage(TE) + round_up_sz((size_t)TE * NN * sizeof(T), 16); }

  __device__ static void tile(const Req& q, int64_t e0, int ne, char* sm, unsigned* err) {
    const int TE = q.tile;
    double* xs = reinterpret_cast<double*>(sm);
    double* cs = reinterpret_cast<double*>(sm + off_c(TE));
    T* geo = reinterpret_cast<T*>(sm + off_geo(TE));
    T* stage = reinterpret_cast<T*>(sm + off_stage(TE));
    const TabLayout L = tab_layout(q.Q, NS, 36);
    const T* Rg = reinterpret_cast<const T*>(q.tab) + L.offR;  // [(k,al,be)][a][b]
    const int tid = threadIdx.x;

    load_doubles<NT>(xs, q.coords + e0 * 12, ne * 12);
    load_doubles<NT>(cs, q.coeffs + e0 * CLEN, ne * CLEN);
    __syncthreads();
    if (tid < ne) pre_vec_record<T>(xs + 12 * tid, cs + CLEN * tid, geo + GEO * tid, err);
    __syncthreads();

    for (int k = tid; k < NP; k += NT) {
      const unsigned ab = kSymPairs<NS>.c[k];
      const int a = (int)(ab & 0xffu), b = (int)(ab >> 8);
      const int s = a * NS + b;
      T R[36];
#pragma unroll
      for (int r = 0; r < 36; ++r) R[r] = __ldg(Rg + (size_t)r * S + s);
      for (int e = 0; e < ne; ++e) {
        T v[9];
        pre_vec_block<T>(geo + GEO * e, R, v);
        put_sym_block<N, T>(stage + (size_t)e * NN, a, b, v);
      }
    }
    __syncthreads();
    store_tile<NT, T>(q.out, e0 * NN, stage, ne * NN, q.out_f32);
    __syncthreads();
  }
};

}  // namespace fea
