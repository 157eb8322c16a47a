// Element vectors: the linear forms (arity 1) of the paper's setting
// (Section 2: a form of arity 1 gives a vector per element, with no
// test/trial sharing to exploit).
//
//  * LoadVecTile (Helmholtz right-hand side): b_i = int f phi_i with f in the
//    basis' own P_p space.  Pre-evaluated (Algorithm 2): b_e = |det J_e| M f_e
//    with the reference mass matrix M_ik = int phi_i phi_k (the mass form's
//    table), one FP64 |det J| per element and an n x n GEMV.
//  * ResVecTile (Neo-Hookean residual): R_(a,c) = int P(F)_{cx} dphi_a/dx_x
//    with P = mu (F - F^-T) + lam ln det F F^-T.  Factorised through the
//    reference gradients: with T_q = s_q P_q J^-T (3 x 3, per point),
//    R_(a,c) = sum_q sum_k dphi_a/dX_k (X_q) T_q[c][k].  Per point the
//    cofactors of F, det F and ln det F are FP64 (F = I + grad u widened).
//
// Output [E][n] row-major (n = n_p for the load vector, 3 n_p with index
// 3 a + c for the residual), double or float.  Degenerate elements give NaN
// entries and set the error word.
#pragma once
#include "common.cuh"
#include "log_f64.cuh"

namespace fea {

template <typename T>
__device__ __forceinline__ void put_out(void* out, int64_t idx, T v, int out_f32) {
  if (out_f32) reinterpret_cast<float*>(out)[idx] = (float)v;
  else reinterpret_cast<double*>(out)[idx] = widen<T>(v);
}

template <int P, typename T>
struct LoadVecTile {
  static constexpr int NS = nbasis_c(P);
  static constexpr int TE = 256;                 // elements per tile: FP64 geometry on full warps

  FEA_HD static int max_tile() { return TE; }
  FEA_HD static int pref_tile() { return TE; }
  FEA_HD static size_t off_f(int te) { return round_up_sz((size_t)te * 12 * 8, 16); }
  FEA_HD static size_t off_ft(int te) { return off_f(te) + round_up_sz((size_t)te * NS * 8, 16); }
  FEA_HD static size_t off_m(int te) { return off_ft(te) + round_up_sz((size_t)te * NS * sizeof(T), 16); }
  FEA_HD static size_t off_det(int te) { return off_m(te) + round_up_sz((size_t)NS * NS * sizeof(T), 16); }
  FEA_HD static size_t smem(int te, int Q) { (void)Q; return off_det(te) + round_up_sz((size_t)te * sizeof(T), 16); }

  __device__ static void tile(const Req& q, int64_t e0, int ne, char* sm, unsigned* err) {
    const int te = q.tile;
    double* xs = reinterpret_cast<double*>(sm);
    double* fs = reinterpret_cast<double*>(sm + off_f(te));
    T* ft = reinterpret_cast<T*>(sm + off_ft(te));
    T* M = reinterpret_cast<T*>(sm + off_m(te));
    T* adet = reinterpret_cast<T*>(sm + off_det(te));
    const TabLayout L = tab_layout(q.Q, NS, 1);
    const T* Mg = reinterpret_cast<const T*>(q.tab) + L.offR;  // mass form's R_0 = int phi_i phi_k
    const int tid = threadIdx.x;
    load_doubles<NT>(xs, q.coords + e0 * 12, ne * 12);
    load_doubles<NT>(fs, q.coeffs + e0 * NS, ne * NS);
    for (int k = tid; k < NS * NS; k += NT) M[k] = Mg[k];
    __syncthreads();
    if (tid < ne) {  // FP64 det J only (J, then one cofactor expansion)
      const double* x = xs + 12 * tid;
      double J[3][3];
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) J[r][c] = x[3 * (c + 1) + r] - x[r];
      const double det = fma(J[0][0], fma(J[1][1], J[2][2], -J[1][2] * J[2][1]),
                             fma(J[0][1], fma(J[1][2], J[2][0], -J[1][0] * J[2][2]),
                                 J[0][2] * fma(J[1][0], J[2][1], -J[1][1] * J[2][0])));
      const bool bad = !(fabs(det) > 0.0) || !isfinite(det);
      if (bad) flag_error(err, ERR_DEGENERATE);
      adet[tid] = bad ? T(__int_as_float(0x7fc00000)) : from_double<T>(fabs(det));
    }
    for (int k = tid; k < ne * NS; k += NT) ft[k] = from_double<T>(fs[k]);  // each DOF converted once
    __syncthreads();
    for (int w = tid; w < ne * NS; w += NT) {
      const int e = w / NS, i = w - e * NS;
      const T* f = ft + NS * e;
      const T* m = M + NS * i;
      T acc = T(0);
#pragma unroll 5
      for (int k = 0; k < NS; ++k) acc = fma(m[k], f[k], acc);
      put_out<T>(q.out, e0 * NS + w, adet[e] * acc, q.out_f32);
    }
    __syncthreads();
  }
};

template <int P, typename T>
struct ResVecTile {
  static constexpr int NS = nbasis_c(P);
  static constexpr int N = 3 * NS;
  static constexpr int CLEN = 3 * NS;
  static constexpr int TE = P <= 2 ? 32 : P == 3 ? 16 : 8;
  static constexpr int GEO = 12;                 // Jinv[9], |det|
  static constexpr int TW = 12;                  // T_q[3][3] padded
  static constexpr int MINB = sizeof(T) == 4 && P <= 2 ? 3 : 1;  // resident CTAs per SM

  FEA_HD static int max_tile() { return TE; }
  FEA_HD static int pref_tile() { return TE; }
  FEA_HD static size_t off_c(int te) { return round_up_sz((size_t)te * 12 * 8, 16); }
  FEA_HD static size_t off_ct(int te) { return off_c(te) + round_up_sz((size_t)te * CLEN * 8, 16); }
  FEA_HD static size_t off_geo(int te) { return off_ct(te) + round_up_sz((size_t)te * CLEN * sizeof(T), 16); }
  FEA_HD static size_t off_t(int te) { return off_geo(te) + round_up_sz((size_t)te * GEO * sizeof(T), 16); }
  FEA_HD static size_t smem(int te, int Q) { return off_t(te) + round_up_sz((size_t)te * Q * TW * sizeof(T), 16); }

  // The default tile with the form's own rule, (P + 1)^3 points, runs with both as
  // compile-time constants (index arithmetic folds); other tiles and rules at run time.
  static constexpr int QDEF = (P + 1) * (P + 1) * (P + 1);
  __device__ static void tile(const Req& q, int64_t e0, int ne, char* sm, unsigned* err) {
    if (q.tile == TE && q.Q == QDEF) tile_t<TE, QDEF>(q, e0, ne, sm, err);
    else tile_t<0, 0>(q, e0, ne, sm, err);
  }

  template <int TEC, int QC>
  __device__ static void tile_t(const Req& q, int64_t e0, int ne, char* sm, unsigned* err) {
    const int te = TEC ? TEC : q.tile, Q = QC ? QC : q.Q;
    double* xs = reinterpret_cast<double*>(sm);
    double* cs = reinterpret_cast<double*>(sm + off_c(te));
    T* ct = reinterpret_cast<T*>(sm + off_ct(te));
    T* geo = reinterpret_cast<T*>(sm + off_geo(te));
    T* Ts = reinterpret_cast<T*>(sm + off_t(te));
    const TabLayout L = tab_layout(Q, NS, 0);
    const T* tab = reinterpret_cast<const T*>(q.tab);
    const T* Wt = tab + L.offW;
    const T* dphi = tab + L.offDphi;
    const T nan = T(__int_as_float(0x7fc00000));
    const int tid = threadIdx.x;

    load_doubles<NT>(xs, q.coords + e0 * 12, ne * 12);
    load_doubles<NT>(cs, q.coeffs + e0 * CLEN, ne * CLEN);
    __syncthreads();
    if (tid < ne) {
      double adj[9];
      const double det = geometry_fp64(xs + 12 * tid, adj);
      const bool bad = !(fabs(det) > 0.0) || !isfinite(det);
      if (bad) flag_error(err, ERR_DEGENERATE);
      T* g = geo + GEO * tid;
      if constexpr (sizeof(T) == 4) {  // the division is a well-conditioned scaling after rounding
        const float df = d2f(det), inv = 1.0f / df;
#pragma unroll
        for (int k = 0; k < 9; ++k) g[k] = bad ? nan : d2f(adj[k]) * inv;
        g[9] = bad ? nan : fabsf(df);
      } else {
        const double inv = 1.0 / det;
#pragma unroll
        for (int k = 0; k < 9; ++k) g[k] = bad ? nan : adj[k] * inv;
        g[9] = bad ? nan : fabs(det);
      }
    }
    for (int k = tid; k < ne * CLEN; k += NT) ct[k] = from_double<T>(cs[k]);
    __syncthreads();
    const T mu = from_double<T>(q.coeffs[q.E * CLEN]);
    const T lam = from_double<T>(q.coeffs[q.E * CLEN + 1]);

    // per (element, point): T_q = s P J^-T
    for (int w = tid; w < ne * Q; w += NT) {
      const int e = w / Q, qq = w - e * Q;
      const T* Ji = geo + GEO * e;
      const T* u = ct + CLEN * e;
      T gr[9];  // sum_a u_a (x) grad_X phi_a
#pragma unroll
      for (int k = 0; k < 9; ++k) gr[k] = T(0);
      for (int a = 0; a < NS; ++a) {
        const T* dp = dphi + (qq * NS + a) * 3;
        const T d0 = dp[0], d1 = dp[1], d2 = dp[2];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          const T ui = u[3 * a + i];
          gr[3 * i] = fma(ui, d0, gr[3 * i]);
          gr[3 * i + 1] = fma(ui, d1, gr[3 * i + 1]);
          gr[3 * i + 2] = fma(ui, d2, gr[3 * i + 2]);
        }
      }
      T gu[9];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int x = 0; x < 3; ++x) gu[3 * i + x] = gr[3 * i] * Ji[x] + gr[3 * i + 1] * Ji[3 + x] + gr[3 * i + 2] * Ji[6 + x];
      double F[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) F[k] = widen<T>(gu[k]);
      F[0] += 1.0; F[4] += 1.0; F[8] += 1.0;
      double cof[9];  // det(F) F^-1
      cof[0] = fma(F[4], F[8], -F[5] * F[7]);
      cof[1] = fma(F[2], F[7], -F[1] * F[8]);
      cof[2] = fma(F[1], F[5], -F[2] * F[4]);
      cof[3] = fma(F[5], F[6], -F[3] * F[8]);
      cof[4] = fma(F[0], F[8], -F[2] * F[6]);
      cof[5] = fma(F[2], F[3], -F[0] * F[5]);
      cof[6] = fma(F[3], F[7], -F[4] * F[6]);
      cof[7] = fma(F[1], F[6], -F[0] * F[7]);
      cof[8] = fma(F[0], F[4], -F[1] * F[3]);
      const double dF = fma(F[0], cof[0], fma(F[1], cof[3], F[2] * cof[6]));
      const bool bad = !(dF > 0.0) || !isfinite(dF);
      if (bad) flag_error(err, ERR_DEGENERATE);
      const T idF = T(1) / from_double<T>(dF);
      const T lnJ = from_double<T>(log_f64(dF));
      const T s = Wt[qq] * Ji[9];
      // P = mu (F - F^-T) + lam lnJ F^-T with F - F^-T = grad u + F^-T grad u^T
      // (I - F^-T = F^-T (F^T - I)): no cancellation for small displacements.
      // Fi[x][c] = cof[3x + c] / det F.
      T Fi[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) Fi[k] = from_double<T>(cof[k]) * idF;
      T Pm[9];
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int x = 0; x < 3; ++x) {
          const T ft = Fi[c] * gu[3 * x] + Fi[3 + c] * gu[3 * x + 1] + Fi[6 + c] * gu[3 * x + 2];
          Pm[3 * c + x] = mu * (gu[3 * c + x] + ft) + lam * lnJ * Fi[3 * x + c];
        }
      T* o = Ts + (size_t)TW * w;
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int k = 0; k < 3; ++k)  // T[c][k] = s sum_x P[c][x] Jinv[k][x]
          o[3 * c + k] = bad ? nan : s * (Pm[3 * c] * Ji[3 * k] + Pm[3 * c + 1] * Ji[3 * k + 1] + Pm[3 * c + 2] * Ji[3 * k + 2]);
    }
    __syncthreads();

    // R_(a,c) = sum_q sum_k dphi_a/dX_k T_q[c][k]
    for (int w = tid; w < ne * NS; w += NT) {
      const int e = w / NS, a = w - e * NS;
      const T* Te = Ts + (size_t)TW * Q * e;
      T r0 = T(0), r1 = T(0), r2 = T(0);
      for (int qq = 0; qq < Q; ++qq) {
        const T* dp = dphi + (qq * NS + a) * 3;
        const T* t = Te + TW * qq;
        const T d0 = dp[0], d1 = dp[1], d2 = dp[2];
        r0 = fma(t[0], d0, fma(t[1], d1, fma(t[2], d2, r0)));
        r1 = fma(t[3], d0, fma(t[4], d1, fma(t[5], d2, r1)));
        r2 = fma(t[6], d0, fma(t[7], d1, fma(t[8], d2, r2)));
      }
      const int64_t base = (e0 + e) * N + 3 * a;
      put_out<T>(q.out, base, r0, q.out_f32);
      put_out<T>(q.out, base + 1, r1, q.out_f32);
      put_out<T>(q.out, base + 2, r2, q.out_f32);
    }
    __syncthreads();
  }
};

}  // namespace fea
