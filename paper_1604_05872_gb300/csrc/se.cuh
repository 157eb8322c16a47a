// Quadrature variant after sharing elimination (Section 3.2, Algorithm 1;
// Figure "poisson" (b) is the 2-D instance).  The reduction over quadrature
// points stays; what depends only on (e, q) or on (e, q, test index) is
// hoisted out of the test/trial nest and evaluated once:
//
//   G_a(q)  = J^-T grad Phi_a(X_q)              physical gradients (per e, q, a)
//   D_q     = w_q |det J| (pointwise kernel)    per (e, q)
//   L_(a,c) = sum_I G_a^I D_q[c,I][d,J]          left operands (per e, q, a, c)
//   A_e[(a,c)][(b,d)] += sum_J L_(a,c)[d,J] G_b^J   (3 FMA per entry)
//
// Scalar forms use the 4-vectors (G^0, G^1, G^2, Phi):
//   Helmholtz  L_a = s (G_a^0, G_a^1, G_a^2, f_q Phi_a),  A_ab += L_a . (G_b, Phi_b)
//   mass       L_a = s Phi_a,                            A_ab += L_a Phi_b
// Vector forms never form the block-sparse 9 x 3n_p operator: the zero blocks
// (Section 6.3) are skipped by construction.
// Neo-Hookean: F = I + grad u in FP32 sums, then det F, F^-1 and ln det F in
// FP64 for every (element, point) of the tile before the contraction;
//   D[c,I][d,J] = s (mu d_cd d_IJ + (mu - lam ln J) Fi_Jc Fi_Id + lam Fi_Ic Fi_Jd).
#pragma once
#include "common.cuh"
#include "log_f64.cuh"

namespace fea {

template <int FORM, int P, typename T>
struct SeTile {
  static constexpr int NS = nbasis_c(P);
  static constexpr int NC = ncomp_c(FORM);
  static constexpr int N = NC * NS;
  static constexpr int NN = N * N;
  static constexpr int CLEN = coeff_len_c(FORM, P);
  static constexpr int VJ = (NC == 1 && NN % 2 == 0) ? 2 : 1;
  static constexpr int S = NC == 1 ? NN / VJ : NS * NS;
  static constexpr int MAXI = NC == 1 ? 8 : (P == 4 ? 5 : 4);  // items per thread (registers: MAXI * VJ or MAXI * 9)
  static constexpr int LK = NC == 1 ? 4 : 12;    // left-vector stride
  static constexpr int GEO = 12;                 // Jinv[9], |det|, pad

  FEA_HD static int max_tile() {
    int t = MAXI * NT / S;
    return t > NT ? NT : t;
  }
  FEA_HD static size_t off_c(int TE) { return round_up_sz((size_t)TE * 12 * 8, 16); }
  FEA_HD static size_t off_geo(int TE) { return off_c(TE) + round_up_sz((size_t)TE * CLEN * 8, 16); }
  FEA_HD static size_t off_g(int TE) { return off_geo(TE) + round_up_sz((size_t)TE * GEO * sizeof(T), 16); }
  FEA_HD static size_t off_pt(int TE) { return off_g(TE) + round_up_sz((size_t)TE * NS * 4 * sizeof(T), 16); }
  FEA_HD static size_t off_d(int TE) { return off_pt(TE) + round_up_sz((size_t)TE * 4 * sizeof(T), 16); }
  FEA_HD static size_t off_l(int TE) { return off_d(TE) + (NC == 3 ? round_up_sz((size_t)TE * 81 * sizeof(T), 16) : 0); }
  FEA_HD static size_t off_df(int TE) { return off_l(TE) + round_up_sz((size_t)TE * N * LK * sizeof(T), 16); }
  FEA_HD static size_t off_stage(int TE, int Q) {
    return off_df(TE) + (FORM == 3 ? round_up_sz((size_t)TE * Q * 12 * sizeof(T), 16) : 0);
  }
  FEA_HD static size_t smem(int TE, int Q) { return off_stage(TE, Q) + round_up_sz((size_t)TE * NN * sizeof(T), 16); }

  __device__ static void tile(const Req& q, int64_t e0, int ne, char* sm, unsigned* err) {
    const int TE = q.tile, Q = q.Q;
    double* xs = reinterpret_cast<double*>(sm);
    double* cs = reinterpret_cast<double*>(sm + off_c(TE));
    T* geo = reinterpret_cast<T*>(sm + off_geo(TE));
    T* Gq = reinterpret_cast<T*>(sm + off_g(TE));
    T* pt = reinterpret_cast<T*>(sm + off_pt(TE));
    T* D = reinterpret_cast<T*>(sm + off_d(TE));
    T* Lv = reinterpret_cast<T*>(sm + off_l(TE));
    T* DF = reinterpret_cast<T*>(sm + off_df(TE));
    T* stage = reinterpret_cast<T*>(sm + off_stage(TE, Q));
    const TabLayout L = tab_layout(Q, NS, 0);
    const T* tab = reinterpret_cast<const T*>(q.tab);
    const T* Wt = tab + L.offW;
    const T* phi = tab + L.offPhi;
    const T* dphi = tab + L.offDphi;
    const T* phi1 = tab + L.offPhi1;
    const T nan = T(__int_as_float(0x7fc00000));

    load_doubles<NT>(xs, q.coords + e0 * 12, ne * 12);
    if constexpr (CLEN > 0) load_doubles<NT>(cs, q.coeffs + e0 * CLEN, ne * CLEN);
    __syncthreads();
    if ((int)threadIdx.x < ne) {
      double adj[9];
      const double det = geometry_fp64(xs + 12 * threadIdx.x, adj);
      const bool bad = !(fabs(det) > 0.0) || !isfinite(det);
      if (bad) flag_error(err, ERR_DEGENERATE);
      T* g = geo + GEO * threadIdx.x;
      if constexpr (sizeof(T) == 4) {
        const float df = d2f(det), inv = 1.0f / df;
#pragma unroll
        for (int k = 0; k < 9; ++k) g[k] = bad ? nan : d2f(adj[k]) * inv;  // J^-1 = adj / det
        g[9] = bad ? nan : fabsf(df);
      } else {
        const double inv = 1.0 / det;
#pragma unroll
        for (int k = 0; k < 9; ++k) g[k] = bad ? nan : adj[k] * inv;
        g[9] = bad ? nan : fabs(det);
      }
    }
    __syncthreads();

    if constexpr (FORM == 3) {  // Neo-Hookean: F^-1 and ln det F for every (e, q) of the tile
      const int nsub = CLEN;  // u[NS][3]
      for (int w = threadIdx.x; w < ne * Q; w += NT) {
        const int e = w / Q, qq = w - e * Q;
        const T* Ji = geo + GEO * e;
        const double* u = cs + nsub * e;
        T gu[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) gu[k] = T(0);
        for (int a = 0; a < NS; ++a) {
          const T* dp = dphi + (qq * NS + a) * 3;
          T G[3];
#pragma unroll
          for (int x = 0; x < 3; ++x) G[x] = Ji[x] * dp[0] + Ji[3 + x] * dp[1] + Ji[6 + x] * dp[2];
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            const T ui = from_double<T>(u[3 * a + i]);
#pragma unroll
            for (int x = 0; x < 3; ++x) gu[3 * i + x] = fma(ui, G[x], gu[3 * i + x]);
          }
        }
        double F[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) {
          if constexpr (sizeof(T) == 4) F[k] = f2d(gu[k]);
          else F[k] = gu[k];
        }
        F[0] += 1.0; F[4] += 1.0; F[8] += 1.0;
        double cof[9];  // cofactor^T = det(F) F^-1
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
        const double idF = 1.0 / dF;
        T* o = DF + 12 * w;
#pragma unroll
        for (int k = 0; k < 9; ++k) o[k] = bad ? nan : from_double<T>(cof[k] * idF);
        o[9] = bad ? nan : from_double<T>(log_f64(dF));
      }
      __syncthreads();
    }

    const int nitems = ne * S;
    T acc[MAXI][NC == 1 ? VJ : 9];
#pragma unroll
    for (int k = 0; k < MAXI; ++k)
#pragma unroll
      for (int v = 0; v < (NC == 1 ? VJ : 9); ++v) acc[k][v] = T(0);

    const T mu_c = FORM == 3 ? from_double<T>(q.coeffs[q.E * CLEN]) : T(0);
    const T lam_c = FORM == 3 ? from_double<T>(q.coeffs[q.E * CLEN + 1]) : T(0);

    for (int qq = 0; qq < Q; ++qq) {
      // physical gradients and values at X_q
      for (int w = threadIdx.x; w < ne * NS; w += NT) {
        const int e = w / NS, a = w - e * NS;
        const T* Ji = geo + GEO * e;
        const T* dp = dphi + (qq * NS + a) * 3;
        T* o = Gq + 4 * w;
#pragma unroll
        for (int x = 0; x < 3; ++x) o[x] = Ji[x] * dp[0] + Ji[3 + x] * dp[1] + Ji[6 + x] * dp[2];
        o[3] = phi[qq * NS + a];
      }
      // pointwise scalars
      for (int e = threadIdx.x; e < ne; e += NT) {
        const T s = Wt[qq] * geo[GEO * e + 9];
        pt[4 * e] = s;
        if constexpr (FORM == 1) {
          T f = T(0);
          for (int k = 0; k < NS; ++k) f = fma(from_double<T>(cs[CLEN * e + k]), phi[qq * NS + k], f);
          pt[4 * e + 1] = s * f;
        } else if constexpr (FORM == 2) {
          T mu = T(0), lam = T(0);
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            mu = fma(from_double<T>(cs[CLEN * e + k]), phi1[qq * 4 + k], mu);
            lam = fma(from_double<T>(cs[CLEN * e + 4 + k]), phi1[qq * 4 + k], lam);
          }
          pt[4 * e + 1] = s * mu;
          pt[4 * e + 2] = s * lam;
        }
      }
      __syncthreads();
      if constexpr (NC == 3) {  // pointwise tangent D[c,I][d,J]
        for (int w = threadIdx.x; w < ne * 81; w += NT) {
          const int e = w / 81, k = w - e * 81;
          const int c = k / 27, I = (k / 9) % 3, d = (k / 3) % 3, J = k % 3;
          T v;
          if constexpr (FORM == 2) {
            const T smu = pt[4 * e + 1], slam = pt[4 * e + 2];
            v = smu * (T((c == d) && (I == J)) + T((I == d) && (c == J))) + slam * T((c == I) && (d == J));
          } else {
            const T* fi = DF + 12 * (e * Q + qq);
            const T s = pt[4 * e], lnJ = fi[9];
            v = s * (mu_c * T((c == d) && (I == J)) + (mu_c - lam_c * lnJ) * fi[3 * J + c] * fi[3 * I + d] +
                     lam_c * fi[3 * I + c] * fi[3 * J + d]);
          }
          D[w] = v;
        }
        __syncthreads();
      }
      // left operands
      if constexpr (NC == 1) {
        for (int w = threadIdx.x; w < ne * NS; w += NT) {
          const int e = w / NS;
          const T* g = Gq + 4 * w;
          T* o = Lv + LK * w;
          const T s = pt[4 * e];
          if constexpr (FORM == 0) {
            o[0] = s * g[3];
          } else {
            o[0] = s * g[0];
            o[1] = s * g[1];
            o[2] = s * g[2];
            o[3] = pt[4 * e + 1] * g[3];
          }
        }
      } else {
        for (int w = threadIdx.x; w < ne * NS * 9; w += NT) {  // (e, a, c, d): 3 J values
          const int e = w / (NS * 9), rem = w - e * NS * 9, a = rem / 9, cd = rem % 9, c = cd / 3, d = cd % 3;
          const T* g = Gq + 4 * (e * NS + a);
          const T* Dp = D + 81 * e + c * 27 + d * 3;  // D[c,I][d,J] at I = 0
          T* o = Lv + LK * (e * N + 3 * a + c) + 3 * d;
#pragma unroll
          for (int J = 0; J < 3; ++J) o[J] = g[0] * Dp[J] + g[1] * Dp[9 + J] + g[2] * Dp[18 + J];
        }
      }
      __syncthreads();
      // accumulate the owned entries
#pragma unroll
      for (int k = 0; k < MAXI; ++k) {
        const int w = threadIdx.x + k * NT;
        if (w < nitems) {
          const int e = w / S, slot = w - e * S;
          if constexpr (NC == 1) {
#pragma unroll
            for (int v = 0; v < VJ; ++v) {
              const int ij = slot * VJ + v, i = ij / N, j = ij - i * N;
              const T* l = Lv + LK * (e * NS + i);
              const T* b = Gq + 4 * (e * NS + j);
              if constexpr (FORM == 0) acc[k][v] = fma(l[0], b[3], acc[k][v]);
              else acc[k][v] = fma(l[0], b[0], fma(l[1], b[1], fma(l[2], b[2], fma(l[3], b[3], acc[k][v]))));
            }
          } else {
            const int a = slot / NS, bb = slot - a * NS;
            const T* gb = Gq + 4 * (e * NS + bb);
            const T g0 = gb[0], g1 = gb[1], g2 = gb[2];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              const T* l = Lv + LK * (e * N + 3 * a + c);
#pragma unroll
              for (int d = 0; d < 3; ++d)
                acc[k][3 * c + d] = fma(l[3 * d], g0, fma(l[3 * d + 1], g1, fma(l[3 * d + 2], g2, acc[k][3 * c + d])));
            }
          }
        }
      }
      __syncthreads();
    }
    // stage and store
#pragma unroll
    for (int k = 0; k < MAXI; ++k) {
      const int w = threadIdx.x + k * NT;
      if (w < nitems) {
        const int e = w / S, slot = w - e * S;
        if constexpr (NC == 1) {
#pragma unroll
          for (int v = 0; v < VJ; ++v) stage[e * NN + slot * VJ + v] = acc[k][v];
        } else {
          const int a = slot / NS, bb = slot - a * NS;
#pragma unroll
          for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int d = 0; d < 3; ++d) stage[e * NN + (3 * a + c) * N + 3 * bb + d] = acc[k][3 * c + d];
        }
      }
    }
    __syncthreads();
    store_tile<NT, T>(q.out, e0 * NN, stage, ne * NN, q.out_f32);
    __syncthreads();
  }
};

}  // namespace fea
