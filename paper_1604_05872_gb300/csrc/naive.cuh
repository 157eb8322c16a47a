// Plain quadrature loop nest in normal form, FP64 (the comparator).
//
// Figure "loopnest" with nothing hoisted out of the test/trial nest: every
// (q, i, j) iteration re-evaluates the full integrand of equation
// "quadrature" (Section 2.2) -- the physical gradients J^-T grad Phi of both
// basis functions, the pointwise coefficient kernel, the weight and |det J| --
// as the unoptimised form-compiler output that Figure "poisson" (a) shows.
// Only what the paper computes outside the nest is shared: the element
// geometry (z_0, z_1, ... of Figure "poisson") and coefficient values at the
// point (one FFC-style evaluation per (e, q)).
#pragma once
#include "common.cuh"

namespace fea {

template <int FORM, int P>
struct NaiveTile {
  using T = double;
  static constexpr int NS = nbasis_c(P);
  static constexpr int NC = ncomp_c(FORM);
  static constexpr int N = NC * NS;
  static constexpr int NN = N * N;
  static constexpr int CLEN = coeff_len_c(FORM, P);
  static constexpr int MAXI = 8;
  static constexpr int GEO = 12;  // Jinv[9], |det|
  static constexpr int PT = 12;   // per (e, q): f | mu, lam | Finv[9], lnJ

  FEA_HD static int max_tile() {
    int t = MAXI * NT / NN;
    if (t < 1) t = 1;
    return t > NT ? NT : t;
  }
  static constexpr int MAXI_EFF = NN > MAXI * NT ? (NN + NT - 1) / NT : MAXI;
  FEA_HD static size_t off_c(int TE) { return round_up_sz((size_t)TE * 12 * 8, 16); }
  FEA_HD static size_t off_geo(int TE) { return off_c(TE) + round_up_sz((size_t)TE * CLEN * 8, 16); }
  FEA_HD static size_t off_pt(int TE) { return off_geo(TE) + round_up_sz((size_t)TE * GEO * 8, 16); }
  FEA_HD static size_t smem(int TE, int Q) { (void)Q; return off_pt(TE) + round_up_sz((size_t)TE * PT * 8, 16); }

  __device__ static void tile(const Req& q, int64_t e0, int ne, char* sm, unsigned* err) {
    const int TE = q.tile, Q = q.Q;
    double* xs = reinterpret_cast<double*>(sm);
    double* cs = reinterpret_cast<double*>(sm + off_c(TE));
    double* geo = reinterpret_cast<double*>(sm + off_geo(TE));
    double* pt = reinterpret_cast<double*>(sm + off_pt(TE));
    const TabLayout L = tab_layout(Q, NS, 0);
    const double* tab = reinterpret_cast<const double*>(q.tab);
    const double* Wt = tab + L.offW;
    const double* phi = tab + L.offPhi;
    const double* dphi = tab + L.offDphi;
    const double* phi1 = tab + L.offPhi1;

    load_doubles<NT>(xs, q.coords + e0 * 12, ne * 12);
    if constexpr (CLEN > 0) load_doubles<NT>(cs, q.coeffs + e0 * CLEN, ne * CLEN);
    __syncthreads();
    if ((int)threadIdx.x < ne) {
      double adj[9];
      const double det = geometry_fp64(xs + 12 * threadIdx.x, adj);
      const bool bad = !(fabs(det) > 0.0) || !isfinite(det);
      if (bad) flag_error(err, ERR_DEGENERATE);
      double* g = geo + GEO * threadIdx.x;
      for (int k = 0; k < 9; ++k) g[k] = bad ? __longlong_as_double(0x7ff8000000000000ll) : adj[k] / det;
      g[9] = bad ? __longlong_as_double(0x7ff8000000000000ll) : fabs(det);
    }
    __syncthreads();
    const double mu_c = FORM == 3 ? q.coeffs[q.E * CLEN] : 0.0;
    const double lam_c = FORM == 3 ? q.coeffs[q.E * CLEN + 1] : 0.0;

    const int nitems = ne * NN;
    double acc[MAXI_EFF];
#pragma unroll
    for (int k = 0; k < MAXI_EFF; ++k) acc[k] = 0.0;

    for (int qq = 0; qq < Q; ++qq) {
      for (int e = threadIdx.x; e < ne; e += NT) {  // coefficient values at X_q
        double* o = pt + PT * e;
        const double* Ji = geo + GEO * e;
        if constexpr (FORM == 1) {
          double f = 0.0;
          for (int k = 0; k < NS; ++k) f += cs[CLEN * e + k] * phi[qq * NS + k];
          o[0] = f;
        } else if constexpr (FORM == 2) {
          double mu = 0.0, lam = 0.0;
          for (int k = 0; k < 4; ++k) {
            mu += cs[CLEN * e + k] * phi1[qq * 4 + k];
            lam += cs[CLEN * e + 4 + k] * phi1[qq * 4 + k];
          }
          o[0] = mu;
          o[1] = lam;
        } else if constexpr (FORM == 3) {
          double F[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
          for (int a = 0; a < NS; ++a) {
            const double* dp = dphi + (qq * NS + a) * 3;
            for (int x = 0; x < 3; ++x) {
              const double G = Ji[x] * dp[0] + Ji[3 + x] * dp[1] + Ji[6 + x] * dp[2];
              for (int i = 0; i < 3; ++i) F[3 * i + x] += cs[CLEN * e + 3 * a + i] * G;
            }
          }
          const double c0 = F[4] * F[8] - F[5] * F[7], c3 = F[5] * F[6] - F[3] * F[8], c6 = F[3] * F[7] - F[4] * F[6];
          const double dF = F[0] * c0 + F[1] * c3 + F[2] * c6;
          if (!(dF > 0.0) || !isfinite(dF)) flag_error(err, ERR_DEGENERATE);
          o[0] = c0 / dF;
          o[1] = (F[2] * F[7] - F[1] * F[8]) / dF;
          o[2] = (F[1] * F[5] - F[2] * F[4]) / dF;
          o[3] = c3 / dF;
          o[4] = (F[0] * F[8] - F[2] * F[6]) / dF;
          o[5] = (F[2] * F[3] - F[0] * F[5]) / dF;
          o[6] = c6 / dF;
          o[7] = (F[1] * F[6] - F[0] * F[7]) / dF;
          o[8] = (F[0] * F[4] - F[1] * F[3]) / dF;
          o[9] = log(dF);
        }
      }
      __syncthreads();
      const double w = Wt[qq];
#pragma unroll
      for (int k = 0; k < MAXI_EFF; ++k) {
        const int it = threadIdx.x + k * NT;
        if (it < nitems) {
          const int e = it / NN, ij = it - e * NN, i = ij / N, j = ij - i * N;
          const double* Ji = geo + GEO * e;
          const double* o = pt + PT * e;
          const int a = i / NC, c = i - a * NC, b = j / NC, d = j - b * NC;
          const double* da = dphi + (qq * NS + a) * 3;
          const double* db = dphi + (qq * NS + b) * 3;
          double v;
          if constexpr (FORM == 0) {
            v = phi[qq * NS + a] * phi[qq * NS + b];
          } else {
            double Ga[3], Gb[3];
#pragma unroll
            for (int x = 0; x < 3; ++x) {
              Ga[x] = Ji[x] * da[0] + Ji[3 + x] * da[1] + Ji[6 + x] * da[2];
              Gb[x] = Ji[x] * db[0] + Ji[3 + x] * db[1] + Ji[6 + x] * db[2];
            }
            if constexpr (FORM == 1) {
              v = Ga[0] * Gb[0] + Ga[1] * Gb[1] + Ga[2] * Gb[2] + o[0] * phi[qq * NS + a] * phi[qq * NS + b];
            } else if constexpr (FORM == 2) {
              v = o[0] * ((c == d ? Ga[0] * Gb[0] + Ga[1] * Gb[1] + Ga[2] * Gb[2] : 0.0) + Ga[d] * Gb[c]) +
                  o[1] * Ga[c] * Gb[d];
            } else {
              const double* fi = o;
              const double lnJ = o[9];
              v = 0.0;
#pragma unroll
              for (int I = 0; I < 3; ++I)
#pragma unroll
                for (int J = 0; J < 3; ++J)
                  v += Ga[I] * (mu_c * ((c == d) && (I == J) ? 1.0 : 0.0) + (mu_c - lam_c * lnJ) * fi[3 * J + c] * fi[3 * I + d] +
                                lam_c * fi[3 * I + c] * fi[3 * J + d]) * Gb[J];
            }
          }
          acc[k] += v * w * Ji[9];
        }
      }
      __syncthreads();
    }
    // write (thread per entry: consecutive threads store consecutive entries)
#pragma unroll
    for (int k = 0; k < MAXI_EFF; ++k) {
      const int it = threadIdx.x + k * NT;
      if (it < nitems) {
        if (q.out_f32) reinterpret_cast<float*>(q.out)[e0 * NN + it] = (float)acc[k];
        else reinterpret_cast<double*>(q.out)[e0 * NN + it] = acc[k];
      }
    }
    __syncthreads();
  }
};

}  // namespace fea
