// Sharing-elimination variant for the vector forms (elasticity, Neo-Hookean),
// register-blocked.  Same arithmetic as SeTile (Section 3.2, Algorithm 1):
//
//   per point q:  G_a = J^-T grad Phi_a(X_q)                        (per e, a)
//                 D[c,I][d,J] = s_q * tangent                        (per e)
//                 L_(a,c)[d,J] = sum_I G_a^I D[c,I][d,J]             (per e, a, c)
//                 A[(a,c)][(b,d)] += sum_J L_(a,c)[d,J] G_b^J        (3 FMA per entry)
//
// Schedule: each thread owns one test function a and a chunk of up to five
// trial functions b of one element, i.e. 5 x 9 accumulators in registers; per
// point it loads L_(a,.) once (27 values) and G_b once per b, so every shared
// load feeds several FMAs.  Pointwise data of all (element, point) pairs of a
// tile (FP64 det F, F^-1, ln det F for Neo-Hookean; s mu_q, s lam_q for
// elasticity) is computed up front by all threads, and the G/D phase of point
// q + 1 runs together with the accumulation of point q (G is double-buffered),
// so each point costs two barriers.
#pragma once
#include "common.cuh"

namespace fea {

template <int FORM, int P, typename T>
struct SeVecTile {
  static_assert(FORM == 2 || FORM == 3, "vector forms");
  static constexpr int NS = nbasis_c(P);
  static constexpr int N = 3 * NS;
  static constexpr int NN = N * N;
  static constexpr int CLEN = coeff_len_c(FORM, P);
  static constexpr int BB = 5;                       // trial functions per thread
  static constexpr int NB = (NS + BB - 1) / BB;      // b-chunks per element
  static constexpr int TPE = NS * NB;                // threads per element
  static constexpr int GEO = 12;                     // Jinv[9], |det|
  static constexpr int PW = 12;                      // pointwise record per (e, q)
  static constexpr int LK = 12;                      // L_(a,c) row: 9 values (d, J) + pad
  static constexpr int DP = 84;                      // D: 81 + pad

  FEA_HD static int max_tile() { return NT / TPE; }
  FEA_HD static size_t off_c(int TE) { return round_up_sz((size_t)TE * 12 * 8, 16); }
  FEA_HD static size_t off_geo(int TE) { return off_c(TE) + round_up_sz((size_t)TE * CLEN * 8, 16); }
  FEA_HD static size_t off_pw(int TE) { return off_geo(TE) + round_up_sz((size_t)TE * GEO * sizeof(T), 16); }
  FEA_HD static size_t off_g(int TE, int Q) { return off_pw(TE) + round_up_sz((size_t)TE * Q * PW * sizeof(T), 16); }
  FEA_HD static size_t off_d(int TE, int Q) { return off_g(TE, Q) + round_up_sz((size_t)2 * TE * NS * 4 * sizeof(T), 16); }
  FEA_HD static size_t off_l(int TE, int Q) { return off_d(TE, Q) + round_up_sz((size_t)TE * DP * sizeof(T), 16); }
  FEA_HD static size_t off_stage(int TE, int Q) { return off_l(TE, Q) + round_up_sz((size_t)TE * NS * 3 * LK * sizeof(T), 16); }
  FEA_HD static size_t smem(int TE, int Q) { return off_stage(TE, Q) + round_up_sz((size_t)TE * NN * sizeof(T), 16); }

  __device__ static void tile(const Req& q, int64_t e0, int ne, char* sm, unsigned* err) {
    const int TE = q.tile, Q = q.Q;
    double* xs = reinterpret_cast<double*>(sm);
    double* cs = reinterpret_cast<double*>(sm + off_c(TE));
    T* geo = reinterpret_cast<T*>(sm + off_geo(TE));
    T* PWs = reinterpret_cast<T*>(sm + off_pw(TE));
    T* Gs = reinterpret_cast<T*>(sm + off_g(TE, Q));       // [2][TE][NS][4]
    T* D = reinterpret_cast<T*>(sm + off_d(TE, Q));        // [TE][DP]
    T* Lv = reinterpret_cast<T*>(sm + off_l(TE, Q));       // [TE][NS][3][LK]
    T* stage = reinterpret_cast<T*>(sm + off_stage(TE, Q));
    const TabLayout L = tab_layout(Q, NS, 0);
    const T* tab = reinterpret_cast<const T*>(q.tab);
    const T* Wt = tab + L.offW;
    const T* dphi = tab + L.offDphi;
    const T* phi1 = tab + L.offPhi1;
    const T nan = T(__int_as_float(0x7fc00000));
    const int tid = threadIdx.x;

    load_doubles<NT>(xs, q.coords + e0 * 12, ne * 12);
    load_doubles<NT>(cs, q.coeffs + e0 * CLEN, ne * CLEN);
    __syncthreads();
    if (tid < ne) {  // FP64 geometry
      double adj[9];
      const double det = geometry_fp64(xs + 12 * tid, adj);
      const bool bad = !(fabs(det) > 0.0) || !isfinite(det);
      if (bad) flag_error(err, ERR_DEGENERATE);
      T* g = geo + GEO * tid;
      if constexpr (sizeof(T) == 4) {
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
    __syncthreads();
    const T mu_c = FORM == 3 ? from_double<T>(q.coeffs[q.E * CLEN]) : T(0);
    const T lam_c = FORM == 3 ? from_double<T>(q.coeffs[q.E * CLEN + 1]) : T(0);

    // pointwise data of every (element, point) of the tile
    for (int w = tid; w < ne * Q; w += NT) {
      const int e = w / Q, qq = w - e * Q;
      const T* Ji = geo + GEO * e;
      T* o = PWs + PW * w;
      const T s = Wt[qq] * Ji[9];
      if constexpr (FORM == 2) {
        T mu = T(0), lam = T(0);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          mu = fma(from_double<T>(cs[CLEN * e + k]), phi1[qq * 4 + k], mu);
          lam = fma(from_double<T>(cs[CLEN * e + 4 + k]), phi1[qq * 4 + k], lam);
        }
        o[0] = s * mu;
        o[1] = s * lam;
        o[11] = s;
      } else {
        const double* u = cs + CLEN * e;
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
        const double idF = 1.0 / dF;
#pragma unroll
        for (int k = 0; k < 9; ++k) o[k] = bad ? nan : from_double<T>(cof[k] * idF);
        o[9] = bad ? nan : from_double<T>(log(dF));
        o[11] = s;
      }
    }
    __syncthreads();

    // phase A of point qq: G into buffer qq & 1, and D
    auto phase_a = [&](int qq) {
      T* Gb = Gs + (size_t)(qq & 1) * TE * NS * 4;
      for (int w = tid; w < ne * NS; w += NT) {
        const int e = w / NS, a = w - e * NS;
        const T* Ji = geo + GEO * e;
        const T* dp = dphi + (qq * NS + a) * 3;
        T* o = Gb + 4 * w;
#pragma unroll
        for (int x = 0; x < 3; ++x) o[x] = Ji[x] * dp[0] + Ji[3 + x] * dp[1] + Ji[6 + x] * dp[2];
        o[3] = T(0);
      }
      for (int w = tid; w < ne * 81; w += NT) {
        const int e = w / 81, k = w - e * 81;
        const int c = k / 27, I = (k / 9) % 3, d = (k / 3) % 3, J = k % 3;
        const T* pw = PWs + PW * (e * Q + qq);
        T v;
        if constexpr (FORM == 2) {
          v = pw[0] * (T((c == d) && (I == J)) + T((I == d) && (c == J))) + pw[1] * T((c == I) && (d == J));
        } else {
          v = pw[11] * (mu_c * T((c == d) && (I == J)) + (mu_c - lam_c * pw[9]) * pw[3 * J + c] * pw[3 * I + d] +
                        lam_c * pw[3 * I + c] * pw[3 * J + d]);
        }
        D[e * DP + k] = v;
      }
    };
    // phase B of point qq: left operands L_(a,c)[d,J]
    auto phase_b = [&](int qq) {
      const T* Gb = Gs + (size_t)(qq & 1) * TE * NS * 4;
      for (int w = tid; w < ne * NS * 9; w += NT) {
        const int e = w / (NS * 9), rem = w - e * NS * 9, a = rem / 9, cd = rem % 9, c = cd / 3, d = cd % 3;
        const T* g = Gb + 4 * (e * NS + a);
        const T* Dp = D + e * DP + c * 27 + d * 3;
        T* o = Lv + (size_t)((e * NS + a) * 3 + c) * LK + 3 * d;
        const T g0 = g[0], g1 = g[1], g2 = g[2];
#pragma unroll
        for (int J = 0; J < 3; ++J) o[J] = g0 * Dp[J] + g1 * Dp[9 + J] + g2 * Dp[18 + J];
      }
    };

    // this thread's block: element e, test function a, trial functions b0 .. b0 + nb - 1
    const int te = tid / TPE, r = tid - te * TPE;
    const int a = r / NB, b0 = (r - a * NB) * BB;
    const int nb = NS - b0 < BB ? NS - b0 : BB;
    const bool owner = te < ne;
    T acc[BB][9];
#pragma unroll
    for (int i = 0; i < BB; ++i)
#pragma unroll
      for (int k = 0; k < 9; ++k) acc[i][k] = T(0);

    phase_a(0);
    __syncthreads();
    phase_b(0);
    __syncthreads();
    for (int qq = 0; qq < Q; ++qq) {
      if (owner) {
        const T* Gb = Gs + (size_t)(qq & 1) * TE * NS * 4 + (size_t)(te * NS + b0) * 4;
        const T* lv = Lv + (size_t)(te * NS + a) * 3 * LK;
        T l[27];
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int k = 0; k < 9; ++k) l[9 * c + k] = lv[c * LK + k];
#pragma unroll
        for (int i = 0; i < BB; ++i) {
          if (i < nb) {
            const T g0 = Gb[4 * i], g1 = Gb[4 * i + 1], g2 = Gb[4 * i + 2];
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
              for (int d = 0; d < 3; ++d)
                acc[i][3 * c + d] =
                    fma(l[9 * c + 3 * d], g0, fma(l[9 * c + 3 * d + 1], g1, fma(l[9 * c + 3 * d + 2], g2, acc[i][3 * c + d])));
          }
        }
      }
      if (qq + 1 < Q) phase_a(qq + 1);  // other G buffer; D was consumed by phase_b(qq)
      __syncthreads();
      if (qq + 1 < Q) {
        phase_b(qq + 1);  // Lv of point qq was consumed by the accumulation above
        __syncthreads();
      }
    }
    if (owner) {
      T* o = stage + (size_t)te * NN + (3 * a) * N + 3 * b0;
#pragma unroll
      for (int i = 0; i < BB; ++i)
        if (i < nb)
#pragma unroll
          for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int d = 0; d < 3; ++d) o[c * N + 3 * i + d] = acc[i][3 * c + d];
    }
    __syncthreads();
    store_tile<NT, T>(q.out, e0 * NN, stage, ne * NN, q.out_f32);
    __syncthreads();
  }
};

}  // namespace fea
