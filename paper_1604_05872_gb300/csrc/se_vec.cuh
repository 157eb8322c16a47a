// Sharing-elimination variant for the vector forms (elasticity, Neo-Hookean).
//
// Both tangents have the structure
//   A[c,I][d,J] = mu d_cd d_IJ + alpha Fi_Jc Fi_Id + lam Fi_Ic Fi_Jd
// (Neo-Hookean: Fi = F^-1, alpha = mu - lam ln det F, mu and lam constants;
// elasticity: Fi = I, alpha = mu, with mu, lam the P1 fields at the point).
// Factorising the test/trial contraction through it (Section 3.2: expansion,
// factorisation and code motion of what depends on (e, q) or (e, q, a) only):
//
//   G_a = J^-T grad Phi_a(X_q),   Y_a = Fi^T G_a                      (per e, q, a)
//   A_e[(a,c)][(b,d)] += s_q ( mu d_cd (G_a . G_b) + alpha Y_a[d] Y_b[c] + lam Y_a[c] Y_b[d] )
//
// 24 FMA per (a, b) block of nine entries and point, and no per-point tangent
// or left-operand tables.  Each thread owns one test function a and up to five
// trial functions b of one element (45 accumulators); per point it reads
// (G_a, Y_a) once and (G_b, Y_b) per b, two 16-byte shared loads each.  The
// FP64 work (Neo-Hookean det F, F^-1 and ln det F) for every (element, point)
// of a tile is done up front by all threads; the (G, Y) rows of point q + 1 are
// formed while point q accumulates (double buffer): one barrier per point.
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
  static constexpr int PW = 12;                      // per (e, q): Fi[9] (Neo-Hookean), s mu, s alpha, s lam
  static constexpr int GY = 8;                       // per (e, a): G[3], pad, Y[3], pad

  FEA_HD static int max_tile() { return NT / TPE; }
  FEA_HD static size_t off_c(int TE) { return round_up_sz((size_t)TE * 12 * 8, 16); }
  FEA_HD static size_t off_geo(int TE) { return off_c(TE) + round_up_sz((size_t)TE * CLEN * 8, 16); }
  FEA_HD static size_t off_pw(int TE) { return off_geo(TE) + round_up_sz((size_t)TE * GEO * sizeof(T), 16); }
  FEA_HD static size_t off_gy(int TE, int Q) { return off_pw(TE) + round_up_sz((size_t)TE * Q * PW * sizeof(T), 16); }
  FEA_HD static size_t off_stage(int TE, int Q) { return off_gy(TE, Q) + round_up_sz((size_t)2 * TE * NS * GY * sizeof(T), 16); }
  FEA_HD static size_t smem(int TE, int Q) { return off_stage(TE, Q) + round_up_sz((size_t)TE * NN * sizeof(T), 16); }

  template <int K>
  __device__ static __forceinline__ void ld(const T* p, T (&v)[K]) {
#pragma unroll
    for (int k = 0; k < K; k += 16 / (int)sizeof(T)) {
      if constexpr (sizeof(T) == 4) {
        const float4 x = *reinterpret_cast<const float4*>(p + k);
        v[k] = x.x; v[k + 1] = x.y; v[k + 2] = x.z; v[k + 3] = x.w;
      } else {
        const double2 x = *reinterpret_cast<const double2*>(p + k);
        v[k] = x.x; v[k + 1] = x.y;
      }
    }
  }

  __device__ static void tile(const Req& q, int64_t e0, int ne, char* sm, unsigned* err) {
    const int TE = q.tile, Q = q.Q;
    double* xs = reinterpret_cast<double*>(sm);
    double* cs = reinterpret_cast<double*>(sm + off_c(TE));
    T* geo = reinterpret_cast<T*>(sm + off_geo(TE));
    T* PWs = reinterpret_cast<T*>(sm + off_pw(TE));
    T* GYs = reinterpret_cast<T*>(sm + off_gy(TE, Q));      // [2][TE][NS][GY]
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
        o[9] = s * mu;
        o[10] = s * mu;
        o[11] = s * lam;
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
        for (int k = 0; k < 9; ++k) o[k] = bad ? nan : from_double<T>(cof[k] * idF);  // o[3 i + j] = Fi[i][j]
        const T lnJ = bad ? nan : from_double<T>(log(dF));
        o[9] = s * mu_c;
        o[10] = s * (mu_c - lam_c * lnJ);
        o[11] = s * lam_c;
      }
    }
    __syncthreads();

    // (G_a, Y_a) of point qq for every (element, a) into buffer qq & 1
    auto rows = [&](int qq) {
      T* Gb = GYs + (size_t)(qq & 1) * TE * NS * GY;
      for (int w = tid; w < ne * NS; w += NT) {
        const int e = w / NS, a = w - e * NS;
        const T* Ji = geo + GEO * e;
        const T* dp = dphi + (qq * NS + a) * 3;
        T G[3];
#pragma unroll
        for (int x = 0; x < 3; ++x) G[x] = Ji[x] * dp[0] + Ji[3 + x] * dp[1] + Ji[6 + x] * dp[2];
        T* o = Gb + GY * w;
        o[0] = G[0]; o[1] = G[1]; o[2] = G[2]; o[3] = T(0);
        if constexpr (FORM == 3) {
          const T* fi = PWs + PW * (e * Q + qq);
#pragma unroll
          for (int x = 0; x < 3; ++x) o[4 + x] = G[0] * fi[x] + G[1] * fi[3 + x] + G[2] * fi[6 + x];
        } else {
          o[4] = G[0]; o[5] = G[1]; o[6] = G[2];
        }
        o[7] = T(0);
      }
    };

    const int te = tid / TPE, r = tid - te * TPE;
    const int a = r / NB, b0 = (r - a * NB) * BB;
    const int nb = NS - b0 < BB ? NS - b0 : BB;
    const bool owner = te < ne;
    T acc[BB][9];
#pragma unroll
    for (int i = 0; i < BB; ++i)
#pragma unroll
      for (int k = 0; k < 9; ++k) acc[i][k] = T(0);

    rows(0);
    __syncthreads();
    for (int qq = 0; qq < Q; ++qq) {
      if (owner) {
        const T* Gb = GYs + (size_t)(qq & 1) * TE * NS * GY + (size_t)te * NS * GY;
        const T* pw = PWs + PW * (te * Q + qq);
        const T smu = pw[9], sal = pw[10], slam = pw[11];
        T ga[8];
        ld<8>(Gb + GY * a, ga);
        // scaled test rows: alpha Y_a and lam Y_a
        const T ay0 = sal * ga[4], ay1 = sal * ga[5], ay2 = sal * ga[6];
        const T ly0 = slam * ga[4], ly1 = slam * ga[5], ly2 = slam * ga[6];
        const T ay[3] = {ay0, ay1, ay2}, ly[3] = {ly0, ly1, ly2};
#pragma unroll
        for (int i = 0; i < BB; ++i) {
          if (i < nb) {
            T gb[8];
            ld<8>(Gb + GY * (b0 + i), gb);
            const T dot = smu * (ga[0] * gb[0] + ga[1] * gb[1] + ga[2] * gb[2]);
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
              for (int d = 0; d < 3; ++d)
                acc[i][3 * c + d] = fma(ay[d], gb[4 + c], fma(ly[c], gb[4 + d], acc[i][3 * c + d] + (c == d ? dot : T(0))));
          }
        }
      }
      if (qq + 1 < Q) rows(qq + 1);  // the other buffer, last read at point qq - 1
      __syncthreads();
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
