// Helmholtz element matrices in the Bernstein-Bezier basis by sum factorisation
// (the paper names sum factorisation as future work, Section 8; on simplices it
// needs a basis that factors over the collapsed rule, which the Lagrange basis
// does not).
//
// Basis: B_a = p!/a! l^a over |a| = p (l the barycentric coordinates), DOF order
// a3 slowest, then a2, then a1 (a0 = p - a1 - a2 - a3).  With the collapsed
// coordinates of the quadrature rule, X = (t(1-s)(1-r), s(1-r), r), the
// barycentrics are l3 = r, l2 = s(1-r), l1 = t(1-s)(1-r), l0 = (1-t)(1-s)(1-r),
// so every Bernstein polynomial factors into 1-D ones, b^d_k(x) = C(d,k) x^k (1-x)^(d-k):
//
//   B^p_a(X(r,s,t)) = b^p_a3(r) b^(p-a3)_a2(s) b^(p-a3-a2)_a1(t).
//
// Helmholtz A = K + M_f with
//   K_ab = sum_kl Kt_kl Rbar^kl_ab      (|det J| J^-1 J^-T against pre-evaluated
//                                        reference tables, Section 3.3),
//   M_ab = int f B_a B_b = C(a+b, a) / C(2p, p) mu_(a+b),   mu_g = int f B^2p_g,
// since B^p_a B^p_b = C(a+b, a) / C(2p, p) B^2p_(a+b).  The moments of f are where
// sum factorisation applies: f = sum_k c_k B^p_k at the m^3 points in three 1-D
// passes (over t, then s, then r), and mu in three more (over r, s, t), in
// O(p^4) operations instead of the n_s^3 of a pre-evaluated f-mass term.
// The rule (m = ceil((3p+1)/2) points per direction) integrates f B^2p exactly.
//
// One warp per element; a CTA of 8 warps takes tiles of 32 elements, the FP64
// geometry of a tile one element per lane of warp 0.  FP32 arithmetic after the
// geometry; FP64 (exact widening) or FP32 output.
#include <cuda_runtime.h>

#include <array>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/fea.h"
#include "common.cuh"
#include "host_model.h"
#include "launch.cuh"
#include "layout.h"

namespace fea {

int set_error(int code, const char* msg);
struct DevState;
int get_dev_state(DevState** out);
int device_sms(DevState* st);
unsigned* device_error_word(DevState* st);
int check_device_ptr(const void* p, const char* what, bool allow_null);
const void* table_ptr(DevState* st, int form, int p, int prec, int* rc);

constexpr int kBernPrec = 3;  // table key of the Bernstein variant (beside FP64 0, FP32 1, split-BF16 2)

template <int P>
struct BernSF {
  static constexpr int NS = nbasis_c(P);
  static constexpr int M = (3 * P + 2) / 2;  // points per direction: ceil((3p+1)/2)
  static constexpr int Q = M * M * M;
  static constexpr int N2 = 2 * P;                        // degree of the moments
  static constexpr int NM = (N2 + 1) * (N2 + 2) * (N2 + 3) / 6;
  static constexpr int NP1 = (P + 1) * (P + 2) / 2;       // pairs (a3, a2) of degree p
  static constexpr int NP2 = (N2 + 1) * (N2 + 2) / 2;     // pairs (g3, g2) of degree 2p; also rows (d, k) of a 1-D table
  static constexpr int NN = NS * NS;
  static constexpr int NW = 8, TE = 32;                   // warps per CTA, elements per tile
  static constexpr int EW = TE / NW;                      // elements per warp per tile
  // device table, 32-bit words: 1-D tables Tb[3 (r, s, t)][NP2 rows (d, k)][M], W[Q], coef[NN],
  // gidx[NN] (int), Rs[6][NN], pairs of degree p (a3, a2, first DOF) [NP1][3], pairs of degree 2p
  // (g3, g2, first moment) [NP2][3], moments (pair, g1) [NM][2]
  static constexpr int O_TB = 0, O_W = 3 * NP2 * M, O_COEF = O_W + Q, O_GIDX = O_COEF + NN, O_RS = O_GIDX + NN;
  static constexpr int O_P1 = O_RS + 6 * NN, O_P2 = O_P1 + 3 * NP1, O_MUD = O_P2 + 3 * NP2;
  static constexpr int WORDS = round_up(O_MUD + 2 * NM, 4);
  // shared memory: the small tables (words O_TB .. O_COEF and O_P1 .. WORDS); the mass and stiffness
  // tables (O_COEF .. O_P1) are read through L1
  static constexpr int SMALL1 = O_COEF, SMALL2 = WORDS - O_P1, SWORDS = round_up(SMALL1 + SMALL2, 4);
  // per-warp scratch (floats): A = g1 [NP1][M] / h2 [NP2][M]; B = g2 [P+1][M*M] / h1 [N2+1][M*M]; F [Q];
  // mu [EW][NM]; c [NS]
  static constexpr int SA = (NP1 > NP2 ? NP1 : NP2) * M;
  static constexpr int SB = (N2 + 1) * M * M;
  static constexpr int SW = round_up(SA + SB + Q + EW * NM + NS, 4);
  static constexpr size_t SMEM = (size_t)SWORDS * 4 + (size_t)NW * SW * 4 + (size_t)TE * 8 * 4 + 64;
  FEA_HD static constexpr int row1(int d, int k) { return d * (d + 1) / 2 + k; }  // row of b^d_k in a 1-D table
};

// ------------------------------------------------------------------ host tables

static double binom(int n, int k) {
  double r = 1.0;
  for (int i = 1; i <= k; ++i) r = r * (double)(n - k + i) / (double)i;
  return r;
}
static double fact(int n) {
  double r = 1.0;
  for (int i = 2; i <= n; ++i) r *= (double)i;
  return r;
}
// B^d_g(l) = d!/g! l^g for a multi-index g of 4 entries summing to d (0 if any entry is negative)
static double bern(int d, const int g[4], const double l[4]) {
  double v = fact(d);
  for (int i = 0; i < 4; ++i) {
    if (g[i] < 0) return 0.0;
    v /= fact(g[i]);
    for (int k = 0; k < g[i]; ++k) v *= l[i];
  }
  return v;
}
// multi-indices of degree d in the DOF order (a3 slowest, then a2, then a1)
static std::vector<std::array<int, 4>> bern_order(int d) {
  std::vector<std::array<int, 4>> v;
  for (int a3 = 0; a3 <= d; ++a3)
    for (int a2 = 0; a2 <= d - a3; ++a2)
      for (int a1 = 0; a1 <= d - a3 - a2; ++a1) v.push_back({d - a1 - a2 - a3, a1, a2, a3});
  return v;
}

template <int P>
static void bern_table(std::vector<uint32_t>* words) {
  using C = BernSF<P>;
  words->assign(C::WORDS, 0u);
  uint32_t* w = words->data();
  auto putf = [&](int i, double x) {
    const float f = (float)x;
    std::memcpy(&w[i], &f, 4);
  };
  auto puti = [&](int i, int x) { w[i] = (uint32_t)x; };
  const Rule rule = make_rule(C::M);  // points r slowest, t fastest: X = (t(1-s)(1-r), s(1-r), r)
  std::vector<double> r(C::M), sv(C::M), t(C::M);
  for (int i = 0; i < C::M; ++i) r[i] = rule.X[3 * (i * C::M * C::M) + 2];
  for (int j = 0; j < C::M; ++j) sv[j] = rule.X[3 * (j * C::M) + 1] / (1.0 - r[0]);
  for (int k = 0; k < C::M; ++k) t[k] = rule.X[3 * k] / ((1.0 - sv[0]) * (1.0 - r[0]));
  const std::vector<double>* x1[3] = {&r, &sv, &t};
  for (int c = 0; c < 3; ++c)
    for (int d = 0; d <= C::N2; ++d)
      for (int k = 0; k <= d; ++k)
        for (int q = 0; q < C::M; ++q) {
          const double x = (*x1[c])[q];
          putf(C::O_TB + (c * C::NP2 + C::row1(d, k)) * C::M + q, binom(d, k) * std::pow(x, k) * std::pow(1.0 - x, d - k));
        }
  for (int q = 0; q < C::Q; ++q) putf(C::O_W + q, rule.W[q]);
  const auto A = bern_order(P), G = bern_order(C::N2);
  auto gindex = [&](const std::array<int, 4>& g) {
    for (size_t i = 0; i < G.size(); ++i)
      if (G[i] == g) return (int)i;
    return -1;
  };
  // mass: coefficient C(a+b, a) / C(2p, p) of the moment mu_(a+b)
  for (int i = 0; i < C::NS; ++i)
    for (int j = 0; j < C::NS; ++j) {
      std::array<int, 4> g;
      double cf = 1.0 / binom(C::N2, P);
      for (int k = 0; k < 4; ++k) {
        g[k] = A[i][k] + A[j][k];
        cf *= binom(g[k], A[i][k]);
      }
      putf(C::O_COEF + i * C::NS + j, cf);
      puti(C::O_GIDX + i * C::NS + j, gindex(g));
    }
  // stiffness: Rbar^kl_ij = int dB_i/dX_k dB_j/dX_l over the reference tetrahedron (the rule is exact
  // for degree 2p - 2), dB^p_a/dX_k = p (B^(p-1)_(a - e_(k+1)) - B^(p-1)_(a - e_0)); symmetric pairs k <= l
  std::vector<double> Rk(9 * C::NN, 0.0);
  for (int q = 0; q < rule.Q; ++q) {
    const double* X = &rule.X[3 * q];
    const double l[4] = {1.0 - X[0] - X[1] - X[2], X[0], X[1], X[2]};
    std::vector<double> dB(3 * C::NS);
    for (int i = 0; i < C::NS; ++i)
      for (int k = 0; k < 3; ++k) {
        int gk[4] = {A[i][0], A[i][1], A[i][2], A[i][3]}, g0[4] = {A[i][0], A[i][1], A[i][2], A[i][3]};
        gk[k + 1] -= 1;
        g0[0] -= 1;
        dB[3 * i + k] = P * (bern(P - 1, gk, l) - bern(P - 1, g0, l));
      }
    for (int i = 0; i < C::NS; ++i)
      for (int j = 0; j < C::NS; ++j)
        for (int k = 0; k < 3; ++k)
          for (int m = 0; m < 3; ++m) Rk[(3 * k + m) * C::NN + i * C::NS + j] += rule.W[q] * dB[3 * i + k] * dB[3 * j + m];
  }
  int i6 = 0;
  for (int k = 0; k < 3; ++k)
    for (int m = k; m < 3; ++m, ++i6)
      for (int ij = 0; ij < C::NN; ++ij)
        putf(C::O_RS + i6 * C::NN + ij, Rk[(3 * k + m) * C::NN + ij] + (m != k ? Rk[(3 * m + k) * C::NN + ij] : 0.0));
  // pair decodings
  int pi = 0, base = 0;
  for (int a3 = 0; a3 <= P; ++a3)
    for (int a2 = 0; a2 <= P - a3; ++a2, ++pi) {
      puti(C::O_P1 + 3 * pi, a3);
      puti(C::O_P1 + 3 * pi + 1, a2);
      puti(C::O_P1 + 3 * pi + 2, base);
      base += P - a3 - a2 + 1;
    }
  pi = 0;
  base = 0;
  for (int g3 = 0; g3 <= C::N2; ++g3)
    for (int g2 = 0; g2 <= C::N2 - g3; ++g2, ++pi) {
      puti(C::O_P2 + 3 * pi, g3);
      puti(C::O_P2 + 3 * pi + 1, g2);
      puti(C::O_P2 + 3 * pi + 2, base);
      for (int g1 = 0; g1 <= C::N2 - g3 - g2; ++g1) {
        puti(C::O_MUD + 2 * (base + g1), pi);
        puti(C::O_MUD + 2 * (base + g1) + 1, g1);
      }
      base += C::N2 - g3 - g2 + 1;
    }
}


// Device-table words of the Bernstein variant of degree p; false if there is none.
bool bernstein_table_words(int form, int p, std::vector<uint32_t>* words) {
  if (form != HELMHOLTZ) return false;
  switch (p) {
    case 1: bern_table<1>(words); return true;
    case 2: bern_table<2>(words); return true;
    case 3: bern_table<3>(words); return true;
    case 4: bern_table<4>(words); return true;
  }
  return false;
}

// ------------------------------------------------------------------ device

// The moments mu_g = int f B^2p_g of one element by one warp: f at the points
// (three passes), then the moments (three more).  sw: the small tables in
// shared memory (1-D tables and weights, then the pair decodings); adet: |det J|.
template <int P>
__device__ __forceinline__ void bern_sf_moments(const Req& q, int64_t e, float adet, const uint32_t* sw, float* scr,
                                                float* mu, int lane) {
  using C = BernSF<P>;
  constexpr int M = C::M, MM = M * M;
  const float* Tr = reinterpret_cast<const float*>(sw + C::O_TB);
  const float* Ts = Tr + C::NP2 * M;
  const float* Tt = Ts + C::NP2 * M;
  const float* W = reinterpret_cast<const float*>(sw + C::O_W);
  const int* P1 = reinterpret_cast<const int*>(sw + C::SMALL1);
  const int* P2 = P1 + 3 * C::NP1;
  float* gA = scr;          // g1 [NP1][M], then h2 [NP2][M]
  float* gB = gA + C::SA;   // g2 [P+1][M M], then h1 [N2+1][M M]
  float* F = gB + C::SB;    // w |det J| f at the points [Q]
  float* c = F + C::Q + C::EW * C::NM;  // Bernstein coefficients of f [NS]
  for (int i = lane; i < C::NS; i += 32) c[i] = d2f(q.coeffs[e * C::NS + i]);
  __syncwarp();
  // Each pass is a small product: a lane takes one column of its output and keeps
  // the column's entries (one per value of the short index) in registers.
  // f at (r_i, s_j, t_k): over a1 (t), column (a3, a2), entries k
  for (int pr = lane; pr < C::NP1; pr += 32) {
    const int d = P - P1[3 * pr] - P1[3 * pr + 1], base = P1[3 * pr + 2];
    float acc[M];
#pragma unroll
    for (int k = 0; k < M; ++k) acc[k] = 0.f;
#pragma unroll
    for (int a1 = 0; a1 <= P; ++a1)
      if (a1 <= d) {
        const float cv = c[base + a1];
        const float* tr = Tt + C::row1(d, a1) * M;
#pragma unroll
        for (int k = 0; k < M; ++k) acc[k] = fmaf(tr[k], cv, acc[k]);
      }
#pragma unroll
    for (int k = 0; k < M; ++k) gA[pr * M + k] = acc[k];
  }
  __syncwarp();
  // over a2 (s): column (a3, k), entries j
  for (int col = lane; col < (P + 1) * M; col += 32) {
    const int a3 = col / M, k = col - a3 * M, d = P - a3;
    const int pb = a3 * (P + 1) - a3 * (a3 - 1) / 2;  // pairs (a3', a2) with a3' < a3
    float acc[M];
#pragma unroll
    for (int j = 0; j < M; ++j) acc[j] = 0.f;
#pragma unroll
    for (int a2 = 0; a2 <= P; ++a2)
      if (a2 <= d) {
        const float g = gA[(pb + a2) * M + k];
        const float* tr = Ts + C::row1(d, a2) * M;
#pragma unroll
        for (int j = 0; j < M; ++j) acc[j] = fmaf(tr[j], g, acc[j]);
      }
#pragma unroll
    for (int j = 0; j < M; ++j) gB[a3 * MM + j * M + k] = acc[j];
  }
  __syncwarp();
  // over a3 (r): column (j, k), entries i; then w |det J| f
  for (int col = lane; col < MM; col += 32) {
    float acc[M];
#pragma unroll
    for (int i = 0; i < M; ++i) acc[i] = 0.f;
#pragma unroll
    for (int a3 = 0; a3 <= P; ++a3) {
      const float g = gB[a3 * MM + col];
      const float* tr = Tr + C::row1(P, a3) * M;
#pragma unroll
      for (int i = 0; i < M; ++i) acc[i] = fmaf(tr[i], g, acc[i]);
    }
#pragma unroll
    for (int i = 0; i < M; ++i) F[i * MM + col] = W[i * MM + col] * adet * acc[i];
  }
  __syncwarp();
  // moments mu_g = sum_q F_q B^2p_g(X_q): over r, column (j, k), entries g3
  for (int col = lane; col < MM; col += 32) {
    float acc[C::N2 + 1];
#pragma unroll
    for (int g3 = 0; g3 <= C::N2; ++g3) acc[g3] = 0.f;
#pragma unroll
    for (int i = 0; i < M; ++i) {
      const float f = F[i * MM + col];
#pragma unroll
      for (int g3 = 0; g3 <= C::N2; ++g3) acc[g3] = fmaf(Tr[C::row1(C::N2, g3) * M + i], f, acc[g3]);
    }
#pragma unroll
    for (int g3 = 0; g3 <= C::N2; ++g3) gB[g3 * MM + col] = acc[g3];
  }
  __syncwarp();
  // over s: column (g3, k), entries g2 <= 2p - g3
  for (int col = lane; col < (C::N2 + 1) * M; col += 32) {
    const int g3 = col / M, k = col - g3 * M, d = C::N2 - g3;
    const int pb = g3 * (C::N2 + 1) - g3 * (g3 - 1) / 2;  // pairs (g3', g2) with g3' < g3
    float acc[C::N2 + 1];
#pragma unroll
    for (int g2 = 0; g2 <= C::N2; ++g2) acc[g2] = 0.f;
#pragma unroll
    for (int j = 0; j < M; ++j) {
      const float h = gB[g3 * MM + j * M + k];
#pragma unroll
      for (int g2 = 0; g2 <= C::N2; ++g2)
        if (g2 <= d) acc[g2] = fmaf(Ts[C::row1(d, g2) * M + j], h, acc[g2]);
    }
#pragma unroll
    for (int g2 = 0; g2 <= C::N2; ++g2)
      if (g2 <= d) gA[(pb + g2) * M + k] = acc[g2];
  }
  __syncwarp();
  // over t: column (g3, g2), entries g1 <= 2p - g3 - g2
  for (int pr = lane; pr < C::NP2; pr += 32) {
    const int d = C::N2 - P2[3 * pr] - P2[3 * pr + 1], base = P2[3 * pr + 2];
    float acc[C::N2 + 1];
#pragma unroll
    for (int g1 = 0; g1 <= C::N2; ++g1) acc[g1] = 0.f;
#pragma unroll
    for (int k = 0; k < M; ++k) {
      const float h = gA[pr * M + k];
#pragma unroll
      for (int g1 = 0; g1 <= C::N2; ++g1)
        if (g1 <= d) acc[g1] = fmaf(Tt[C::row1(d, g1) * M + k], h, acc[g1]);
    }
#pragma unroll
    for (int g1 = 0; g1 <= C::N2; ++g1)
      if (g1 <= d) mu[base + g1] = acc[g1];
  }
  __syncwarp();
}

// The element matrices of a warp's ne (<= EW) elements e0 + NW k, k < ne:
// A_ab = C(a+b, a) / C(2p, p) mu_(a+b) + sum_kl Kt_kl Rbar^kl_ab, each table
// entry read once (through L1) for all of them.  gm: per element |det J| and
// Kt (geometry rows 8 apart for consecutive elements of the warp).
template <int P>
__device__ __forceinline__ void bern_sf_output(const Req& q, int64_t e0, int ne, const float* gm, const uint32_t* tab,
                                               const float* mu, int lane) {
  using C = BernSF<P>;
  const float* coef = reinterpret_cast<const float*>(tab + C::O_COEF);
  const int* gidx = reinterpret_cast<const int*>(tab + C::O_GIDX);
  const float* Rs = reinterpret_cast<const float*>(tab + C::O_RS);
  float kt[C::EW][6];
#pragma unroll
  for (int k = 0; k < C::EW; ++k)
#pragma unroll
    for (int i = 0; i < 6; ++i) kt[k][i] = k < ne ? gm[8 * C::NW * k + 1 + i] : 0.f;
  for (int o = lane; o < C::NN; o += 32) {
    const float cf = __ldg(coef + o);
    const int g = __ldg(gidx + o);
    float r[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) r[i] = __ldg(Rs + i * C::NN + o);
#pragma unroll
    for (int k = 0; k < C::EW; ++k) {
      if (k < ne) {
        float v = cf * mu[k * C::NM + g];
#pragma unroll
        for (int i = 0; i < 6; ++i) v = fmaf(kt[k][i], r[i], v);
        const int64_t e = e0 + (int64_t)C::NW * k;
        if (q.out_f32)
          __stcs(static_cast<float*>(q.out) + e * C::NN + o, v);
        else
          __stcs(static_cast<double*>(q.out) + e * C::NN + o, f2d(v));
      }
    }
  }
  __syncwarp();
}

template <int P>
__global__ void __launch_bounds__(256) bern_sf_kernel(Req q, unsigned* err) {
  using C = BernSF<P>;
  extern __shared__ __align__(16) char sm[];
  if (C::SMEM > dynamic_smem_bytes()) {
    if (threadIdx.x == 0) flag_error(err, ERR_LAUNCH);
    return;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t* sw = reinterpret_cast<uint32_t*>(sm);  // the small tables
  float* scr = reinterpret_cast<float*>(sm + (size_t)C::SWORDS * 4) + warp * C::SW;
  float* mu = scr + C::SA + C::SB + C::Q;  // [EW][NM]
  float* geo = reinterpret_cast<float*>(sm + (size_t)C::SWORDS * 4 + (size_t)C::NW * C::SW * 4);  // [TE][8]
  const uint32_t* tab = static_cast<const uint32_t*>(q.tab);
  for (int i = threadIdx.x; i < C::SMALL1; i += blockDim.x) sw[i] = __ldg(tab + i);
  for (int i = threadIdx.x; i < C::SMALL2; i += blockDim.x) sw[C::SMALL1 + i] = __ldg(tab + C::O_P1 + i);
  __syncthreads();
  const int64_t ntiles = (q.E + C::TE - 1) / C::TE;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t e0 = t * C::TE;
    const int ne = (int)(q.E - e0 < C::TE ? q.E - e0 : C::TE);
    if (warp == 0 && lane < ne) {  // FP64 geometry, one element per lane
      double adj[9];
      const double det = geometry_fp64(q.coords + (e0 + lane) * 12, adj);
      const uint64_t bits = (uint64_t)__double_as_longlong(det);
      const bool bad = ((bits << 1) == 0) || ((bits >> 52 & 0x7ff) == 0x7ff);
      if (bad) flag_error(err, ERR_DEGENERATE);
      const float ad = fabsf(d2f(det)), inv = 1.0f / ad, nan = __int_as_float(0x7fc00000);
      float a[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) a[k] = d2f(adj[k]);
      float* g = geo + 8 * lane;
      g[0] = bad ? nan : ad;
      int i6 = 1;
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int l = k; l < 3; ++l, ++i6)  // |det J| (J^-1 J^-T)_kl = (adj adj^T)_kl / |det J|
          g[i6] = bad ? nan : (a[3 * k] * a[3 * l] + a[3 * k + 1] * a[3 * l + 1] + a[3 * k + 2] * a[3 * l + 2]) * inv;
    }
    __syncthreads();
    const int nw = warp < ne ? (ne - warp + C::NW - 1) / C::NW : 0;  // elements warp, warp + NW, ... of the tile
    for (int k = 0; k < nw; ++k) bern_sf_moments<P>(q, e0 + warp + C::NW * k, geo[8 * (warp + C::NW * k)], sw, scr, mu + k * C::NM, lane);
    if (nw > 0) bern_sf_output<P>(q, e0 + warp, nw, geo + 8 * warp, tab, mu, lane);
    __syncthreads();
  }
}

template <int P>
static const void* bern_fn() { return reinterpret_cast<const void*>(&bern_sf_kernel<P>); }
template <int P>
static size_t bern_smem() { return BernSF<P>::SMEM; }

int assemble_bernstein_impl(int form, int degree, int64_t E, const double* coords, const double* coeffs, void* out,
                            int out_f32, void* stream) {
  if (form != HELMHOLTZ) return set_error(FEA_EINVAL, "the Bernstein variant covers the Helmholtz form");
  if (degree < 1 || degree > 4) return set_error(FEA_EINVAL, "unsupported degree");
  if (E < 0) return set_error(FEA_EINVAL, "negative element count");
  if (out_f32 != 0 && out_f32 != 1) return set_error(FEA_EINVAL, "out_f32 must be 0 or 1");
  DevState* st = nullptr;
  int rc = get_dev_state(&st);
  if (rc) return rc;
  const void* tab = table_ptr(st, HELMHOLTZ, degree, kBernPrec, &rc);
  if (rc) return rc;
  if (E == 0) return FEA_OK;
  if ((rc = check_device_ptr(coords, "coords", false))) return rc;
  if ((rc = check_device_ptr(coeffs, "coeffs", false))) return rc;
  if ((rc = check_device_ptr(out, "out", false))) return rc;
  const void* fn = degree == 1 ? bern_fn<1>() : degree == 2 ? bern_fn<2>() : degree == 3 ? bern_fn<3>() : bern_fn<4>();
  const size_t smem = degree == 1 ? bern_smem<1>() : degree == 2 ? bern_smem<2>() : degree == 3 ? bern_smem<3>() : bern_smem<4>();
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per_sm = 0;
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 256, smem);
  if (e != cudaSuccess) return set_error(FEA_ECUDA, cudaGetErrorString(e));
  if (per_sm < 1) return set_error(FEA_EINVAL, "kernel cannot be resident");
  Req q;
  std::memset(&q, 0, sizeof(q));
  q.coords = coords;
  q.coeffs = coeffs;
  q.out = out;
  q.tab = tab;
  q.E = E;
  q.form = form;
  q.p = degree;
  q.tile = 32;
  q.out_f32 = out_f32;
  const int64_t ntiles = (E + 31) / 32;
  const unsigned grid = (unsigned)std::min<int64_t>(ntiles, (int64_t)device_sms(st) * per_sm);
  unsigned* err = device_error_word(st);
  void* args[] = {&q, &err};
  e = cudaLaunchKernel(fn, dim3(grid), dim3(256), args, smem, (cudaStream_t)stream);
  if (e != cudaSuccess) return set_error(FEA_ECUDA, cudaGetErrorString(e));
  return FEA_OK;
}

}  // namespace fea

extern "C" int fea_assemble_bernstein(int form, int degree, int64_t E, const double* coords, const double* coeffs,
                                      void* out, int out_f32, void* stream) {
  return fea::assemble_bernstein_impl(form, degree, E, coords, coeffs, out, out_f32, stream);
}
