// Pre-evaluated variant for elasticity, register-blocked (Algorithm 2):
//
//   A_e[3a+c][3b+d] = sum_r R_r[a][b] H_e[r][c][d],   r = (k, al, be), 36 terms
//
// with H_e[(k,al,be)][c][d] = |det J| (mu_k (d_cd M_al,be + Ji_al,d Ji_be,c) + lam_k Ji_al,c Ji_be,d)
// formed once per element from the FP64 geometry.  Each thread owns one test
// function a and up to five trial functions b of one element (45 accumulators):
// per term r it reads the element's 9 geometry entries (three 16-byte shared
// loads, shared by the element's threads) and five R_r[a][b] values (L1), and
// issues 45 FMAs.  Results are staged in shared memory and written with
// coalesced 16-byte stores.
#pragma once
#include "common.cuh"

namespace fea {

template <int P, typename T>
struct PreVecTile {
  static constexpr int FORM = 2;
  static constexpr int NS = nbasis_c(P);
  static constexpr int N = 3 * NS;
  static constexpr int NN = N * N;
  static constexpr int R = 36;
  static constexpr int HB = 12;                 // H entries per term (9 + pad)
  static constexpr int CLEN = 8;
  static constexpr int BB = 5;
  static constexpr int NB = (NS + BB - 1) / BB;
  static constexpr int TPE = NS * NB;
  static constexpr int GEO = 12;

  FEA_HD static int max_tile() { return NT / TPE; }
  FEA_HD static size_t off_c(int TE) { return round_up_sz((size_t)TE * 12 * 8, 16); }
  FEA_HD static size_t off_geo(int TE) { return off_c(TE) + round_up_sz((size_t)TE * CLEN * 8, 16); }
  FEA_HD static size_t off_h(int TE) { return off_geo(TE) + round_up_sz((size_t)TE * GEO * sizeof(T), 16); }
  FEA_HD static size_t off_stage(int TE) { return off_h(TE) + round_up_sz((size_t)TE * R * HB * sizeof(T), 16); }
  FEA_HD static size_t smem(int TE, int Q) { (void)Q; return off_stage(TE) + round_up_sz((size_t)TE * NN * sizeof(T), 16); }

  __device__ static void tile(const Req& q, int64_t e0, int ne, char* sm, unsigned* err) {
    const int TE = q.tile;
    double* xs = reinterpret_cast<double*>(sm);
    double* cs = reinterpret_cast<double*>(sm + off_c(TE));
    T* geo = reinterpret_cast<T*>(sm + off_geo(TE));
    T* H = reinterpret_cast<T*>(sm + off_h(TE));
    T* stage = reinterpret_cast<T*>(sm + off_stage(TE));
    const TabLayout L = tab_layout(q.Q, NS, R);
    const T* Rg = reinterpret_cast<const T*>(q.tab) + L.offR;  // [r][a][b]
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
      const T nan = T(__int_as_float(0x7fc00000));
#pragma unroll
      for (int k = 0; k < 9; ++k) g[k] = from_double<T>(adj[k]);
      const T ad = from_double<T>(fabs(det));
      g[9] = bad ? nan : ad;
      g[10] = bad ? nan : T(1) / ad;
    }
    __syncthreads();
    for (int w = tid; w < ne * R * HB; w += NT) {  // geometry tensors
      const int e = w / (R * HB), h = w - e * (R * HB), rr = h / HB, cd = h - rr * HB;
      T v = T(0);
      if (cd < 9) {
        const T* g = geo + GEO * e;
        const double* c = cs + CLEN * e;
        const int k = rr / 9, al = (rr / 3) % 3, be = rr % 3, cc = cd / 3, d = cd % 3;
        const T M = g[3 * al] * g[3 * be] + g[3 * al + 1] * g[3 * be + 1] + g[3 * al + 2] * g[3 * be + 2];
        const T mu = from_double<T>(c[k]), lam = from_double<T>(c[4 + k]);
        v = (mu * ((cc == d ? M : T(0)) + g[3 * al + d] * g[3 * be + cc]) + lam * g[3 * al + cc] * g[3 * be + d]) * g[10];
      }
      H[w] = v;
    }
    __syncthreads();

    const int te = tid / TPE, r0 = tid - te * TPE;
    const int a = r0 / NB, b0 = (r0 - a * NB) * BB;
    const int nb = NS - b0 < BB ? NS - b0 : BB;
    if (te < ne) {
      T acc[BB][9];
#pragma unroll
      for (int i = 0; i < BB; ++i)
#pragma unroll
        for (int k = 0; k < 9; ++k) acc[i][k] = T(0);
      const T* h = H + (size_t)te * R * HB;
      const T* rp = Rg + (size_t)a * NS + b0;
#pragma unroll 4
      for (int r = 0; r < R; ++r) {
        T hv[12];
        if constexpr (sizeof(T) == 4) {
#pragma unroll
          for (int k = 0; k < 12; k += 4) {
            const float4 x = *reinterpret_cast<const float4*>(h + r * HB + k);
            hv[k] = x.x; hv[k + 1] = x.y; hv[k + 2] = x.z; hv[k + 3] = x.w;
          }
        } else {
#pragma unroll
          for (int k = 0; k < 10; k += 2) {
            const double2 x = *reinterpret_cast<const double2*>(h + r * HB + k);
            hv[k] = x.x; hv[k + 1] = x.y;
          }
        }
        T rv[BB];
#pragma unroll
        for (int i = 0; i < BB; ++i) rv[i] = i < nb ? __ldg(rp + (size_t)r * NS * NS + i) : T(0);
#pragma unroll
        for (int i = 0; i < BB; ++i)
#pragma unroll
          for (int k = 0; k < 9; ++k) acc[i][k] = fma(rv[i], hv[k], acc[i][k]);
      }
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
