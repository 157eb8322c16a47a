// Pre-evaluated variant (Section 3.3, Algorithm 2; Figure "loopnest-opt", the
// loop nest for pre-evaluated monomials).  The reduction over quadrature
// points is summed once on the host into reference tensors R_r (the library's
// tables); per element only the geometry tensor H_e is formed and contracted:
//
//   scalar forms   A_e[i][j]             = sum_r R_r[i][j]  H_e[r]
//   vector forms   A_e[3a+c][3b+d]       = sum_r R_r[a][b]  H_e[r][c][d]
//
//   mass        r = 1        H = |det J|
//   Helmholtz   r = 6 + n_p  H = (K_00, K_11, K_22, K_01, K_02, K_12, |det J| f_k)
//               with K = |det J| J^-1 J^-T  (the tensor-contraction geometry of Section 2.3)
//   elasticity  r = 4*3*3    H_(k,al,be)[c][d] = |det J| (mu_k (d_cd M_al,be + Ji_al,d Ji_be,c)
//                                                         + lam_k Ji_al,c Ji_be,d),  M = Ji Ji^T
//
// One CTA processes a tile of elements; each thread owns fixed output slots,
// keeps its column of R in registers and sweeps the tile's elements, reading
// H_e with broadcast 16-byte shared loads.  Results are staged in shared
// memory and written with coalesced 16-byte stores.
#pragma once
#include "common.cuh"

namespace fea {

template <int FORM, int P, typename T>
struct PreTile {
  static constexpr int NS = nbasis_c(P);
  static constexpr int NC = ncomp_c(FORM);
  static constexpr int N = NC * NS;
  static constexpr int NN = N * N;
  static constexpr int R = pre_terms_c(FORM, P);
  static constexpr int HV = 16 / (int)sizeof(T);                   // T per 16-byte load
  static constexpr int HB = NC == 1 ? 1 : round_up(NC * NC, HV);   // H entries per r (padded)
  static constexpr int NHE = R * HB;
  static constexpr int NHP = round_up(NHE, HV);
  static constexpr int CLEN = coeff_len_c(FORM, P);
  static constexpr int VJ = (NC == 1 && NN % 2 == 0) ? 2 : 1;     // outputs per slot (scalar)
  static constexpr int S = NC == 1 ? NN / VJ : NS * NS;            // slots per element
  static constexpr int G = S >= NT ? 1 : NT / S;                   // element groups
  static constexpr int GEO = 12;                                   // adj[9], |det|, 1/|det|, pad
  static constexpr int MINB = sizeof(T) == 4 && P == 4 ? 3 : 1;     // resident CTAs per SM

  FEA_HD static size_t off_c(int TE) { return round_up_sz((size_t)TE * 12 * 8, 16); }
  FEA_HD static size_t off_geo(int TE) { return off_c(TE) + round_up_sz((size_t)TE * CLEN * 8, 16); }
  FEA_HD static size_t off_h(int TE) { return off_geo(TE) + round_up_sz((size_t)TE * GEO * sizeof(T), 16); }
  FEA_HD static size_t off_stage(int TE) { return off_h(TE) + round_up_sz((size_t)TE * NHP * sizeof(T), 16); }
  FEA_HD static size_t smem(int TE) { return off_stage(TE) + round_up_sz((size_t)TE * NN * sizeof(T), 16); }
  FEA_HD static size_t smem(int TE, int Q) { (void)Q; return smem(TE); }
  FEA_HD static int max_tile() { return NT; }

  // One entry of the geometry tensor.
  __device__ static __forceinline__ T h_entry(int h, const T* g, const double* c) {
    if constexpr (FORM == 0) {
      return g[9];
    } else if constexpr (FORM == 1) {
      if (h < 6) {
        const int al = h < 3 ? h : (h == 5 ? 1 : 0);
        const int be = h < 3 ? h : (h == 3 ? 1 : 2);
        const T k = g[3 * al] * g[3 * be] + g[3 * al + 1] * g[3 * be + 1] + g[3 * al + 2] * g[3 * be + 2];
        return k * g[10];
      }
      return g[9] * from_double<T>(c[h - 6]);
    } else {
      const int rr = h / HB, cd = h - rr * HB;
      if (cd >= 9) return T(0);
      const int k = rr / 9, al = (rr / 3) % 3, be = rr % 3, cc = cd / 3, d = cd % 3;
      const T M = g[3 * al] * g[3 * be] + g[3 * al + 1] * g[3 * be + 1] + g[3 * al + 2] * g[3 * be + 2];
      const T mu = from_double<T>(c[k]), lam = from_double<T>(c[4 + k]);
      T v = mu * ((cc == d ? M : T(0)) + g[3 * al + d] * g[3 * be + cc]) + lam * g[3 * al + cc] * g[3 * be + d];
      return v * g[10];
    }
  }

  template <int K>
  __device__ static __forceinline__ void ld(const T* p, T (&v)[K]) {
    static_assert(K % HV == 0, "vector load");
#pragma unroll
    for (int k = 0; k < K; k += HV) {
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
    const int TE = q.tile;
    double* xs = reinterpret_cast<double*>(sm);
    double* cs = reinterpret_cast<double*>(sm + off_c(TE));
    T* geo = reinterpret_cast<T*>(sm + off_geo(TE));
    T* H = reinterpret_cast<T*>(sm + off_h(TE));
    T* stage = reinterpret_cast<T*>(sm + off_stage(TE));
    const TabLayout L = tab_layout(q.Q, NS, R);
    const T* Rg = reinterpret_cast<const T*>(q.tab) + L.offR;

    load_doubles<NT>(xs, q.coords + e0 * 12, ne * 12);
    if constexpr (CLEN > 0) load_doubles<NT>(cs, q.coeffs + e0 * CLEN, ne * CLEN);
    __syncthreads();
    if ((int)threadIdx.x < ne) {  // FP64 geometry, one thread per element
      double adj[9];
      const double det = geometry_fp64(xs + 12 * threadIdx.x, adj);
      const bool bad = !(fabs(det) > 0.0) || !isfinite(det);
      if (bad) flag_error(err, ERR_DEGENERATE);
      T* g = geo + GEO * threadIdx.x;
#pragma unroll
      for (int k = 0; k < 9; ++k) g[k] = from_double<T>(adj[k]);
      const T ad = from_double<T>(fabs(det));
      const T nan = T(__int_as_float(0x7fc00000));
      g[9] = bad ? nan : ad;
      g[10] = bad ? nan : T(1) / ad;
    }
    __syncthreads();
    for (int w = threadIdx.x; w < ne * NHP; w += NT) {  // geometry tensors
      const int e = w / NHP, h = w - e * NHP;
      H[w] = h < NHE ? h_entry(h, geo + GEO * e, cs + CLEN * e) : T(0);
    }
    __syncthreads();

    if constexpr (NC == 1) {
      const int t = threadIdx.x;
      if (S >= NT || t < G * S) {
        const int g0 = S >= NT ? 0 : t / S;
        for (int slot = S >= NT ? t : t % S; slot < S; slot += (S >= NT ? NT : S)) {
          T rr[VJ][R];
#pragma unroll
          for (int v = 0; v < VJ; ++v)
#pragma unroll
            for (int r = 0; r < R; ++r) rr[v][r] = __ldg(Rg + (size_t)r * NN + slot * VJ + v);
          for (int e = g0; e < ne; e += G) {
            const T* h = H + e * NHP;
            T acc[VJ];
#pragma unroll
            for (int v = 0; v < VJ; ++v) acc[v] = T(0);
#pragma unroll
            for (int r0 = 0; r0 < NHP; r0 += HV) {
              T hv[HV];
              ld<HV>(h + r0, hv);
#pragma unroll
              for (int k = 0; k < HV; ++k)
                if (r0 + k < R)
#pragma unroll
                  for (int v = 0; v < VJ; ++v) acc[v] = fma(rr[v][r0 + k], hv[k], acc[v]);
            }
            T* o = stage + e * NN + slot * VJ;
            if constexpr (VJ == 2 && sizeof(T) == 4) {
              *reinterpret_cast<float2*>(o) = make_float2(acc[0], acc[1]);
            } else {
#pragma unroll
              for (int v = 0; v < VJ; ++v) o[v] = acc[v];
            }
          }
        }
      }
    } else {
      for (int slot = threadIdx.x; slot < S; slot += NT) {  // slot = (a, b)
        const int a = slot / NS, b = slot - a * NS;
        T rr[R];
#pragma unroll
        for (int r = 0; r < R; ++r) rr[r] = __ldg(Rg + (size_t)r * NS * NS + slot);
        for (int e = 0; e < ne; ++e) {
          const T* h = H + e * NHP;
          T acc[9];
#pragma unroll
          for (int k = 0; k < 9; ++k) acc[k] = T(0);
#pragma unroll
          for (int r = 0; r < R; ++r) {
            T hv[HB];
            ld<HB>(h + r * HB, hv);
#pragma unroll
            for (int k = 0; k < 9; ++k) acc[k] = fma(rr[r], hv[k], acc[k]);
          }
          T* o = stage + e * NN + (3 * a) * N + 3 * b;
#pragma unroll
          for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int d = 0; d < 3; ++d) o[c * N + d] = acc[3 * c + d];
        }
      }
    }
    __syncthreads();
    store_tile<NT, T>(q.out, e0 * NN, stage, ne * NN, q.out_f32);
    __syncthreads();
  }
};

}  // namespace fea
