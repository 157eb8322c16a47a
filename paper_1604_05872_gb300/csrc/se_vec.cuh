// Sharing-elimination variant for the vector forms (elasticity, Neo-Hookean).
//
// Both tangents have the structure
//   A[(a,c)][(b,d)] = sum_q s_q ( mu d_cd G_a.G_b + alpha Y_a[d] Y_b[c] + lam Y_a[c] Y_b[d] )
// with G_a = J^-T grad Phi_a(X_q) and
//   elasticity:   Y = G,           alpha = mu,  mu and lam the P1 fields at the point;
//   Neo-Hookean:  Y = F^-T G,      alpha = mu - lam ln det F, mu and lam constants.
// Factorising the test/trial contraction through this structure (Section 3.2:
// expansion, factorisation and code motion of what depends on (e, q) or
// (e, q, a) only) leaves, per block (a, b), three accumulations over the points:
//
//   W1 = sum_q s alpha Y_a (x) Y_b,   W2 = sum_q s lam Y_a (x) Y_b,   D = sum_q s mu G_a.G_b
//   A[(a,.)][(b,.)] = D I + W1^T + W2
//
// For elasticity D = tr W1.  For Neo-Hookean D = Z_a . Y_b with Z_a = s mu F G_a
// (since G_b = F^T Y_b).  The tangents are symmetric, so only blocks a <= b are
// accumulated (runs of up to BB trial functions per thread, see sym.cuh) and
// each is written as itself and transposed.
//
// Per block and point: one 16-byte shared load of Y_b = (Y0, Y1, Y2, Y2) and
// ten (elasticity) or twelve (Neo-Hookean) packed/scalar FMAs; the a-side
// factors (s alpha Y_a, s lam Y_a, Z_a) sit in registers for the whole run.
//
// Thread layout: EF consecutive lanes take EF elements of the tile with the same
// run, so a warp holds 32 / EF runs of (nearly) equal length and reads the rows
// of EF elements at once (element rows are an odd number of 16-byte slots
// apart: conflict-free).  Pointwise data are computed for every (element,
// point) up front; for Neo-Hookean, F = I + grad u is widened to FP64 and
// det F, F^-1 and ln det F are evaluated in FP64 (FP32 path included).  The
// (Y, Z) rows of the next QG points are formed while the current QG points
// accumulate (double buffer, one barrier per QG points; the point count is
// padded to a multiple of QG with zero-weight points so that the point loop
// unrolls).  The staged element matrices reuse the pointwise and row buffers,
// which are dead once the last point group has been accumulated.
#pragma once
#include "common.cuh"
#include "log_f64.cuh"
#include "sym.cuh"

namespace fea {

// Four T to 16-byte aligned shared memory.
template <typename T>
__device__ __forceinline__ void st4(T* p, T x, T y, T z, T w) {
  if constexpr (sizeof(T) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(x, y, z, w);
  } else {
    *reinterpret_cast<double2*>(p) = make_double2(x, y);
    *reinterpret_cast<double2*>(p + 2) = make_double2(z, w);
  }
}

// floor(w / d) without an integer division: truncate (w + 1/2) * fl(1/d) in
// FP32 (correctly rounded reciprocal and product).  Exact for 0 <= w < 16384
// and 1 <= d < 8192, checked exhaustively; the tile loops stay far inside.
__device__ __forceinline__ int small_div(int w, float inv_d) { return (int)(((float)w + 0.5f) * inv_d); }

template <int FORM, int P, typename T>
struct SeVecTile {
  static_assert(FORM == 2 || FORM == 3, "vector forms");
  static constexpr bool NEO = FORM == 3;
  static constexpr bool F32 = sizeof(T) == 4;
  static constexpr int NS = nbasis_c(P);
  static constexpr int N = 3 * NS;
  static constexpr int NN = N * N;
  static constexpr int CLEN = coeff_len_c(FORM, P);
  // trial functions per thread, elements interleaved per warp, resident CTAs per SM
  static constexpr int BB = P == 4 ? 3 : 2;
  static constexpr int EF = P <= 2 ? 8 : P == 3 ? 2 : 1;
  static constexpr int MINB = F32 ? (P <= 3 ? 3 : 2) : 1;
  using Chunks = SymChunks<NS, BB>;
  static constexpr int NCH = Chunks::NCH;
  static constexpr int GROUPS = NT / (EF * NCH);
  static_assert(GROUPS >= 1, "one element group must fit the CTA");
  static constexpr int TEMAX = EF * GROUPS;
  static constexpr int NSP = NS | 1;                 // row slots per element (odd)
  // points per barrier (measured best per degree; Neo-Hookean P2 and P4: their 27 and 125 points in
  // groups of nine and 25, without padding)
  static constexpr int QG = NEO && P == 2 ? 9 : NEO && P == 4 ? 25 : P >= 3 ? 16 : 4;
  static constexpr int GEO = 12;                     // Jinv[9], |det|, pad
  static constexpr int PW = NEO ? 20 : 4;            // per (e, q): [Fi[9], s mu F[9],] s alpha, s lam
  static constexpr int RW = NEO ? 2 : 1;             // 16-byte rows per (e, a): Y [, Z]
  using V2 = typename Vec2Of<T>::type;

  FEA_HD static int max_tile() { return TEMAX; }
  FEA_HD static int pref_tile() { return TEMAX; }
  FEA_HD static int qpad(int Q) { return (Q + QG - 1) / QG * QG; }
  FEA_HD static size_t off_c(int TE) { return round_up_sz((size_t)TE * 12 * 8, 16); }
  FEA_HD static size_t off_ct(int TE) { return off_c(TE) + round_up_sz((size_t)TE * CLEN * 8, 16); }
  FEA_HD static size_t off_geo(int TE) { return off_ct(TE) + round_up_sz((size_t)TE * CLEN * sizeof(T), 16); }
  FEA_HD static size_t off_pw(int TE) { return off_geo(TE) + round_up_sz((size_t)TE * GEO * sizeof(T), 16); }
  FEA_HD static size_t off_rows(int TE, int Q) { return off_pw(TE) + round_up_sz((size_t)TE * qpad(Q) * PW * sizeof(T), 16); }
  FEA_HD static size_t rows_len(int TE) { return (size_t)QG * TE * NSP * 4; }  // T per buffer and row kind
  FEA_HD static size_t off_stage(int TE) { return off_pw(TE); }                  // aliases pointwise data and rows
  FEA_HD static size_t smem(int TE, int Q) {
    const size_t a = off_stage(TE) + round_up_sz((size_t)TE * NN * sizeof(T), 16);
    const size_t b = off_rows(TE, Q) + (size_t)2 * RW * rows_len(TE) * sizeof(T);
    return a > b ? a : b;
  }

  // The tile the thread layout is built for (TEMAX) runs with the tile size and
  // the point count as compile-time constants (shared-memory offsets and row
  // strides fold into immediates); other tiles take the same code with runtime
  // sizes.
  __device__ static void tile(const Req& q, int64_t e0, int ne, char* sm, unsigned* err) {
    if (q.tile == TEMAX) tile_t<TEMAX>(q, e0, ne, sm, err);
    else tile_t<0>(q, e0, ne, sm, err);
  }

  template <int TEC>
  __device__ static void tile_t(const Req& q, int64_t e0, int ne, char* sm, unsigned* err) {
    const int TE = TEC ? TEC : q.tile, Q = q.Q;
    double* xs = reinterpret_cast<double*>(sm);
    double* cs = reinterpret_cast<double*>(sm + off_c(TE));
    T* ct = reinterpret_cast<T*>(sm + off_ct(TE));
    T* geo = reinterpret_cast<T*>(sm + off_geo(TE));
    T* PWs = reinterpret_cast<T*>(sm + off_pw(TE));
    T* rows = reinterpret_cast<T*>(sm + off_rows(TE, Q));   // [2][RW][QG][TE][NSP][4]
    T* stage = reinterpret_cast<T*>(sm + off_stage(TE));
    const size_t RL = rows_len(TE);
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
      if constexpr (F32) {
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
    const T mu_c = NEO ? from_double<T>(q.coeffs[q.E * CLEN]) : T(0);
    const T lam_c = NEO ? from_double<T>(q.coeffs[q.E * CLEN + 1]) : T(0);

    // pointwise data of every (element, point) of the tile; padded points get zero weight
    const int QP = qpad(Q);
    const float inv_qp = 1.0f / (float)QP;
    for (int w = tid; w < ne * QP; w += NT) {
      const int e = small_div(w, inv_qp), qq = w - e * QP;
      T* o = PWs + PW * w;
      if (qq >= Q) {
#pragma unroll
        for (int k = 0; k < PW; ++k) o[k] = T(0);
        continue;
      }
      const T* Ji = geo + GEO * e;
      const T s = Wt[qq] * Ji[9];
      if constexpr (!NEO) {
        T mu = T(0), lam = T(0);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          mu = fma(ct[CLEN * e + k], phi1[qq * 4 + k], mu);
          lam = fma(ct[CLEN * e + 4 + k], phi1[qq * 4 + k], lam);
        }
        o[PW - 2] = s * mu;   // alpha = mu
        o[PW - 1] = s * lam;
      } else {
        // grad u = (sum_a u_a (x) grad_X Phi_a) J^-1 in the tile precision
        const T* u = ct + CLEN * e;
        T gr[9];
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
        // F = I + grad u, det F, F^-1 and ln det F in FP64
        double F[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) {
          if constexpr (F32) F[k] = f2d(gu[k]);
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
        // the cancellation-prone cofactors and det F are FP64; the division by
        // det F is a well-conditioned scaling done after rounding to T
        const T idF = T(1) / from_double<T>(dF);
        const T lnJ = from_double<T>(log_f64(dF));
        const T smu = s * mu_c;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
          o[k] = bad ? nan : from_double<T>(cof[k]) * idF;  // o[3 i + j] = Fi[i][j]
          o[9 + k] = bad ? nan : smu * ((k % 4 == 0 ? T(1) : T(0)) + gu[k]);
        }
        o[PW - 2] = bad ? nan : s * (mu_c - lam_c * lnJ);
        o[PW - 1] = s * lam_c;
      }
    }
    __syncthreads();

    // rows of points [g QG, g QG + QG) into buffer g & 1: Y = (Y0, Y1, Y2, Y2), Z = (Z0, Z1, Z2, 0)
    const int ngroups = QP / QG;
    const int rows_items = ne * NS;
    const float inv_items = 1.0f / (float)rows_items;
    auto make_rows = [&](int g) {
      T* Yb = rows + (size_t)(g & 1) * RW * RL;
      const int q0 = g * QG;
      for (int w = tid; w < QG * rows_items; w += NT) {
        const int qi = small_div(w, inv_items), r = w - qi * rows_items;
        const int e = r / NS, a = r - e * NS;
        const int qq = q0 + qi;
        const T* Ji = geo + GEO * e;
        T j[12];
        ld4(Ji, j[0], j[1], j[2], j[3]);
        ld4(Ji + 4, j[4], j[5], j[6], j[7]);
        ld4(Ji + 8, j[8], j[9], j[10], j[11]);
        const T live = qq < Q ? T(1) : T(0);   // padded points: zero rows
        const T* dp = dphi + ((qq < Q ? qq : 0) * NS + a) * 3;
        const T d0 = live * dp[0], d1 = live * dp[1], d2 = live * dp[2];
        T G[3];
#pragma unroll
        for (int x = 0; x < 3; ++x) G[x] = j[x] * d0 + j[3 + x] * d1 + j[6 + x] * d2;
        const size_t slot = (((size_t)qi * TE + e) * NSP + a) * 4;
        T Y[3];
        if constexpr (NEO) {
          const T* pw = PWs + PW * (e * QP + qq);
          T f[20];
#pragma unroll
          for (int k = 0; k < 20; k += 4) ld4(pw + k, f[k], f[k + 1], f[k + 2], f[k + 3]);
#pragma unroll
          for (int x = 0; x < 3; ++x) Y[x] = G[0] * f[x] + G[1] * f[3 + x] + G[2] * f[6 + x];
          T z[3];
#pragma unroll
          for (int i = 0; i < 3; ++i) z[i] = f[9 + 3 * i] * G[0] + f[10 + 3 * i] * G[1] + f[11 + 3 * i] * G[2];
          st4(Yb + RL + slot, z[0], z[1], z[2], T(0));
        } else {
          Y[0] = G[0]; Y[1] = G[1]; Y[2] = G[2];
        }
        st4(Yb + slot, Y[0], Y[1], Y[2], Y[2]);
      }
    };

    // this thread's run of trial functions
    const int el = tid % EF, slot = tid / EF;
    const int grp = slot / NCH, ch = slot - grp * NCH;
    const int te = grp * EF + el;
    const bool owner = grp < GROUPS && te < ne;
    const unsigned cw = owner ? kSymChunks<NS, BB>.c[ch] : 0u;
    const int a = (int)(cw & 0xffu), b0 = (int)((cw >> 8) & 0xffu), nb = (int)(cw >> 16);

    V2 w1r[BB][3], w2r[BB][3], w1c[BB], w2c[BB], dd[BB];
    T w1s[BB], w2s[BB], ds[BB];
#pragma unroll
    for (int i = 0; i < BB; ++i) {
#pragma unroll
      for (int c = 0; c < 3; ++c) w1r[i][c] = w2r[i][c] = vmk(T(0), T(0));
      w1c[i] = w2c[i] = dd[i] = vmk(T(0), T(0));
      w1s[i] = w2s[i] = ds[i] = T(0);
    }

    make_rows(0);
    __syncthreads();
    for (int g = 0; g < ngroups; ++g) {
      if (owner) {
        const T* Yb = rows + (size_t)(g & 1) * RW * RL;
        const int q0 = g * QG;
#pragma unroll
        for (int qi = 0; qi < QG; ++qi) {
          const T* yr = Yb + (((size_t)qi * TE + te) * NSP) * 4;
          const T* pw = PWs + PW * (te * QP + q0 + qi);
          const V2 sw = *reinterpret_cast<const V2*>(pw + PW - 2);
          const T sal = sw.x, slam = sw.y;
          T y0, y1, y2, y3;
          ld4(yr + 4 * a, y0, y1, y2, y3);
          // a-side factors: (s alpha Y_a[c]) and (s lam Y_a[c]) duplicated, and the
          // column pairs (Y_a[0], Y_a[1]) of the d = 2 entries
          const T p0 = sal * y0, p1 = sal * y1, p2 = sal * y2;
          const T l0 = slam * y0, l1 = slam * y1, l2 = slam * y2;
          const V2 P0 = vmk(p0, p0), P1 = vmk(p1, p1), P2 = vmk(p2, p2), PC = vmk(p0, p1);
          const V2 L0 = vmk(l0, l0), L1 = vmk(l1, l1), L2 = vmk(l2, l2), LC = vmk(l0, l1);
          V2 Z01 = vmk(T(0), T(0));
          T Z2 = T(0);
          if constexpr (NEO) {
            T z0, z1, z2, z3;
            ld4(yr + RL + 4 * a, z0, z1, z2, z3);
            Z01 = vmk(z0, z1);
            Z2 = z2;
          }
#pragma unroll
          for (int i = 0; i < BB; ++i) {
            if (i < nb) {
              T b0v, b1v, b2v, b3v;
              ld4(yr + 4 * (b0 + i), b0v, b1v, b2v, b3v);
              const V2 Y01 = vmk(b0v, b1v), Y22 = vmk(b2v, b3v);
              w1r[i][0] = vfma(P0, Y01, w1r[i][0]);
              w1r[i][1] = vfma(P1, Y01, w1r[i][1]);
              w1r[i][2] = vfma(P2, Y01, w1r[i][2]);
              w1c[i] = vfma(PC, Y22, w1c[i]);
              w1s[i] = fma(p2, b2v, w1s[i]);
              w2r[i][0] = vfma(L0, Y01, w2r[i][0]);
              w2r[i][1] = vfma(L1, Y01, w2r[i][1]);
              w2r[i][2] = vfma(L2, Y01, w2r[i][2]);
              w2c[i] = vfma(LC, Y22, w2c[i]);
              w2s[i] = fma(l2, b2v, w2s[i]);
              if constexpr (NEO) {
                dd[i] = vfma(Z01, Y01, dd[i]);
                ds[i] = fma(Z2, b2v, ds[i]);
              }
            }
          }
        }
      }
      if (g + 1 < ngroups) make_rows(g + 1);  // the other buffer, last read in group g - 1
      __syncthreads();
    }
    if (owner) {
      T* st = stage + (size_t)te * NN;
#pragma unroll
      for (int i = 0; i < BB; ++i) {
        if (i < nb) {
          // W[c][d]: rows c = 0..2 hold d = 0, 1; the column pair holds (0, 2), (1, 2); the scalar (2, 2)
          const T W1[9] = {w1r[i][0].x, w1r[i][0].y, w1c[i].x, w1r[i][1].x, w1r[i][1].y, w1c[i].y,
                           w1r[i][2].x, w1r[i][2].y, w1s[i]};
          const T W2[9] = {w2r[i][0].x, w2r[i][0].y, w2c[i].x, w2r[i][1].x, w2r[i][1].y, w2c[i].y,
                           w2r[i][2].x, w2r[i][2].y, w2s[i]};
          const T D = NEO ? (dd[i].x + dd[i].y) + ds[i] : (W1[0] + W1[4]) + W1[8];
          T v[9];
#pragma unroll
          for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int d = 0; d < 3; ++d) v[3 * c + d] = (c == d ? D : T(0)) + W1[3 * d + c] + W2[3 * c + d];
          put_sym_block<N, T>(st, a, b0 + i, v);
        }
      }
    }
    __syncthreads();
    store_tile<NT, T>(q.out, e0 * NN, stage, ne * NN, q.out_f32);
    __syncthreads();
  }
};

}  // namespace fea
