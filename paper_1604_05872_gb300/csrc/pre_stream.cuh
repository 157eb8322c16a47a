// Streaming form of the pre-evaluated variant for scalar forms with an even
// number of matrix entries (mass and Helmholtz, P1-P3), FP32 contraction.
//
// Same arithmetic as PreTile (Algorithm 2: A_e = sum_r R_r H_e[r]); the
// schedule is built for the HBM stream on sm_103a:
//   * persistent CTAs; each tile's coordinates and coefficients arrive by a
//     1-D bulk tensor copy (cp.async.bulk, the TMA engine) into one of two
//     shared buffers, completing on an mbarrier, one tile ahead of use;
//   * one thread per element does the FP64 geometry and writes the FP32
//     geometry tensor H_e straight to shared memory;
//   * each thread keeps two columns of R in registers and sweeps its elements
//     two at a time, storing each finished pair of entries with one 16-byte
//     streaming store (no staging: the element's entries are contiguous and
//     16-byte aligned).
// Every mbarrier wait is bounded; a wait that gives up sets the error word and
// the whole CTA leaves the kernel.
//
// The same schedule also serves local and global assembly in one pass
// (pre_stream_scatter_kernel): instead of storing the pair of entries, the
// thread adds them into the CSR values of the global matrix at the positions
// map[e][i][j] (one 8- or 16-byte map load per pair, two FP64 atomics), so the
// element matrices never reach HBM.
#pragma once
#include "common.cuh"
#include "mbar.cuh"

namespace fea {

template <int FORM, int P>
struct PreStream {
  static_assert(FORM == 0 || FORM == 1, "scalar forms");
  static constexpr int NS = nbasis_c(P);
  static constexpr int NN = NS * NS;
  static_assert(NN % 2 == 0, "even entry count");
  static constexpr int R = pre_terms_c(FORM, P);
  static constexpr int NHP = round_up(R, 4);
  static constexpr int CLEN = coeff_len_c(FORM, P);
  static constexpr int S = NN / 2;                 // pair slots
  static constexpr int G = S >= NT ? 1 : NT / S;   // element groups
  static constexpr int IN = 12 + CLEN;             // doubles of input per element
  static constexpr int NOUT = NN;                  // output entries per element
  static constexpr int RTAB = R;                   // terms of the device table
  static constexpr int RSTRIDE = NN;               // floats between consecutive terms of R

  FEA_HD static size_t off_h(int TE) { return round_up_sz((size_t)2 * TE * IN * 8, 16); }
  FEA_HD static size_t off_bar(int TE) { return off_h(TE) + round_up_sz((size_t)2 * TE * NHP * 4, 16); }
  FEA_HD static size_t smem(int TE, int Q) { (void)Q; return off_bar(TE) + 16 + 16; }
  FEA_HD static int max_tile() { return NT; }

  __device__ static void geometry_h(const double* x, const double* c, float* h, unsigned* err) {
    double adj[9];
    const double det = geometry_fp64(x, adj);
    const uint64_t bits = (uint64_t)__double_as_longlong(det);
    const bool bad = ((bits << 1) == 0) || ((bits >> 52 & 0x7ff) == 0x7ff);  // zero, inf or NaN
    if (bad) flag_error(err, ERR_DEGENERATE);
    const float ad = __uint_as_float(__float_as_uint(d2f(det)) & 0x7fffffffu);
    const float nan = __int_as_float(0x7fc00000);
    float v[NHP];
#pragma unroll
    for (int k = 0; k < NHP; ++k) v[k] = 0.f;
    if constexpr (FORM == 0) {
      v[0] = ad;
    } else {
      float a[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) a[k] = d2f(adj[k]);
      const float inv = 1.0f / ad;
      const int al[6] = {0, 1, 2, 0, 0, 1}, be[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
      for (int k = 0; k < 6; ++k)
        v[k] = (a[3 * al[k]] * a[3 * be[k]] + a[3 * al[k] + 1] * a[3 * be[k] + 1] + a[3 * al[k] + 2] * a[3 * be[k] + 2]) * inv;
#pragma unroll
      for (int k = 0; k < NS; ++k) v[6 + k] = ad * d2f(c[k]);
    }
#pragma unroll
    for (int k = 0; k < NHP; k += 4) {
      float4 w;
      w.x = bad ? nan : v[k]; w.y = bad ? nan : v[k + 1]; w.z = bad ? nan : v[k + 2]; w.w = bad ? nan : v[k + 3];
      *reinterpret_cast<float4*>(h + k) = w;
    }
  }
};

// The Helmholtz load vector b_e = |det J| M f_e (mass reference matrix M =
// int phi_i phi_k, the mass form's one-term table; P1-P3, NS even) on the same
// schedule: the "terms" are the NS coefficient DOFs, the geometry tensor is
// |det J| f_e (FP64 det J, FP32 product), each thread holds two rows of M.
template <int P>
struct PreStreamLoad {
  static constexpr int NS = nbasis_c(P);
  static_assert(NS % 2 == 0, "even entry count");
  static constexpr int NOUT = NS;
  static constexpr int R = NS;
  static constexpr int NHP = round_up(R, 4);
  static constexpr int CLEN = NS;
  static constexpr int S = NOUT / 2;
  static constexpr int G = S >= NT ? 1 : NT / S;
  static constexpr int IN = 12 + CLEN;
  static constexpr int RTAB = 1;
  static constexpr int RSTRIDE = NS;  // M is symmetric: term k of the pair (i, i + 1) is M[k][i], M[k][i + 1]

  FEA_HD static size_t off_h(int TE) { return round_up_sz((size_t)2 * TE * IN * 8, 16); }
  FEA_HD static size_t off_bar(int TE) { return off_h(TE) + round_up_sz((size_t)2 * TE * NHP * 4, 16); }
  FEA_HD static size_t smem(int TE, int Q) { (void)Q; return off_bar(TE) + 16 + 16; }
  FEA_HD static int max_tile() { return NT; }

  __device__ static void geometry_h(const double* x, const double* c, float* h, unsigned* err) {
    double J[3][3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int k = 0; k < 3; ++k) J[r][k] = x[3 * (k + 1) + r] - x[r];
    const double det = fma(J[0][0], fma(J[1][1], J[2][2], -J[1][2] * J[2][1]),
                           fma(J[0][1], fma(J[1][2], J[2][0], -J[1][0] * J[2][2]),
                               J[0][2] * fma(J[1][0], J[2][1], -J[1][1] * J[2][0])));
    const uint64_t bits = (uint64_t)__double_as_longlong(det);
    const bool bad = ((bits << 1) == 0) || ((bits >> 52 & 0x7ff) == 0x7ff);  // zero, inf or NaN
    if (bad) flag_error(err, ERR_DEGENERATE);
    const float ad = __uint_as_float(__float_as_uint(d2f(det)) & 0x7fffffffu);
    const float nan = __int_as_float(0x7fc00000);
    float v[NHP];
#pragma unroll
    for (int k = 0; k < NHP; ++k) v[k] = k < NS ? ad * d2f(c[k]) : 0.f;
#pragma unroll
    for (int k = 0; k < NHP; k += 4) {
      float4 w;
      w.x = bad ? nan : v[k]; w.y = bad ? nan : v[k + 1]; w.z = bad ? nan : v[k + 2]; w.w = bad ? nan : v[k + 3];
      *reinterpret_cast<float4*>(h + k) = w;
    }
  }
};

// Exact widening of a finite float that is normal or zero (no subnormals arise
// under flush-to-zero); NaN rows of degenerate elements are written separately.
__device__ __forceinline__ double f2d_finite(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t a = u & 0x7fffffffu;
  const uint32_t hi = (a ? (a >> 3) + 0x38000000u : 0u) | (u & 0x80000000u);
  return __hiloint2double((int)hi, (int)(a << 29));
}

// The fused global assembly adds values[map[e][i][j]] += A_e[i][j] (ScatterArgs),
// map int32 (MAPW 4) or int64 (MAPW 8); positions outside [0, nnz) are skipped
// and flagged.
template <int MAPW>
__device__ __forceinline__ void scatter_pair(const ScatterArgs& sc, int64_t k, double v0, double v1, unsigned* err) {
  int64_t m0, m1;
  if constexpr (MAPW == 4) {
    const int2 m = __ldg(reinterpret_cast<const int2*>(static_cast<const int32_t*>(sc.map) + k));
    m0 = m.x;
    m1 = m.y;
  } else {
    const longlong2 m = __ldg(reinterpret_cast<const longlong2*>(static_cast<const int64_t*>(sc.map) + k));
    m0 = m.x;
    m1 = m.y;
  }
  // -2: a lower-triangle entry under symmetric storage, not stored
  if (m0 >= 0 && m0 < sc.nnz) atomicAdd(sc.values + m0, v0);
  else if (m0 != -2) flag_error(err, ERR_PATTERN);
  if (m1 >= 0 && m1 < sc.nnz) atomicAdd(sc.values + m1, v1);
  else if (m1 != -2) flag_error(err, ERR_PATTERN);
}

// MAPW 0: store the element matrices; 4 or 8: add them into the CSR values.
template <class K, int MAPW>
__device__ __forceinline__ void pre_stream_body(const Req& q, unsigned* err, const ScatterArgs& sc) {
  extern __shared__ __align__(16) char sm[];
  const int TE = q.tile;
  double* in = reinterpret_cast<double*>(sm);                 // [2][TE][IN]: coords block, then coeffs block
  float* H = reinterpret_cast<float*>(sm + K::off_h(TE));      // [2][TE][NHP]
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + K::off_bar(TE));
  __shared__ int s_abort;
  const TabLayout L = tab_layout(q.Q, K::NS, K::RTAB);
  const float* Rg = reinterpret_cast<const float*>(q.tab) + L.offR;
  const int64_t ntiles = (q.E + TE - 1) / TE;
  const int64_t first = blockIdx.x;
  if (first >= ntiles) return;
  {
    unsigned dyn;
    asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
    if (K::smem(TE, q.Q) > dyn) {  // refuse a tile that does not fit the launch
      if (threadIdx.x == 0) flag_error(err, 4u);
      return;
    }
  }
  const int64_t stride = gridDim.x;
  const int my_tiles = (int)((ntiles - first + stride - 1) / stride);  // tiles this CTA runs: j = 0 .. my_tiles-1

  // thread -> (pair slot, element group); R columns live in registers
  const int t = threadIdx.x;
  const bool active = t < K::G * K::S;
  const int slot = t % K::S, g0 = t / K::S;

  auto tile_ne = [&](int j) {
    const int64_t e0 = (first + (int64_t)j * stride) * TE;
    return (int)(q.E - e0 < TE ? q.E - e0 : TE);
  };
  // one thread: bulk copies of the inputs of this CTA's j-th tile into buffer j & 1
  auto issue = [&](int j) {
    const int64_t e0 = (first + (int64_t)j * stride) * TE;
    if (q.skip_copy == first + (int64_t)j * stride + 1) return;  // test hook: this tile's inputs never come
    const int ne = tile_ne(j), b = j & 1;
    double* dst = in + (size_t)b * TE * K::IN;
    const unsigned cb = (unsigned)ne * 96u, fb = (unsigned)ne * K::CLEN * 8u;
    fence_proxy_async();
    mbar_expect_tx(&bar[b], cb + fb);
    bulk_g2s(dst, q.coords + e0 * 12, cb, &bar[b]);
    if (K::CLEN) bulk_g2s(dst + (size_t)TE * 12, q.coeffs + e0 * K::CLEN, fb, &bar[b]);
  };
  // all threads: wait for tile j's inputs (bounded); false after a time-out
  auto wait_in = [&](int j) { return mbar_wait(&bar[j & 1], (unsigned)(j >> 1) & 1u); };
  // threads < ne: FP64 geometry of tile j into H buffer j & 1
  auto geometry = [&](int j) {
    const int ne = tile_ne(j), b = j & 1;
    const double* xs = in + (size_t)b * TE * K::IN;
    if (t < ne) K::geometry_h(xs + 12 * t, xs + (size_t)TE * 12 + K::CLEN * t, H + (size_t)(b * TE + t) * K::NHP, err);
  };
  auto abort_all = [&](int j_lo, int j_hi) {
    // a copy in flight must land before the CTA leaves: bounded waits on the pending tiles
    for (int j = j_lo; j <= j_hi && j < my_tiles; ++j) wait_in(j);
  };

  if (t == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_barrier_init();
    s_abort = 0;
  }
  __syncthreads();
  if (t == 0) {
    issue(0);
    if (my_tiles > 1) issue(1);
  }
  if (!wait_in(0)) {
    flag_error(err, ERR_TIMEOUT);
    s_abort = 1;
  }
  __syncthreads();
  if (s_abort) {
    abort_all(0, 1);
    return;
  }
  geometry(0);
  __syncthreads();

  for (int j = 0; j < my_tiles; ++j) {
    const int64_t e0 = (first + (int64_t)j * stride) * TE;
    const int ne = tile_ne(j);
    // inputs of tile j + 2 go into the buffer tile j used (consumed before the last barrier)
    if (t == 0 && j + 2 < my_tiles) issue(j + 2);
    if (active) {
      // this thread's two columns of R, reloaded per tile (L1 hits) so that they
      // are not live across the FP64 geometry
      float r0[K::R], r1[K::R];
#pragma unroll
      for (int r = 0; r < K::R; ++r) {
        const float2 x = __ldg(reinterpret_cast<const float2*>(Rg + (size_t)r * K::RSTRIDE) + slot);
        r0[r] = x.x;
        r1[r] = x.y;
      }
      const float* Hb = H + (size_t)(j & 1) * TE * K::NHP;
      double2* o = reinterpret_cast<double2*>(reinterpret_cast<double*>(q.out) + e0 * K::NOUT) + slot;
      float2* of = reinterpret_cast<float2*>(reinterpret_cast<float*>(q.out) + e0 * K::NOUT) + slot;
      const double2 nan2 = make_double2(__longlong_as_double(0x7ff8000000000000ll), __longlong_as_double(0x7ff8000000000000ll));
      // two elements per iteration: independent accumulation chains
      int e = g0;
      for (; e + K::G < ne; e += 2 * K::G) {
        const float* h = Hb + K::NHP * e;
        const float* h2 = h + K::NHP * K::G;
        float a0 = 0.f, a1 = 0.f, b0 = 0.f, b1 = 0.f;
#pragma unroll
        for (int r4 = 0; r4 < K::NHP; r4 += 4) {
          const float4 hv = *reinterpret_cast<const float4*>(h + r4);
          const float4 gv = *reinterpret_cast<const float4*>(h2 + r4);
          const float hh[4] = {hv.x, hv.y, hv.z, hv.w};
          const float gg[4] = {gv.x, gv.y, gv.z, gv.w};
#pragma unroll
          for (int k = 0; k < 4; ++k)
            if (r4 + k < K::R) {
              a0 = fmaf(r0[r4 + k], hh[k], a0);
              a1 = fmaf(r1[r4 + k], hh[k], a1);
              b0 = fmaf(r0[r4 + k], gg[k], b0);
              b1 = fmaf(r1[r4 + k], gg[k], b1);
            }
        }
        if constexpr (MAPW != 0) {
          const double2 v = h[0] != h[0] ? nan2 : make_double2(f2d_finite(a0), f2d_finite(a1));
          const double2 w = h2[0] != h2[0] ? nan2 : make_double2(f2d_finite(b0), f2d_finite(b1));
          scatter_pair<MAPW>(sc, (e0 + e) * K::NOUT + 2 * slot, v.x, v.y, err);
          scatter_pair<MAPW>(sc, (e0 + e + K::G) * K::NOUT + 2 * slot, w.x, w.y, err);
        } else if (q.out_f32) {
          __stcs(of + (size_t)e * (K::NOUT / 2), make_float2(a0, a1));
          __stcs(of + (size_t)(e + K::G) * (K::NOUT / 2), make_float2(b0, b1));
        } else {
          const double2 v = h[0] != h[0] ? nan2 : make_double2(f2d_finite(a0), f2d_finite(a1));
          const double2 w = h2[0] != h2[0] ? nan2 : make_double2(f2d_finite(b0), f2d_finite(b1));
          __stcs(o + (size_t)e * (K::NOUT / 2), v);
          __stcs(o + (size_t)(e + K::G) * (K::NOUT / 2), w);
        }
      }
      for (; e < ne; e += K::G) {
        const float* h = Hb + K::NHP * e;
        float a0 = 0.f, a1 = 0.f;
#pragma unroll
        for (int r4 = 0; r4 < K::NHP; r4 += 4) {
          const float4 hv = *reinterpret_cast<const float4*>(h + r4);
          const float hh[4] = {hv.x, hv.y, hv.z, hv.w};
#pragma unroll
          for (int k = 0; k < 4; ++k)
            if (r4 + k < K::R) {
              a0 = fmaf(r0[r4 + k], hh[k], a0);
              a1 = fmaf(r1[r4 + k], hh[k], a1);
            }
        }
        if constexpr (MAPW != 0) {
          const double2 v = h[0] != h[0] ? nan2 : make_double2(f2d_finite(a0), f2d_finite(a1));
          scatter_pair<MAPW>(sc, (e0 + e) * K::NOUT + 2 * slot, v.x, v.y, err);
        } else if (q.out_f32) {
          __stcs(of + (size_t)e * (K::NOUT / 2), make_float2(a0, a1));
        } else {
          __stcs(o + (size_t)e * (K::NOUT / 2), h[0] != h[0] ? nan2 : make_double2(f2d_finite(a0), f2d_finite(a1)));
        }
      }
    }
    // inputs of tile j + 1 (issued one iteration ago) -> geometry into the other H
    // buffer, last read by the contraction of tile j - 1 before the previous barrier
    if (j + 1 < my_tiles) {
      if (wait_in(j + 1)) {
        geometry(j + 1);
      } else {
        flag_error(err, ERR_TIMEOUT);
        s_abort = 1;
      }
    }
    __syncthreads();
    if (s_abort) {
      abort_all(j + 1, j + 2);
      return;
    }
  }
}

template <int FORM, int P>
__global__ void __launch_bounds__(NT) pre_stream_kernel(Req q, unsigned* err) {
  pre_stream_body<PreStream<FORM, P>, 0>(q, err, ScatterArgs{nullptr, 0, nullptr});
}

template <int FORM, int P, int MAPW>
__global__ void __launch_bounds__(NT) pre_stream_scatter_kernel(Req q, ScatterArgs sc, unsigned* err) {
  pre_stream_body<PreStream<FORM, P>, MAPW>(q, err, sc);
}

template <int P>
__global__ void __launch_bounds__(NT) pre_stream_load_kernel(Req q, unsigned* err) {
  pre_stream_body<PreStreamLoad<P>, 0>(q, err, ScatterArgs{nullptr, 0, nullptr});
}

}  // namespace fea
