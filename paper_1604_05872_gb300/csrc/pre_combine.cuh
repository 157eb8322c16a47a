// Local and global assembly in one pass, with the entries that the elements of
// one tile add to the same CSR position combined before the FP64 atomics.
//
// Element part: the streaming pre-evaluated schedule of pre_stream.cuh (bulk
// copies of the inputs one tile ahead, FP64 geometry, FP32 contraction
// A_e = sum_r R_r H_e[r] of Algorithm 2, in the same order, so the same bits).
// Global part (Section 2: the global matrix is the sum of the element matrices
// at their global DOFs): the tile's element entries are staged in shared memory
// (FP32), then every distinct CSR position the tile touches is summed from the
// stage in FP64 (each entry widened exactly, so the result differs from the
// two-pass assembly only in the order of the FP64 additions) and added to the
// CSR values with one FP64 atomic.  On the cube mesh at P2, 57% of a tile's
// entries fall on distinct positions: 57 atomics per element instead of 100.
//
// Which entries meet at which position depends on the mesh alone; the host
// computes it once per mesh, per tile of T elements (fea_csr_combine_plan), as a
// plan of 32-bit words:
//
//   words 0..3          magic, n (local dimension), T (elements per tile), 0
//   words 4..           int64 word offsets of the ntiles + 1 tile records
//   tile record         U (distinct positions), R (largest number of entries at
//                       one position), L (entries of the tile that are added), 0;
//                       cnt[R]: cnt[r] = positions with more than r entries (the
//                       positions are ordered by that number, largest first);
//                       pos[U]: the CSR positions;
//                       idx[L] (16-bit): tile entries e n^2 + i n + j, round r
//                       holding the r-th entry of positions 0 .. cnt[r] - 1;
//                       each of the three arrays padded to a multiple of 4 words.
//
// Each tile's record reaches shared memory by one bulk copy (the TMA engine),
// issued when the tile starts and overlapping its contraction.  After the
// contraction the first warps (one lane per element) form the next tile's FP64
// geometry while the other threads combine: combining thread s sums the entries
// of positions s, s + NCT, ... round by round from shared memory alone, two
// positions per thread in flight.  Tiles hold at
// most 3200 entries (T = min(128, 3200 / n^2): 32 elements at P2, so that with
// 64 registers four CTAs fit on an SM; the combine phase is latency-bound and
// lives on resident warps), so a record never exceeds PW words.  Every plan read stays
// inside the tile record, every stage read inside the tile's entries and every
// atomic inside [0, nnz): a plan that breaks a bound is flagged (ERR_PATTERN) and
// the offending entry or tile skipped.
#pragma once
#include "common.cuh"
#include "kernels.h"
#include "mbar.cuh"
#include "pre_stream.cuh"

namespace fea {

// Exact widening of any float (infinities and NaN included); subnormal inputs,
// which the flush-to-zero contraction does not produce, widen to zero.
__device__ __forceinline__ double f2d_exact(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t a = u & 0x7fffffffu;
  const bool normal = a >= 0x00800000u && a < 0x7f800000u;
  uint32_t hi;
  if (a >= 0x7f800000u) hi = 0x7ff00000u | (a > 0x7f800000u ? 0x00080000u : 0u);  // inf, quiet NaN
  else hi = normal ? (a >> 3) + 0x38000000u : 0u;
  return __hiloint2double((int)(hi | (u & 0x80000000u)), (int)(normal ? a << 29 : 0u));
}

template <int FORM, int P>
struct PreCombine {
  using K = PreStream<FORM, P>;
  static constexpr int TC = (3200 / K::NN) < 2 ? 2 : (3200 / K::NN > 128 ? 128 : (3200 / K::NN) & ~1);  // tile
  static constexpr int PW = 4 + round_up(TC, 4) + round_up(TC * K::NN, 4) + round_up((TC * K::NN + 1) / 2, 4);
  FEA_HD static size_t off_stage(int TE) { return K::off_bar(TE) + 32; }
  FEA_HD static size_t off_plan(int TE) { return off_stage(TE) + round_up_sz((size_t)TE * K::NN * 4, 16); }
  FEA_HD static size_t smem(int TE) { return off_plan(TE) + (size_t)PW * 4; }
};

template <int FORM, int P>
__global__ void __launch_bounds__(NT, P == 2 ? 4 : 1) pre_combine_kernel(Req q, CombineArgs cb, unsigned* err) {
  using K = PreStream<FORM, P>;
  using C = PreCombine<FORM, P>;
  extern __shared__ __align__(16) char sm[];
  const int TE = q.tile;
  double* in = reinterpret_cast<double*>(sm);             // [2][TE][IN]: coords block, then coeffs block
  float* H = reinterpret_cast<float*>(sm + K::off_h(TE));  // [2][TE][NHP]
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + K::off_bar(TE));
  float* stage = reinterpret_cast<float*>(sm + C::off_stage(TE));  // [TE][NN]
  int32_t* rec = reinterpret_cast<int32_t*>(sm + C::off_plan(TE));  // [PW]: the tile's plan record
  __shared__ __align__(8) uint64_t rec_bar;
  __shared__ int s_abort, s_rec_words;
  const TabLayout L = tab_layout(q.Q, K::NS, K::RTAB);
  const float* Rg = reinterpret_cast<const float*>(q.tab) + L.offR;
  const int64_t ntiles = (q.E + TE - 1) / TE;
  const int64_t first = blockIdx.x;
  if (first >= ntiles) return;
  {
    unsigned dyn;
    asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
    if (C::smem(TE) > dyn) {  // refuse a tile that does not fit the launch
      if (threadIdx.x == 0) flag_error(err, 4u);
      return;
    }
  }
  // the plan must be for this local dimension and tile (the host checked its size)
  const int64_t hdr = 4 + 2 * (ntiles + 1);
  if (cb.plan_words < hdr || __ldg(cb.plan) != kCombineMagic || __ldg(cb.plan + 1) != K::NS ||
      __ldg(cb.plan + 2) != TE || TE != C::TC) {
    if (threadIdx.x == 0) flag_error(err, ERR_PATTERN);
    return;
  }
  const int64_t* toff = reinterpret_cast<const int64_t*>(cb.plan + 4);
  const int64_t stride = gridDim.x;
  const int my_tiles = (int)((ntiles - first + stride - 1) / stride);

  const int t = threadIdx.x;
  const bool active = t < K::G * K::S;
  const int slot = t % K::S, g0 = t / K::S;
  // after the contraction the first GWT threads (whole warps, one lane per element)
  // form the next tile's geometry while the other NCT threads combine this tile
  constexpr int GWT = (C::TC + 31) / 32 * 32, NCT = NT - GWT;
  static_assert(NCT >= 64, "combining threads");

  auto tile_ne = [&](int j) {
    const int64_t e0 = (first + (int64_t)j * stride) * TE;
    return (int)(q.E - e0 < TE ? q.E - e0 : TE);
  };
  auto issue = [&](int j) {
    const int64_t e0 = (first + (int64_t)j * stride) * TE;
    const int ne = tile_ne(j), b = j & 1;
    double* dst = in + (size_t)b * TE * K::IN;
    const unsigned cbytes = (unsigned)ne * 96u, fbytes = (unsigned)ne * K::CLEN * 8u;
    fence_proxy_async();
    mbar_expect_tx(&bar[b], cbytes + fbytes);
    bulk_g2s(dst, q.coords + e0 * 12, cbytes, &bar[b]);
    if (K::CLEN) bulk_g2s(dst + (size_t)TE * 12, q.coeffs + e0 * K::CLEN, fbytes, &bar[b]);
  };
  auto wait_in = [&](int j) { return mbar_wait(&bar[j & 1], (unsigned)(j >> 1) & 1u); };
  auto geometry = [&](int j) {
    const int ne = tile_ne(j), b = j & 1;
    const double* xs = in + (size_t)b * TE * K::IN;
    if (t < ne) K::geometry_h(xs + 12 * t, xs + (size_t)TE * 12 + K::CLEN * t, H + (size_t)(b * TE + t) * K::NHP, err);
  };
  auto abort_all = [&](int j_lo, int j_hi) {
    for (int j = j_lo; j <= j_hi && j < my_tiles; ++j) wait_in(j);
  };
  // thread 0: bulk copy of the plan record of tile j (offsets a, b) into rec, or
  // a bare arrival when the record breaks a bound (s_rec_words = -1)
  auto issue_rec = [&](int64_t a, int64_t b) {
    const bool ok = a >= hdr && !(a & 3) && b <= cb.plan_words && a + 4 <= b && b - a <= C::PW;
    s_rec_words = ok ? (int)(b - a) : -1;
    fence_proxy_async();
    mbar_expect_tx(&rec_bar, ok ? (unsigned)(b - a) * 4u : 0u);
    if (ok) bulk_g2s(rec, cb.plan + a, (unsigned)(b - a) * 4u, &rec_bar);
  };
  // one FP64 atomic per distinct position of tile j, its entries summed from the stage
  auto combine = [&](int j) {
    const int tc = t - GWT;  // this thread's rank among the combining threads
    const int lim = tile_ne(j) * K::NN;
    const int words = s_rec_words;
    if (words < 0) {
      if (tc == 0) flag_error(err, ERR_PATTERN);
      return;
    }
    const int U = rec[0], R = rec[1], Ln = rec[2];
    if (U < 0 || R < 0 || R > TE || Ln < U || Ln > lim || (U > 0) != (R > 0)) {
      if (tc == 0) flag_error(err, ERR_PATTERN);
      return;
    }
    const int cw = (R + 3) & ~3, pw = (U + 3) & ~3, iw = ((Ln + 1) / 2 + 3) & ~3;
    if (4 + cw + pw + iw > words || (R > 0 && rec[4] != U)) {
      if (tc == 0) flag_error(err, ERR_PATTERN);
      return;
    }
    const int32_t* cnt = rec + 4;
    const int32_t* pos = cnt + cw;
    const uint16_t* idx = reinterpret_cast<const uint16_t*>(pos + pw);
    constexpr int IL = 2;  // positions per thread in flight (independent FP64 chains)
    for (int s0 = tc; s0 < U; s0 += IL * NCT) {
      int kk[IL];
      double acc[IL];
      bool bad = false;
#pragma unroll
      for (int i = 0; i < IL; ++i) {
        const int s = s0 + i * NCT;
        kk[i] = s < U ? idx[s] : 0;
        bad |= kk[i] >= lim;
        acc[i] = (s < U && kk[i] < lim) ? f2d_exact(stage[kk[i]]) : 0.0;
      }
      int off = U;
      for (int r = 1; r < R; ++r) {
        const int c = cnt[r];
        if (s0 >= c) break;
#pragma unroll
        for (int i = 0; i < IL; ++i) {
          const int s = s0 + i * NCT, o = off + s;
          const bool on = s < c && o < Ln;
          if (s < c && o >= Ln) bad = true;
          kk[i] = on ? idx[o] : 0;
          if (on) {
            if (kk[i] < lim) acc[i] += f2d_exact(stage[kk[i]]);
            else bad = true;
          }
        }
        off += c;
      }
#pragma unroll
      for (int i = 0; i < IL; ++i) {
        const int s = s0 + i * NCT;
        if (s < U) {
          const int64_t m = pos[s];
          if (m >= 0 && m < cb.nnz) atomicAdd(cb.values + m, acc[i]);
          else bad = true;
        }
      }
      if (bad) flag_error(err, ERR_PATTERN);
    }
  };

  if (t == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_init(&rec_bar, 1);
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

  // record offsets of the next tile, loaded one tile ahead by thread 0
  int64_t ra = 0, rb = 0;
  if (t == 0) {
    ra = __ldg(toff + first);
    rb = __ldg(toff + first + 1);
  }
  for (int j = 0; j < my_tiles; ++j) {
    const int ne = tile_ne(j);
    if (t == 0) {
      if (j + 2 < my_tiles) issue(j + 2);
      issue_rec(ra, rb);  // rec is free: the combine of tile j - 1 ended before the last barrier
      if (j + 1 < my_tiles) {
        ra = __ldg(toff + first + (int64_t)(j + 1) * stride);
        rb = __ldg(toff + first + (int64_t)(j + 1) * stride + 1);
      }
    }
    if (active) {
      float r0[K::R], r1[K::R];
#pragma unroll
      for (int r = 0; r < K::R; ++r) {
        const float2 x = __ldg(reinterpret_cast<const float2*>(Rg + (size_t)r * K::RSTRIDE) + slot);
        r0[r] = x.x;
        r1[r] = x.y;
      }
      const float* Hb = H + (size_t)(j & 1) * TE * K::NHP;
      float2* st = reinterpret_cast<float2*>(stage) + slot;
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
        st[(size_t)e * K::S] = make_float2(a0, a1);
        st[(size_t)(e + K::G) * K::S] = make_float2(b0, b1);
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
        st[(size_t)e * K::S] = make_float2(a0, a1);
      }
    }
    __syncthreads();  // the stage holds tile j
    if (t < GWT) {
      // inputs of tile j + 1 -> geometry into the other H buffer
      if (j + 1 < my_tiles) {
        if (wait_in(j + 1)) {
          geometry(j + 1);
        } else {
          flag_error(err, ERR_TIMEOUT);
          s_abort = 1;
        }
      }
    } else if (mbar_wait(&rec_bar, (unsigned)j & 1u)) {
      combine(j);
    } else {
      flag_error(err, ERR_TIMEOUT);
      s_abort = 1;
    }
    __syncthreads();  // the stage is free, H of tile j + 1 is complete
    if (s_abort) {
      abort_all(j + 1, j + 2);
      return;
    }
  }
}

}  // namespace fea
