// Pre-evaluated scalar forms (mass, Helmholtz; P1, P2) on the tcgen05 tensor
// cores, for FP32 output under the split-BF16 precision.
//
// Algorithm 2 (Section 3.3) contracts, per element, the geometry tensor H_e with
// the pre-evaluated reference tensors: A_e[i][j] = sum_r R_r[i][j] H_e[r].  For a
// tile of 128 elements that is one dense product, computed transposed
//
//   D[M x 128] = R[M x K] * H[128 x K]^T,   K = terms r (padded to 16),
//                                          M = 128 >= entries (i, j),
//
// which with FP32 output is compute-bound on the CUDA cores (the element
// matrices leave at 400 B per element at P2, less than the FMA work takes).
// Both operands are split into three BF16 parts (x = x0 + x1 + x2, each part the
// rounded remainder of the previous ones: 24 bits in all), H per tile in shared
// memory (one row per element, written by the element's own thread), R once per
// CTA from the host-split table; the six products x_i y_j with i + j <= 2
// accumulate in FP32 in tensor memory (two BF16 parts per operand, 16 bits,
// left errors of 1e-5 on cancelling Helmholtz rows).  Lane m of the
// accumulator is entry m and column e is element e, so a warp reads 32
// consecutive entries of one element per column and stores them straight from
// registers as one coalesced 128-byte (FP64: 256-byte) line: no staging in
// shared memory.
//
// Two roles of four warps, double-buffered H rows and accumulators: the
// producers (one thread per element) load the inputs one tile ahead, form the
// FP64 geometry (the streaming kernel's geometry_h) and the split H rows of tile
// j, and one of them issues tile j's product; meanwhile the consumers read tile
// j - 1's accumulator and store it.  Handoffs are mbarriers: full[b] (the
// product in buffer b completed, via tcgen05.commit) and empty[b] (its
// accumulator has been read).  Every wait is bounded; a wait that gives up sets
// the error word, and the CTA waits (bounded) for its products in flight before
// it frees its tensor memory.
#pragma once
#include "common.cuh"
#include "mbar.cuh"
#include "nh_tce.cuh"  // mma_f16_ss
#include "pre_stream.cuh"
#include "tc.cuh"

namespace fea {

// A packed pair (x, y) -> three BF16 pairs: part 0 = x rounded, part 1 = the
// remainder rounded, part 2 = the remainder of that rounded (x low, each
// remainder exact in FP32).
__device__ __forceinline__ void split3_bf16_pair(float2 v, uint32_t& p0, uint32_t& p1, uint32_t& p2) {
  const __nv_bfloat162 b0 = __float22bfloat162_rn(v);
  const float2 r1 = make_float2(v.x - __low2float(b0), v.y - __high2float(b0));
  const __nv_bfloat162 b1 = __float22bfloat162_rn(r1);
  const float2 r2 = make_float2(r1.x - __low2float(b1), r1.y - __high2float(b1));
  const __nv_bfloat162 b2 = __float22bfloat162_rn(r2);
  p0 = *reinterpret_cast<const uint32_t*>(&b0);
  p1 = *reinterpret_cast<const uint32_t*>(&b1);
  p2 = *reinterpret_cast<const uint32_t*>(&b2);
}

template <int FORM, int P>
struct PreTc {
  using K = PreStream<FORM, P>;
  static constexpr int TE = 128, NTH = 256;  // producers: threads 0-127, consumers: 128-255
  static constexpr int KK = round_up(K::R, 16);  // K of the product
  static constexpr int KC = KK / 8;              // 16-byte chunks along K
  static_assert(K::NN <= 128, "the entries fit the 128 accumulator lanes");
  static constexpr int M = 128;                  // accumulator lanes: entries, padded
  static constexpr uint32_t LBO = 128, SBO = KC * 128;
  static constexpr uint32_t TMEM_COLS = 2 * TE;  // two accumulators, one column per element
  static constexpr int H_BYTES = TE * KK * 2, R_BYTES = M * KK * 2;
  static constexpr int O_R = 0, O_H = 3 * R_BYTES;  // parts 0, 1, 2 of R (the A operand), then of H (B), x2
  // at least 80 KB of shared memory: at most two CTAs per SM, whose accumulators
  // (256 columns each) fill the 512 tensor-memory columns (a third would wait in
  // its allocation until another CTA ends)
  static constexpr int SMEM = O_H + 6 * H_BYTES > 81920 ? O_H + 6 * H_BYTES : 81920;
  static constexpr int TABLE_WORDS = R_BYTES / 4;  // 32-bit words of one part of R (parts 0, 1, 2 follow)
  // byte offset of (row, k) in a K-major operand without swizzle
  FEA_HD static constexpr uint32_t kmajor_off(int row, int k) {
    return (uint32_t)(row >> 3) * SBO + (uint32_t)(k >> 3) * LBO + (uint32_t)(row & 7) * 16u + (uint32_t)(k & 7) * 2u;
  }
};

template <int FORM, int P>
__global__ void __launch_bounds__(256) pre_tc_kernel(Req q, unsigned* err) {
  using C = PreTc<FORM, P>;
  using K = typename C::K;
  extern __shared__ __align__(16) char sm[];
  __shared__ __align__(8) uint64_t full_bar[2], empty_bar[2];
  __shared__ uint32_t tbase_s;
  const int t = threadIdx.x, warp = t >> 5;
  const int64_t ntiles = (q.E + C::TE - 1) / C::TE;
  if ((int64_t)blockIdx.x >= ntiles) return;
  {
    unsigned dyn;
    asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
    if ((unsigned)C::SMEM > dyn || q.tile != C::TE || blockDim.x != (unsigned)C::NTH) {
      if (t == 0) flag_error(err, 4u);  // refuse a launch this layout does not fit
      return;
    }
  }
  // A operand: the host-split reference tensors R (parts 0, 1, 2), once per CTA
  {
    const uint4* tab = reinterpret_cast<const uint4*>(q.tab);
    uint4* a = reinterpret_cast<uint4*>(sm + C::O_R);
    for (int i = t; i < 3 * C::R_BYTES / 16; i += C::NTH) a[i] = __ldg(tab + i);
  }
  if (warp == 0) {
    tmem_alloc(&tbase_s, C::TMEM_COLS);
    tmem_relinquish();
  }
  if (t == 0) {
    for (int b = 0; b < 2; ++b) {
      mbar_init(&full_bar[b], 1);
      mbar_init(&empty_bar[b], 4);  // one arrival per consumer warp
    }
    fence_barrier_init();
  }
  fence_proxy_async();  // R, written by threads, is read by the tensor core
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tb = tbase_s;
  const uint32_t sbase = smem_addr(sm);
  constexpr uint32_t idesc = idesc_f16kind(1u, (uint32_t)C::M, (uint32_t)C::TE);
  const int my_tiles = (int)((ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x);
  bool ok = true;
  int issued = 0;  // products issued (producer thread 0)

  if (t < 128) {
    // ------------------------------------------------------------- producers
    double x[12], cf[K::CLEN > 0 ? K::CLEN : 1];
    auto load = [&](int64_t tile) {
      const int64_t e = tile * C::TE + t;
      if (e < q.E) {
        const double2* xs = reinterpret_cast<const double2*>(q.coords + e * 12);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          const double2 v = __ldg(xs + k);
          x[2 * k] = v.x;
          x[2 * k + 1] = v.y;
        }
        if constexpr (K::CLEN > 0) {
#pragma unroll
          for (int k = 0; k < K::CLEN; ++k) cf[k] = __ldg(q.coeffs + e * K::CLEN + k);
        }
      }
    };
    load(blockIdx.x);
    for (int j = 0; j < my_tiles; ++j) {
      const int64_t tile = blockIdx.x + (int64_t)j * gridDim.x;
      const int ne = (int)(q.E - tile * C::TE < C::TE ? q.E - tile * C::TE : C::TE);
      const int b = j & 1;
      __align__(16) float h[K::NHP];
#pragma unroll
      for (int k = 0; k < K::NHP; ++k) h[k] = 0.f;
      if (t < ne) K::geometry_h(x, cf, h, err);
      if (j + 1 < my_tiles) load(tile + gridDim.x);
      // H rows of buffer b were last read by the product of tile j - 2
      if (j >= 2 && !mbar_wait(&full_bar[b], (unsigned)((j - 2) >> 1) & 1u)) ok = false;
      if (!named_and(1, 128, ok)) break;
      char* hb = sm + C::O_H + b * 3 * C::H_BYTES;
#pragma unroll
      for (int kc = 0; kc < C::KC; ++kc) {
        uint32_t w0[4], w1[4], w2[4];
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          const int k = 8 * kc + 2 * w;
          split3_bf16_pair(make_float2(k < K::NHP ? h[k] : 0.f, k + 1 < K::NHP ? h[k + 1] : 0.f), w0[w], w1[w], w2[w]);
        }
        const uint32_t off = C::kmajor_off(t, 8 * kc);
        *reinterpret_cast<uint4*>(hb + off) = make_uint4(w0[0], w0[1], w0[2], w0[3]);
        *reinterpret_cast<uint4*>(hb + C::H_BYTES + off) = make_uint4(w1[0], w1[1], w1[2], w1[3]);
        *reinterpret_cast<uint4*>(hb + 2 * C::H_BYTES + off) = make_uint4(w2[0], w2[1], w2[2], w2[3]);
      }
      fence_proxy_async();  // the H rows, written by threads, are read by the tensor core
      named_sync(1, 128);
      if (t == 0) {
        // accumulator b was last read by the consumers for tile j - 2
        bool free_b = j < 2 || mbar_wait(&empty_bar[b], (unsigned)((j - 2) >> 1) & 1u);
        if (free_b) {
          tc_fence_after();
          // D_b = sum over the parts i + j <= 2 of R_i H_j^T, K in steps of 16 (256 B of descriptor start)
          constexpr int PI[6] = {0, 0, 1, 0, 1, 2}, PJ[6] = {0, 1, 0, 2, 1, 0};
          const uint32_t d = tb + (uint32_t)(b * C::TE);
#pragma unroll
          for (int pr = 0; pr < 6; ++pr) {
            const uint32_t a = sbase + C::O_R + PI[pr] * C::R_BYTES;
            const uint32_t bb = sbase + C::O_H + (b * 3 + PJ[pr]) * C::H_BYTES;
#pragma unroll
            for (int kk = 0; kk < C::KK / 16; ++kk)
              mma_f16_ss(d, smem_desc_kmajor(a + 256u * kk, C::LBO, C::SBO),
                         smem_desc_kmajor(bb + 256u * kk, C::LBO, C::SBO), idesc, (pr > 0 || kk > 0) ? 1u : 0u);
          }
          tc_commit(&full_bar[b]);
          ++issued;
        } else {
          flag_error(err, ERR_TIMEOUT);
          ok = false;
        }
      }
      if (!named_and(1, 128, ok)) break;
    }
  } else {
    // ------------------------------------------------------------- consumers
    const int cw = warp - 4;  // tensor-memory lanes 32 cw .. 32 cw + 31: entries
    const int entry = 32 * cw + (t & 31);
    const bool live = entry < K::NN;
    for (int j = 0; j < my_tiles; ++j) {
      const int64_t tile = blockIdx.x + (int64_t)j * gridDim.x;
      const int64_t e0 = tile * C::TE;
      const int ne = (int)(q.E - e0 < C::TE ? q.E - e0 : C::TE);
      const int b = j & 1;
      if (!mbar_wait(&full_bar[b], (unsigned)(j >> 1) & 1u)) ok = false;
      if (!named_and(2, 128, ok)) break;
      tc_fence_after();
      if (32 * cw < K::NN) {
#pragma unroll 1
        for (int c = 0; c < C::TE / 16; ++c) {
          if (16 * c >= ne) break;
          uint32_t r[16];
          tmem_ld16(tb + ((uint32_t)(32 * cw) << 16) + (uint32_t)(b * C::TE) + 16u * c, r);
          tmem_wait_ld();
          if (q.out_f32) {
            float* o = static_cast<float*>(q.out) + (e0 + 16 * c) * K::NN + entry;
#pragma unroll
            for (int v = 0; v < 16; ++v)
              if (live && 16 * c + v < ne) __stcs(o + v * K::NN, __uint_as_float(r[v]));
          } else {
            double* o = static_cast<double*>(q.out) + (e0 + 16 * c) * K::NN + entry;
#pragma unroll
            for (int v = 0; v < 16; ++v)
              if (live && 16 * c + v < ne) __stcs(o + v * K::NN, f2d_ftz(__uint_as_float(r[v])));
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if ((t & 31) == 0) mbar_arrive(&empty_bar[b]);
    }
  }
  if (!ok && t == 0) {
    flag_error(err, ERR_TIMEOUT);
    // products still in flight land before their memory is freed (bounded)
    for (int j = issued - 2 < 0 ? 0 : issued - 2; j < issued; ++j) mbar_wait(&full_bar[j & 1], (unsigned)(j >> 1) & 1u);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tb, C::TMEM_COLS);
  }
}

}  // namespace fea
