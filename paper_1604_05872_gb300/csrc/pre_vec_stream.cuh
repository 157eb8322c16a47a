// Streaming form of the pre-evaluated elasticity kernel (P1-P3, FP32
// contraction): same arithmetic as PreVecTile (Algorithm 2 with the
// factorised block tr(M X) I + adj^T (X^T + L) adj, blocks a <= b mirrored),
// scheduled for the HBM store stream:
//   * persistent CTAs; every compute thread owns one pair (a, b) of one element
//     slot for the whole launch and keeps its 36 reference values in registers;
//   * the last warp is the producer: it evaluates the FP64 geometry of the next
//     batch of tiles (at least 32 elements, one per lane: an FP64 instruction
//     occupies the SM's FP64 unit for the whole warp whatever its active lanes)
//     while the compute warps contract the current batch;
//   * each finished tile (its element matrices are one contiguous range of the
//     output) leaves shared memory by one bulk asynchronous copy
//     (cp.async.bulk, the TMA engine) issued by thread 0; two stage buffers
//     alternate, so the copy of tile j drains while tile j + 1 is contracted.
// The compute warps meet at a named barrier once per tile; all warps meet once
// per batch.  No spin-waits (the copy engine is waited on with its group-wait
// instruction).
#pragma once
#include "common.cuh"
#include "pre_stream.cuh"
#include "pre_vec.cuh"
#include "sym.cuh"

namespace fea {

__device__ __forceinline__ void bar_sync_named(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
// shared -> global bulk copy (16-byte aligned addresses, size % 16 == 0)
__device__ __forceinline__ void bulk_s2g(void* dst, const void* src, unsigned bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_addr(src)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

template <int P>
struct PreVecStream {
  static constexpr int NS = nbasis_c(P);
  static constexpr int N = 3 * NS;
  static constexpr int NN = N * N;
  static constexpr int S = NS * NS;
  static constexpr int NP = NS * (NS + 1) / 2;
  static constexpr int NCOMP = NT - 32;          // compute threads (7 warps)
  static constexpr int TE = NCOMP / NP;          // element slots per tile
  static_assert(TE >= 1, "one element's pairs must fit the compute warps");
  static constexpr int B = (32 + TE - 1) / TE;   // tiles per geometry batch
  static constexpr int GEO = 32;
  static constexpr int MINB = 3;

  FEA_HD static int max_tile() { return TE; }
  FEA_HD static int pref_tile() { return TE; }
  FEA_HD static size_t stage_bytes(int te) { return round_up_sz((size_t)te * NN * 8, 128); }
  FEA_HD static size_t off_geo(int te) { return 2 * stage_bytes(te); }
  FEA_HD static size_t smem(int te, int Q) { (void)Q; return off_geo(te) + round_up_sz((size_t)2 * B * te * GEO * 4, 16); }
};

template <int P>
__global__ void __launch_bounds__(NT, PreVecStream<P>::MINB) pre_vec_stream_kernel(Req q, unsigned* err) {
  using K = PreVecStream<P>;
  extern __shared__ __align__(128) char sm[];
  const int TE = q.tile;
  {
    unsigned dyn;
    asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
    if (TE < 1 || TE > K::TE || K::smem(TE, q.Q) > dyn) {  // refuse a tile the layout or the launch cannot hold
      if (threadIdx.x == 0) flag_error(err, 4u);
      return;
    }
  }
  const int64_t ntiles = (q.E + TE - 1) / TE;
  const int64_t first = blockIdx.x;
  if (first >= ntiles) return;
  const int64_t stride = gridDim.x;
  const int my_tiles = (int)((ntiles - first + stride - 1) / stride);
  const int nbatch = (my_tiles + K::B - 1) / K::B;
  const size_t SB = K::stage_bytes(TE);
  const unsigned esz = q.out_f32 ? 4u : 8u;
  char* stage = sm;                                                     // [2][SB]
  float* geo = reinterpret_cast<float*>(sm + K::off_geo(TE));           // [2][B * TE][GEO]

  const int t = threadIdx.x, lane = t & 31;
  auto tile_e0 = [&](int j) { return (first + (int64_t)j * stride) * TE; };
  auto tile_ne = [&](int j) {
    const int64_t e0 = tile_e0(j);
    return (int)(q.E - e0 < TE ? q.E - e0 : TE);
  };
  // producer: FP64 geometry of batch k (tiles k B .. k B + B - 1) into record buffer k & 1
  auto records = [&](int k) {
    for (int m = lane; m < K::B * TE; m += 32) {
      const int j = k * K::B + m / TE, s = m - (m / TE) * TE;
      if (j < my_tiles && s < tile_ne(j)) {
        const int64_t e = tile_e0(j) + s;
        double x[12], c[8];
#pragma unroll
        for (int i = 0; i < 6; ++i) {
          const double2 v = __ldg(reinterpret_cast<const double2*>(q.coords + e * 12) + i);
          x[2 * i] = v.x;
          x[2 * i + 1] = v.y;
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const double2 v = __ldg(reinterpret_cast<const double2*>(q.coeffs + e * 8) + i);
          c[2 * i] = v.x;
          c[2 * i + 1] = v.y;
        }
        pre_vec_record<float>(x, c, geo + ((size_t)(k & 1) * K::B * TE + m) * K::GEO, err);
      }
    }
  };

  if (t >= K::NCOMP) {  // ------------------------------------------------ producer warp
    records(0);
    __syncthreads();
    for (int k = 0; k < nbatch; ++k) {
      if (k + 1 < nbatch) records(k + 1);  // buffer (k + 1) & 1 was last read in batch k - 1
      __syncthreads();
    }
    return;
  }
  // ------------------------------------------------------------------------ compute warps
  const bool comp = t < TE * K::NP;
  const int slot = t / K::NP, pk = t - slot * K::NP;
  int a = 0, b = 0;
  float R[36];
  if (comp) {
    const unsigned ab = kSymPairs<K::NS>.c[pk];
    a = (int)(ab & 0xffu);
    b = (int)(ab >> 8);
    const TabLayout L = tab_layout(q.Q, K::NS, 36);
    const float* Rg = reinterpret_cast<const float*>(q.tab) + L.offR;  // [(k,al,be)][a][b]
#pragma unroll
    for (int r = 0; r < 36; ++r) R[r] = __ldg(Rg + (size_t)r * K::S + a * K::NS + b);
  }
  __syncthreads();  // batch 0 records
  for (int j = 0; j < my_tiles; ++j) {
    const int64_t e0 = tile_e0(j);
    const int ne = tile_ne(j);
    const int buf = j & 1;
    const int k = j / K::B;
    if (comp && slot < ne) {
      const float* g = geo + ((size_t)(k & 1) * K::B * TE + (j - k * K::B) * TE + slot) * K::GEO;
      float v[9];
      pre_vec_block<float>(g, R, v);
      if (q.out_f32) {
        put_sym_block<K::N, float>(reinterpret_cast<float*>(stage + buf * SB) + (size_t)slot * K::NN, a, b, v);
      } else {
        const bool bad = g[26] != g[26];
        double d[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) d[i] = bad ? __longlong_as_double(0x7ff8000000000000ll) : f2d_finite(v[i]);
        put_sym_block<K::N, double>(reinterpret_cast<double*>(stage + buf * SB) + (size_t)slot * K::NN, a, b, d);
      }
      fence_proxy_async();  // the stage is read by the bulk copy (async proxy)
    }
    if (t == 0) bulk_wait_read_0();  // tile j - 1's copy has read the other stage buffer
    bar_sync_named(1, K::NCOMP);
    if (t == 0) {
      bulk_s2g(reinterpret_cast<char*>(q.out) + (size_t)e0 * K::NN * esz, stage + buf * SB, (unsigned)ne * K::NN * esz);
      bulk_commit();
    }
    if (j % K::B == K::B - 1 || j == my_tiles - 1) __syncthreads();  // next batch's records are ready
  }
  if (t == 0) bulk_wait_0();
}

}  // namespace fea
