// Batched streaming schedule of the pre-evaluated FP32 elasticity kernel
// (P1-P3; an HBM-bound store stream of 1.3-29 KB per element):
//   * persistent CTAs; 7 compute warps keep their slice of the reference
//     tensors R in registers for the whole launch;
//   * the 8th warp is the producer: it reads the inputs of the next batch of
//     tiles (at least 32 elements, one per lane) and evaluates their FP64
//     geometry into per-element records in shared memory -- an FP64
//     instruction holds the SM's FP64 unit for the whole warp whatever its
//     active lanes, so the geometry runs on full warps, off the compute path;
//   * every tile's element matrices (one contiguous output range) are staged in
//     shared memory and leave it by one bulk asynchronous copy (cp.async.bulk,
//     the TMA engine) issued by thread 0; two stage buffers alternate, so the
//     copy of tile j drains while tile j + 1 is contracted.
// The compute warps meet at a named barrier once per tile, all warps once per
// batch.  There are no spin-waits (the copy engine is waited on with its
// group-wait instruction).
//
// A policy supplies the arithmetic: its element count per tile TE, the record
// size GEO (floats), record(inputs -> record), and a per-thread Thread object
// whose tile() writes its share of a tile's matrices into the stage.  (The
// scalar forms keep PreStream: their 0.1-3 KB matrices go out faster as direct
// 16-byte stores from registers than through a stage.)
#pragma once
#include "common.cuh"
#include "pre_stream.cuh"

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

constexpr int kStreamCompute = NT - 32;  // compute threads (7 warps); the last warp produces

// Shared-memory layout of the schedule for a policy.
template <class Pol>
struct StreamLayout {
  static constexpr int B = (32 + Pol::TE - 1) / Pol::TE;  // tiles per geometry batch
  FEA_HD static size_t stage_bytes(int te) { return round_up_sz((size_t)te * Pol::NN * 8, 128); }
  FEA_HD static size_t off_geo(int te) { return 2 * stage_bytes(te); }
  FEA_HD static size_t smem(int te, int Q) {
    (void)Q;
    return off_geo(te) + round_up_sz((size_t)2 * B * te * Pol::GEO * 4, 16);
  }
};

template <class Pol>
__global__ void __launch_bounds__(NT, Pol::MINB) stream_batched_kernel(Req q, unsigned* err) {
  using Lay = StreamLayout<Pol>;
  constexpr int B = Lay::B;
  extern __shared__ __align__(128) char sm[];
  const int TE = q.tile;
  {
    unsigned dyn;
    asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
    if (TE < 1 || TE > Pol::TE || Lay::smem(TE, q.Q) > dyn) {  // refuse a tile the layout or the launch cannot hold
      if (threadIdx.x == 0) flag_error(err, 4u);
      return;
    }
  }
  const int64_t ntiles = (q.E + TE - 1) / TE;
  const int64_t first = blockIdx.x;
  if (first >= ntiles) return;
  const int64_t stride = gridDim.x;
  const int my_tiles = (int)((ntiles - first + stride - 1) / stride);
  const int nbatch = (my_tiles + B - 1) / B;
  const size_t SB = Lay::stage_bytes(TE);
  const unsigned esz = q.out_f32 ? 4u : 8u;
  char* stage = sm;                                                 // [2][SB]
  float* geo = reinterpret_cast<float*>(sm + Lay::off_geo(TE));     // [2][B * TE][GEO]

  const int t = threadIdx.x, lane = t & 31;
  auto tile_e0 = [&](int j) { return (first + (int64_t)j * stride) * TE; };
  auto tile_ne = [&](int j) {
    const int64_t e0 = tile_e0(j);
    return (int)(q.E - e0 < TE ? q.E - e0 : TE);
  };

  if (t >= kStreamCompute) {  // -------------------------------------------- producer warp
    // records of batch k (tiles k B .. k B + B - 1) into record buffer k & 1
    auto records = [&](int k) {
      for (int m = lane; m < B * TE; m += 32) {
        const int j = k * B + m / TE, s = m - (m / TE) * TE;
        if (j < my_tiles && s < tile_ne(j))
          Pol::record(q, tile_e0(j) + s, geo + ((size_t)(k & 1) * B * TE + m) * Pol::GEO, err);
      }
    };
    records(0);
    __syncthreads();
    for (int k = 0; k < nbatch; ++k) {
      if (k + 1 < nbatch) records(k + 1);  // buffer (k + 1) & 1 was last read in batch k - 1
      __syncthreads();
    }
    return;
  }
  // --------------------------------------------------------------------------- compute warps
  typename Pol::Thread th(q, t);
  __syncthreads();  // batch 0 records
  for (int j = 0; j < my_tiles; ++j) {
    const int64_t e0 = tile_e0(j);
    const int ne = tile_ne(j);
    const int buf = j & 1;
    const int k = j / B;
    const float* g = geo + ((size_t)(k & 1) * B * TE + (size_t)(j - k * B) * TE) * Pol::GEO;
    if (th.tile(g, ne, stage + buf * SB, q.out_f32)) fence_proxy_async();  // the stage is read by the async proxy
    if (t == 0) bulk_wait_read_0();  // tile j - 1's copy has read the other stage buffer
    bar_sync_named(1, kStreamCompute);
    if (t == 0) {
      bulk_s2g(reinterpret_cast<char*>(q.out) + (size_t)e0 * Pol::NN * esz, stage + buf * SB, (unsigned)ne * Pol::NN * esz);
      bulk_commit();
    }
    if (j % B == B - 1 || j == my_tiles - 1) __syncthreads();  // next batch's records are ready
  }
  if (t == 0) bulk_wait_0();
}

}  // namespace fea
