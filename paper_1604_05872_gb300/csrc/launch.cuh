// Persistent tile loop shared by every standalone kernel.
#pragma once
#include "common.cuh"
#include "kernels.h"

#include <type_traits>

namespace fea {

__device__ __forceinline__ unsigned dynamic_smem_bytes() {
  unsigned r;
  asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(r));
  return r;
}
constexpr unsigned ERR_LAUNCH = 4u;

// Tile functions that need a given number of resident CTAs per SM (register
// budget) say so with a MINB constant.
template <class K, class = void>
struct MinBlocksOf { static constexpr int value = 1; };
template <class K>
struct MinBlocksOf<K, std::void_t<decltype(K::MINB)>> { static constexpr int value = K::MINB; };

template <class K>
__global__ void __launch_bounds__(NT, MinBlocksOf<K>::value) run_tiles(Req q, unsigned* err) {
  extern __shared__ __align__(16) char smem_raw[];
  // a tile larger than the shared memory it was launched with is refused, not run
  if (K::smem(q.tile, q.Q) > dynamic_smem_bytes()) {
    if (threadIdx.x == 0) flag_error(err, ERR_LAUNCH);
    return;
  }
  const int64_t ntiles = (q.E + q.tile - 1) / q.tile;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t e0 = t * q.tile;
    const int64_t left = q.E - e0;
    const int ne = (int)(left < q.tile ? left : q.tile);
    K::tile(q, e0, ne, smem_raw, err);
  }
}

template <class K>
size_t smem_of(int TE, int Q) { return K::smem(TE, Q); }

// Tile functions whose thread layout is built for a given tile say so with
// pref_tile(); the others take the planner's shared-memory rule.
template <class K, class = void>
struct PrefTile { static int get() { return 0; } };
template <class K>
struct PrefTile<K, std::void_t<decltype(K::pref_tile())>> { static int get() { return K::pref_tile(); } };

template <class K>
KernelInfo make_info(int variant, int form, int p, int prec) {
  return KernelInfo{reinterpret_cast<const void*>(&run_tiles<K>), variant, form, p, prec, K::max_tile(), &smem_of<K>,
                    PrefTile<K>::get()};
}

}  // namespace fea
