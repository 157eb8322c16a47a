// Persistent tile loop shared by every standalone kernel.
#pragma once
#include "common.cuh"
#include "kernels.h"

namespace fea {

template <class K>
__global__ void __launch_bounds__(NT) run_tiles(Req q, unsigned* err) {
  extern __shared__ __align__(16) char smem_raw[];
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

template <class K>
KernelInfo make_info(int variant, int form, int p, int prec) {
  return KernelInfo{reinterpret_cast<const void*>(&run_tiles<K>), variant, form, p, prec, K::max_tile(), &smem_of<K>};
}

}  // namespace fea
