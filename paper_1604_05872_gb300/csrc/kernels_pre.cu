// Instantiations of the pre-evaluated variant (mass, Helmholtz, elasticity; P1-P4; FP32 and FP64).
#include <algorithm>

#include "launch.cuh"
#include "pre.cuh"
#include "pre_combine.cuh"
#include "pre_stream.cuh"
#include "pre_vec.cuh"
#include "pre_vec_stream.cuh"

namespace fea {

template <int F, int P>
size_t stream_smem(int TE, int Q) { return PreStream<F, P>::smem(TE, Q); }
template <int F, int P>
KernelInfo stream_info() {
  return KernelInfo{reinterpret_cast<const void*>(&pre_stream_kernel<F, P>), V_PRE, F, P, 1, NT, &stream_smem<F, P>, 0};
}

template <class Pol>
size_t batched_smem(int TE, int Q) { return StreamLayout<Pol>::smem(TE, Q); }
template <class Pol>
KernelInfo batched_info(int variant, int form, int p) {
  return KernelInfo{reinterpret_cast<const void*>(&stream_batched_kernel<Pol>), variant, form, p, 1, Pol::TE,
                    &batched_smem<Pol>, Pol::TE};
}

#define PRE(F, P) make_info<PreTile<F, P, float>>(V_PRE, F, P, 1), make_info<PreTile<F, P, double>>(V_PRE, F, P, 0)
#define PRES(F, P) stream_info<F, P>(), make_info<PreTile<F, P, double>>(V_PRE, F, P, 0)
#define PREV(P) make_info<PreVecTile<P, float>>(V_PRE, 2, P, 1), make_info<PreVecTile<P, double>>(V_PRE, 2, P, 0)
#define PREVS(P) batched_info<VecStreamPolicy<P>>(V_PRE, 2, P), make_info<PreVecTile<P, float>>(V_PRE, 2, P, 1), make_info<PreVecTile<P, double>>(V_PRE, 2, P, 0)
const KernelInfo kPreKernels[] = {
    PRES(0, 1), PRES(0, 2), PRES(0, 3), PRE(0, 4),
    PRES(1, 1), PRES(1, 2), PRES(1, 3), PRE(1, 4),
    PREVS(1), PREVS(2), PREVS(3), PREV(4),
};
#undef PRE
#undef PRES
#undef PREV
#undef PREVS
const int kNumPreKernels = sizeof(kPreKernels) / sizeof(kPreKernels[0]);

// Local and global assembly in one pass (the streaming kernel adding into CSR
// values): the plain streaming kernel it replaces and its int32 / int64 map forms.
struct ScatterKernel {
  int form, p;
  const void* plain;
  const void* map32;
  const void* map64;
};
#define SCAT(F, P)                                                                                      \
  ScatterKernel{F, P, reinterpret_cast<const void*>(&pre_stream_kernel<F, P>),                          \
                reinterpret_cast<const void*>(&pre_stream_scatter_kernel<F, P, 4>),                     \
                reinterpret_cast<const void*>(&pre_stream_scatter_kernel<F, P, 8>)}
const ScatterKernel kScatterKernels[] = {SCAT(0, 1), SCAT(0, 2), SCAT(0, 3), SCAT(1, 1), SCAT(1, 2), SCAT(1, 3)};
#undef SCAT

const void* find_scatter_kernel(const void* plain, int map_i64) {
  for (const ScatterKernel& k : kScatterKernels)
    if (k.plain == plain) return map_i64 ? k.map64 : k.map32;
  return nullptr;
}

// One-pass assembly with the entries of a tile combined per CSR position.
int combine_tile(int n) { return std::min(128, std::max(2, (3200 / (n * n)) & ~1)); }

struct CombineKernel {
  int form, p;
  const void* fn;
  size_t (*smem)(int TE);
};
template <int F, int P>
size_t combine_smem(int TE) { return PreCombine<F, P>::smem(TE); }
#define COMB(F, P) CombineKernel{F, P, reinterpret_cast<const void*>(&pre_combine_kernel<F, P>), &combine_smem<F, P>}
const CombineKernel kCombineKernels[] = {COMB(0, 1), COMB(0, 2), COMB(0, 3), COMB(1, 1), COMB(1, 2), COMB(1, 3)};
#undef COMB

const void* find_combine_kernel(int form, int p, size_t* smem) {
  for (const CombineKernel& k : kCombineKernels)
    if (k.form == form && k.p == p) {
      *smem = k.smem(combine_tile(nbasis_c(p)));
      return k.fn;
    }
  return nullptr;
}

// The FP32 tile functions the batched kernel dispatches to (their shared-memory
// layouts and tile limits plan the batch).
#define PT(F, P) make_info<PreTile<F, P, float>>(V_PRE, F, P, 1)
#define PTV(P) make_info<PreVecTile<P, float>>(V_PRE, 2, P, 1)
const KernelInfo kPreTileF32[] = {PT(0, 1), PT(0, 2), PT(0, 3), PT(0, 4), PT(1, 1), PT(1, 2),
                                  PT(1, 3), PT(1, 4), PTV(1), PTV(2), PTV(3), PTV(4)};
#undef PTV
#undef PT
const int kNumPreTileF32 = sizeof(kPreTileF32) / sizeof(kPreTileF32[0]);

}  // namespace fea
