// Instantiations of the plain FP64 quadrature nest (the comparator; all forms, P1-P4).
#include "launch.cuh"
#include "naive.cuh"

namespace fea {

#define NV(F, P) make_info<NaiveTile<F, P>>(V_NAIVE, F, P, 0)
const KernelInfo kNaiveKernels[] = {
    NV(0, 1), NV(0, 2), NV(0, 3), NV(0, 4),
    NV(1, 1), NV(1, 2), NV(1, 3), NV(1, 4),
    NV(2, 1), NV(2, 2), NV(2, 3), NV(2, 4),
    NV(3, 1), NV(3, 2), NV(3, 3), NV(3, 4),
};
#undef NV
const int kNumNaiveKernels = sizeof(kNaiveKernels) / sizeof(kNaiveKernels[0]);

const KernelInfo* find_kernel(int variant, int form, int p, int prec, size_t budget, int Q) {
  const KernelInfo* tabs[3] = {kNaiveKernels, kSeKernels, kPreKernels};
  const int counts[3] = {kNumNaiveKernels, kNumSeKernels, kNumPreKernels};
  if (variant < 0 || variant > 2) return nullptr;
  const KernelInfo* any = nullptr;
  for (int i = 0; i < counts[variant]; ++i) {
    const KernelInfo& k = tabs[variant][i];
    if (k.form != form || k.p != p || k.prec != prec) continue;
    // the first registered kernel whose smallest tile fits the budget (Constraint 2)
    if (budget == 0 || k.smem(1, Q) <= budget) return &k;
    if (!any) any = &k;
  }
  return any;
}

}  // namespace fea

namespace fea {
const KernelInfo* find_batch_kernel(int variant, int form, int p) {
  if (variant == V_PRE) {
    for (int i = 0; i < kNumPreTileF32; ++i)
      if (kPreTileF32[i].form == form && kPreTileF32[i].p == p) return &kPreTileF32[i];
    return nullptr;
  }
  if (variant == V_SE) return find_kernel(V_SE, form, p, 1, 0, 0);
  return nullptr;
}
}  // namespace fea
