// Instantiations of the element-vector kernels (linear forms; P1-P4; FP32 and FP64).
#include "launch.cuh"
#include "vec_forms.cuh"

namespace fea {

#define LV(P) make_info<LoadVecTile<P, float>>(V_PRE, 1, P, 1), make_info<LoadVecTile<P, double>>(V_PRE, 1, P, 0)
#define RV(P) make_info<ResVecTile<P, float>>(V_SE, 3, P, 1), make_info<ResVecTile<P, double>>(V_SE, 3, P, 0)
const KernelInfo kVecKernels[] = {LV(1), LV(2), LV(3), LV(4), RV(1), RV(2), RV(3), RV(4)};
#undef LV
#undef RV
const int kNumVecKernels = sizeof(kVecKernels) / sizeof(kVecKernels[0]);

const KernelInfo* find_vec_kernel(int form, int p, int prec) {
  for (int i = 0; i < kNumVecKernels; ++i)
    if (kVecKernels[i].form == form && kVecKernels[i].p == p && kVecKernels[i].prec == prec) return &kVecKernels[i];
  return nullptr;
}

}  // namespace fea
