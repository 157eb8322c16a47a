// Instantiations of the sharing-elimination variant (all forms; P1-P4; FP32 and FP64).
#include "launch.cuh"
#include "se.cuh"
#include "se_vec.cuh"

namespace fea {

#define SE(F, P) make_info<SeTile<F, P, float>>(V_SE, F, P, 1), make_info<SeTile<F, P, double>>(V_SE, F, P, 0)
#define SEV(F, P) make_info<SeVecTile<F, P, float>>(V_SE, F, P, 1), make_info<SeVecTile<F, P, double>>(V_SE, F, P, 0)
const KernelInfo kSeKernels[] = {
    SE(0, 1), SE(0, 2), SE(0, 3), SE(0, 4),
    SE(1, 1), SE(1, 2), SE(1, 3), SE(1, 4),
    SEV(2, 1), SEV(2, 2), SEV(2, 3), SEV(2, 4),
    SEV(3, 1), SEV(3, 2), SEV(3, 3), SEV(3, 4),
};
#undef SE
#undef SEV
const int kNumSeKernels = sizeof(kSeKernels) / sizeof(kSeKernels[0]);

}  // namespace fea
