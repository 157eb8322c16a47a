// Instantiations of the pre-evaluated variant (mass, Helmholtz, elasticity; P1-P4; FP32 and FP64).
#include "launch.cuh"
#include "pre.cuh"

namespace fea {

#define PRE(F, P) make_info<PreTile<F, P, float>>(V_PRE, F, P, 1), make_info<PreTile<F, P, double>>(V_PRE, F, P, 0)
const KernelInfo kPreKernels[] = {
    PRE(0, 1), PRE(0, 2), PRE(0, 3), PRE(0, 4),
    PRE(1, 1), PRE(1, 2), PRE(1, 3), PRE(1, 4),
    PRE(2, 1), PRE(2, 2), PRE(2, 3), PRE(2, 4),
};
#undef PRE
const int kNumPreKernels = sizeof(kPreKernels) / sizeof(kPreKernels[0]);

}  // namespace fea
