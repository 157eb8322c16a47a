// Instantiations of the element-vector kernels (linear forms; P1-P4; FP32 and FP64).
#include <algorithm>

#include "../../include/fea.h"
#include "launch.cuh"
#include "pre_stream.cuh"
#include "vec_forms.cuh"

namespace fea {

// the streaming load-vector kernel (P1-P3, FP32) ahead of the tile kernel it replaces
template <int P>
size_t load_stream_smem(int TE, int Q) { return PreStreamLoad<P>::smem(TE, Q); }
template <int P>
KernelInfo load_stream_info() {
  return KernelInfo{reinterpret_cast<const void*>(&pre_stream_load_kernel<P>), V_PRE, 1, P, 1, NT, &load_stream_smem<P>,
                    128};
}
#define LV(P) make_info<LoadVecTile<P, float>>(V_PRE, 1, P, 1), make_info<LoadVecTile<P, double>>(V_PRE, 1, P, 0)
#define LVS(P) load_stream_info<P>(), LV(P)
#define RV(P) make_info<ResVecTile<P, float>>(V_SE, 3, P, 1), make_info<ResVecTile<P, double>>(V_SE, 3, P, 0)
const KernelInfo kVecKernels[] = {LVS(1), LVS(2), LVS(3), LV(4), RV(1), RV(2), RV(3), RV(4)};
#undef LV
#undef LVS
#undef RV
const int kNumVecKernels = sizeof(kVecKernels) / sizeof(kVecKernels[0]);

const KernelInfo* find_vec_kernel(int form, int p, int prec) {
  for (int i = 0; i < kNumVecKernels; ++i)
    if (kVecKernels[i].form == form && kVecKernels[i].p == p && kVecKernels[i].prec == prec) return &kVecKernels[i];
  return nullptr;
}

}  // namespace fea

// ----------------------------------------------------------------------------
// The kernels' FP64 logarithm (log_f64.cuh) over an array, for its accuracy
// tests against the hardware library and the host.
namespace fea {

__global__ void __launch_bounds__(256) log_f64_kernel(const double* __restrict__ x, double* __restrict__ y, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = log_f64(__ldg(x + i));
}

int set_error(int code, const char* msg);
int check_device_ptr(const void* p, const char* what, bool allow_null);

}  // namespace fea

extern "C" int fea_log_f64(const double* x, double* y, int64_t n, void* stream) {
  if (n < 0) return fea::set_error(FEA_EINVAL, "negative length");
  if (n == 0) return FEA_OK;
  int rc;
  if ((rc = fea::check_device_ptr(x, "x", false))) return rc;
  if ((rc = fea::check_device_ptr(y, "y", false))) return rc;
  const int64_t grid = std::min<int64_t>((n + 255) / 256, 152 * 8);  // grid-stride: any grid covers n
  fea::log_f64_kernel<<<(unsigned)grid, 256, 0, (cudaStream_t)stream>>>(x, y, n);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fea::set_error(FEA_ECUDA, cudaGetErrorString(e));
  return FEA_OK;
}
