// The split-BF16 tensor-core kernel of the pre-evaluated mass and Helmholtz
// matrices (P1, P2; FP32 output), its registration and its device table.
#include <cstring>
#include <vector>

#include "host_model.h"
#include "launch.cuh"
#include "pre_tc.cuh"

namespace fea {

template <int F, int P>
size_t pre_tc_smem(int, int) { return PreTc<F, P>::SMEM; }
#define PRETC(F, P)                                                                                            \
  KernelInfo { reinterpret_cast<const void*>(&pre_tc_kernel<F, P>), V_PRE, F, P, 2, PreTc<F, P>::TE,          \
               &pre_tc_smem<F, P>, PreTc<F, P>::TE, PreTc<F, P>::NTH, false }
const KernelInfo kPreTcKernels[] = {PRETC(0, 1), PRETC(0, 2), PRETC(1, 1), PRETC(1, 2)};
#undef PRETC

// The kernel of (form, p), or nullptr.
const KernelInfo* find_pretc_kernel(int form, int p) {
  for (const KernelInfo& k : kPreTcKernels)
    if (k.form == form && k.p == p) return &k;
  return nullptr;
}

// Two CTAs per SM: their accumulators (256 tensor-memory columns each) fill the SM's 512.
bool is_pretc_kernel(const void* fn) {
  for (const KernelInfo& k : kPreTcKernels)
    if (k.fn == fn) return true;
  return false;
}

// bfloat16 from float, round to nearest even (NaN stays NaN).
static uint16_t bf16_rn(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7fffffffu) > 0x7f800000u) return 0x7fc0u;
  u += 0x7fffu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}
static float bf16_val(uint16_t h) {
  const uint32_t u = (uint32_t)h << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}

// The pre-evaluated reference tensors R_r[i][j] as the B operand of pre_tc_kernel:
// row (i, j), K = r, three BF16 parts (the FP32 value rounded, then each remainder
// rounded), part after part, in the K-major shared-memory layout the kernel
// copies as it is.
template <int F, int P>
static void pre_tc_table(std::vector<uint32_t>* words) {
  using C = PreTc<F, P>;
  const Tables t = make_tables(F, P);
  words->assign((size_t)3 * C::TABLE_WORDS, 0u);
  const int ns = C::K::NS;
  for (int r = 0; r < C::K::R; ++r)
    for (int n = 0; n < C::K::NN; ++n) {
      float rem = (float)t.R[(size_t)r * ns * ns + n];
      const uint32_t off = C::kmajor_off(n, r);
      const int sh = (off & 2u) ? 16 : 0;
      for (int part = 0; part < 3; ++part) {
        const uint16_t b = bf16_rn(rem);
        (*words)[(size_t)part * C::TABLE_WORDS + (off >> 2)] |= (uint32_t)b << sh;
        rem -= bf16_val(b);
      }
    }
}

// Device-table words of pre_tc_kernel for (form, p); false if there is none.
bool pretc_table_words(int form, int p, std::vector<uint32_t>* words) {
  if (form == MASS && p == 1) return pre_tc_table<0, 1>(words), true;
  if (form == MASS && p == 2) return pre_tc_table<0, 2>(words), true;
  if (form == HELMHOLTZ && p == 1) return pre_tc_table<1, 1>(words), true;
  if (form == HELMHOLTZ && p == 2) return pre_tc_table<1, 2>(words), true;
  return false;
}

}  // namespace fea
