// Tensor-core kernels of the split-operand precision (FEA_PREC_BF16X2) and the
// device tables they read: the Neo-Hookean tangent at P2 (shared reference
// operand, nh_tc.cuh) and at P3 (one product per element, nh_tce.cuh), and the
// pre-evaluated mass and Helmholtz matrices at P1-P2 with FP32 output
// (pre_tc.cuh).
#include <cstring>
#include <vector>

#include "host_model.h"
#include "launch.cuh"
#include "nh_tc.cuh"
#include "nh_tce.cuh"
#include "pre_tc.cuh"

namespace fea {

template <int P>
size_t nh_tc_smem(int, int) { return NhTc<P>::SMEM; }
template <int P>
size_t nh_tce_smem(int, int) { return NhTcE<P>::SMEM; }
template <int F, int P>
size_t pre_tc_smem(int, int) { return PreTc<F, P>::SMEM; }
#define PRETC(F, P)                                                                                            \
  KernelInfo { reinterpret_cast<const void*>(&pre_tc_kernel<F, P>), V_PRE, F, P, 2, PreTc<F, P>::TE,          \
               &pre_tc_smem<F, P>, PreTc<F, P>::TE, PreTc<F, P>::NTH, false }

const KernelInfo kTcKernels[] = {
    KernelInfo{reinterpret_cast<const void*>(&nh_tc_kernel<2>), V_SE, NEOHOOKEAN, 2, 2, NhTc<2>::TE, &nh_tc_smem<2>,
               NhTc<2>::TE, NhTc<2>::NTH, true},
    KernelInfo{reinterpret_cast<const void*>(&nh_tce_kernel<3>), V_SE, NEOHOOKEAN, 3, 2, NhTcE<3>::TE, &nh_tce_smem<3>,
               NhTcE<3>::TE, NhTcE<3>::NTH, true},
    PRETC(0, 1), PRETC(0, 2), PRETC(1, 1), PRETC(1, 2),
};
#undef PRETC
const int kNumTcKernels = sizeof(kTcKernels) / sizeof(kTcKernels[0]);

const KernelInfo* find_tc_kernel(int form, int p) {
  for (int i = 0; i < kNumTcKernels; ++i)
    if (kTcKernels[i].form == form && kTcKernels[i].p == p) return &kTcKernels[i];
  return nullptr;
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
static uint32_t fbits(double x) {
  const float f = (float)x;
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return u;
}

template <int P>
static void nh_tc_table(std::vector<uint32_t>* words) {
  using C = NhTc<P>;
  const Tables t = make_tables(NEOHOOKEAN, P);
  const TcTabLayout L = tc_tab_layout(C::Q, C::NS, C::K);
  words->assign((size_t)L.total, 0u);
  uint32_t* w = words->data();
  for (int q = 0; q < C::Q; ++q) w[L.offW + q] = fbits(t.W[q]);
  for (int i = 0; i < C::Q * C::NS * 3; ++i) w[L.offDphi + i] = fbits(t.dphi[i]);
  // R_(a,b)[kk] = dPhi_a^k(X_q) dPhi_b^l(X_q) for q < Q, and for q = Q the point sum
  // sum_q w_q dPhi_a^k(X_q) dPhi_b^l(X_q), at kk = kk_of(q, 3 k + l) (points interleaved in pairs);
  // split into BF16 hi and lo
  auto g = [&](int q, int a, int k) { return t.dphi[((size_t)q * C::NS + a) * 3 + k]; };
  for (int pr = 0; pr < C::NPAIR; ++pr) {
    int a = 0, b = 0;
    sym_pair(pr, C::NS, &a, &b);
    uint32_t* hi = w + L.offR + (size_t)(2 * pr) * (C::K / 2);
    uint32_t* lo = hi + C::K / 2;
    for (int q = 0; q <= C::Q; ++q) {
      for (int kl = 0; kl < 9; ++kl) {
        const int kk = C::kk_of(q, kl), k = kl / 3, l = kl % 3;
        double r = 0.0;
        if (q < C::Q) {
          r = g(q, a, k) * g(q, b, l);
        } else {
          for (int p = 0; p < C::Q; ++p) r += t.W[p] * g(p, a, k) * g(p, b, l);
        }
        const uint16_t h = bf16_rn((float)r);
        const uint16_t s = bf16_rn((float)(r - (double)bf16_val(h)));
        const int sh = (kk & 1) ? 16 : 0;  // element 2j in the low half of column j
        hi[kk >> 1] |= (uint32_t)h << sh;
        lo[kk >> 1] |= (uint32_t)s << sh;
      }
    }
  }
}

// W, dPhi and the symmetric point-summed tables Rbar_s[(a, b)][i] of the
// per-element kernel: for (k, l) = (0,0), (0,1), (0,2), (1,1), (1,2), (2,2),
// Rbar^kk and Rbar^kl + Rbar^lk with Rbar_ab^kl = sum_q w_q dPhi_a^k dPhi_b^l.
template <int P>
static void nh_tce_table(std::vector<uint32_t>* words) {
  using C = NhTcE<P>;
  const Tables t = make_tables(NEOHOOKEAN, P);
  const TcETabLayout L = tce_tab_layout(C::Q, C::NS);
  words->assign((size_t)L.total, 0u);
  uint32_t* w = words->data();
  for (int q = 0; q < C::Q; ++q) w[L.offW + q] = fbits(t.W[q]);
  for (int i = 0; i < C::Q * C::NS * 3; ++i) w[L.offDphi + i] = fbits(t.dphi[i]);
  auto g = [&](int q, int a, int k) { return t.dphi[((size_t)q * C::NS + a) * 3 + k]; };
  for (int a = 0; a < C::NS; ++a)
    for (int b = 0; b < C::NS; ++b) {
      int i6 = 0;
      for (int k = 0; k < 3; ++k)
        for (int l = k; l < 3; ++l, ++i6) {
          double r = 0.0;
          for (int q = 0; q < C::Q; ++q) {
            r += t.W[q] * g(q, a, k) * g(q, b, l);
            if (l != k) r += t.W[q] * g(q, a, l) * g(q, b, k);
          }
          w[L.offRbar + 6 * (a * C::NS + b) + i6] = fbits(r);
        }
    }
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

// Device-table words of the tensor-core kernel of (form, p); false if there is none.
bool tc_table_words(int form, int p, std::vector<uint32_t>* words) {
  if (form == MASS && p == 1) return pre_tc_table<0, 1>(words), true;
  if (form == MASS && p == 2) return pre_tc_table<0, 2>(words), true;
  if (form == HELMHOLTZ && p == 1) return pre_tc_table<1, 1>(words), true;
  if (form == HELMHOLTZ && p == 2) return pre_tc_table<1, 2>(words), true;
  if (form == NEOHOOKEAN && p == 2) {
    nh_tc_table<2>(words);
    return true;
  }
  if (form == NEOHOOKEAN && p == 3) {
    nh_tce_table<3>(words);
    return true;
  }
  return false;
}

}  // namespace fea
