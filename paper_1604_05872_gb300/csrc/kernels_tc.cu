// Tensor-core kernels of the split-operand precision (FEA_PREC_BF16X2) and the
// device tables they read: the Neo-Hookean tangent at P2 (shared reference
// operand, nh_tc.cuh) and at P3 (one product per element, nh_tce.cuh).
#include <cstring>
#include <vector>

#include "host_model.h"
#include "launch.cuh"
#include "nh_tc.cuh"
#include "nh_tce.cuh"

namespace fea {

template <int P>
size_t nh_tc_smem(int, int) { return NhTc<P>::SMEM; }
template <int P>
size_t nh_tce_smem(int, int) { return NhTcE<P>::SMEM; }

const KernelInfo kTcKernels[] = {
    KernelInfo{reinterpret_cast<const void*>(&nh_tc_kernel<2>), V_SE, NEOHOOKEAN, 2, 2, NhTc<2>::TE, &nh_tc_smem<2>,
               NhTc<2>::TE, NhTc<2>::NTH, true},
    KernelInfo{reinterpret_cast<const void*>(&nh_tce_kernel<3>), V_SE, NEOHOOKEAN, 3, 2, NhTcE<3>::TE, &nh_tce_smem<3>,
               NhTcE<3>::TE, NhTcE<3>::NTH, true},
};
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

// Device-table words of the tensor-core kernel of (form, p); false if there is none.
bool tc_table_words(int form, int p, std::vector<uint32_t>* words) {
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
