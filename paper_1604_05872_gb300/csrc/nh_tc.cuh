// Neo-Hookean tangent stiffness on the tensor cores (tcgen05), split-BF16
// operands with FP32 accumulation.
//
// Per quadrature point the tangent's integrand factors through the reference
// gradients: with M_q = F^-T J^-T, K = J^-1 J^-T, s_q = w_q |det J| and
// alpha_q = mu - lam ln det F,
//
//   A[(a,c),(b,d)] = sum_q sum_{k,l} H_q[(c,d),(k,l)] dPhi_a^k(X_q) dPhi_b^l(X_q),
//   H_q[(c,d),(k,l)] = s alpha M[d][k] M[c][l] + s lam M[c][k] M[d][l] + delta_cd s mu K[k][l].
//
// This is the paper's pre-evaluation (Section 3.3, Algorithm 2) applied at each
// quadrature point instead of over the whole integral (the integrand is not a
// polynomial, so the point sum cannot be pre-evaluated): the reference tables
// R_(a,b)[(q,k,l)] = dPhi_a^k(X_q) dPhi_b^l(X_q) are built once on the host, and
// per element only the 9 x 9Q tensor H is formed.  The contraction over
// (q, k, l) is one dense product per tile of TE elements:
//
//   D[128 x 128] = R_stack[128 x K] * H_tile[128 x K]^T
//
// rows of D: row 2p holds the BF16 "hi" part of R for the pair p = (a, b),
// a <= b, row 2p + 1 the "lo" part (R - hi rounded to BF16); columns of D:
// (element, c, d) = 64 h + 9 e' + 3 c + d for the element e = 7 h + e' (each
// half tile of 7 elements in its own 64 columns, the last one unused).  H is split the same way and the two halves
// run as two MMAs into the same accumulator, so D[2p] + D[2p + 1] is the sum of
// all four products (hi + lo)(hi + lo) of the split operands, with FP32
// accumulation in tensor memory.  The tangent is symmetric: the pair p gives
// the 3 x 3 block (a, b) and, transposed, (b, a).
//
// The q-independent term delta_cd s mu K sums to mu |det J| K[k][l] times the
// point-summed table sum_q w_q dPhi_a^k dPhi_b^l: it enters as one extra
// "point" (9 more columns of K, in the padding of the MMA's K extent), so the
// per-point H carries only the two M M terms.
//
// Roles (one CTA per SM, persistent over tiles, 28 warps):
//   warp 0       allocates tensor memory; one lane issues the MMAs;
//   warps 1-3    geometry: tile inputs by bulk copy two tiles ahead, the
//                displacement DOFs to FP32, per element J, adj J and det J in
//                FP64, J^-1 and mu |det J| J^-1 J^-T in FP32;
//   warps 4-11   epilogue, two sets of four (one per half tile, each covering
//                the four lane quarters of tensor memory): accumulator ->
//                FP32 staging (both blocks of each pair) -> coalesced 16-byte
//                stores of the element matrices;
//   warps 12-19  kinematics, two groups of four taking alternate tiles: per
//                (element, point) grad u (FP32), then F = I + grad u, its
//                cofactors, det F and ln det F in FP64, M = F^-T J^-T, s, s alpha;
//   warps 20-27  build H, one row (e, c, d) per thread, two groups of four
//                taking half of the points each; split into BF16 hi/lo.
// R (128 rows x K/2 packed BF16 pairs) sits in tensor memory for the whole
// launch; D is double-buffered in tensor memory.  Tiles come from an atomic
// counter when the launch provides one (else CTA c takes c, c + grid, ...): the
// geometry leader draws them two iterations ahead into a ring in shared memory
// that every role reads after the wait that hands it the iteration; -1 past the
// last tile is passed from role to role.  Every mbarrier wait is
// bounded; a role that gives up sets the error word, the others then give up
// too, and the CTA waits for its copies and MMAs in flight before it frees the
// tensor memory and leaves.
#pragma once
#include "common.cuh"
#include "launch.cuh"
#include "log_f64.cuh"
#include "mbar.cuh"
#include "tc.cuh"

#include <cuda_bf16.h>

namespace fea {

template <int P>
struct NhTc {
  static constexpr int NS = nbasis_c(P);
  static constexpr int N3 = 3 * NS;
  static constexpr int NN = N3 * N3;
  static constexpr int CLEN = 3 * NS;
  static constexpr int NPAIR = NS * (NS + 1) / 2;
  static_assert(2 * NPAIR <= 128, "the split reference tables must fit one 128-row MMA tile");
  static constexpr int Q = (P + 1) * (P + 1) * (P + 1);  // collapsed rule, p + 1 points per direction
  static constexpr int TE = 14;                          // elements per tile: 9 TE <= 128 columns
  static constexpr int NCOL = 128;
  // K columns: the points q = 0 .. Q - 1 and the point-summed term as point Q, interleaved in pairs
  // so that the values of points 2 j and 2 j + 1 at the same (k, l) are neighbours (one packed pair)
  FEA_HD static constexpr int kk_of(int q, int kl) { return 18 * (q >> 1) + 2 * kl + (q & 1); }
  static constexpr int NPP = (Q + 2) / 2;                // point pairs, the point-summed term included
  static constexpr int KK = 18 * NPP;
  static constexpr int K = (KK + 15) / 16 * 16;
  static constexpr int KU = K / 8;          // 16-byte core-matrix columns along K
  static constexpr int KS = K / 16;         // MMA steps
  static constexpr int NG = (KU + 8) / 9;   // groups of 4 point pairs (9 core-matrix columns each)
  static_assert(4 * NG >= NPP && NG % 2 == 0, "point groups must cover the rule, two builder halves");
  static constexpr uint32_t LBO = 128, SBO = KU * 128;
  static constexpr int KSA = 9;  // K steps of the first builder group's half (core-matrix columns 0 .. 17)
  static_assert(2 * KSA == 2 * 9 && KSA < KS, "halves of K");
  static constexpr int HPART = NCOL * K * 2;  // bytes of one split part of H
  static constexpr int EH = TE / 2;           // elements of a tile per epilogue set
  static constexpr int ES = (EH + 1) / 2;     // elements staged at a time per set
  // pointwise data, per element and point pair (q, q + 1): (alpha_q, alpha_q+1), then
  // M'[c][k] = sqrt(s) M[c][k] for both points at 2 + 6 c + 2 k (+ 1): 20 floats; element records
  // padded so that neighbouring elements fall on other banks; per element mu |det J| K (9 floats).
  // Three slots (tile iteration % 3): a kinematics group never waits for the builders.
  static constexpr int PW_E = 20 * ((Q + 1) / 2) + 4;
  static constexpr int NPW = 3;
  static constexpr int NTH = 896;
  static constexpr int W_GEO = 1, W_EPI = 4, W_KIN = 12, W_BLD = 20;
  static constexpr int BAR_EPI = 1, BAR_KIN = 3, BAR_GEO = 5;  // epilogue sets 1, 2; kinematics groups 3, 4
  static constexpr uint32_t COL_R = 256, TMEM_COLS = 512;
  static_assert(COL_R + K / 2 <= TMEM_COLS, "tensor memory");

  static constexpr size_t O_HHI = 0, O_HLO = HPART;
  static constexpr size_t O_STAGE = 2 * (size_t)HPART;
  static constexpr size_t O_PW = O_STAGE + 2 * round_up_sz((size_t)ES * NN * 4, 16);
  static constexpr size_t PW_SLOT = (size_t)TE * PW_E * 4;
  static constexpr size_t O_PWK = O_PW + NPW * PW_SLOT;
  static constexpr size_t O_IN = O_PWK + round_up_sz(NPW * (size_t)TE * 9 * 4, 16);
  static constexpr size_t IN_BUF = (size_t)TE * (12 + CLEN) * 8;  // coords, then displacement DOFs
  static constexpr int RS = 36;  // floats per row of u and of dPhi: 16-byte loads of neighbouring rows hit other banks
  static constexpr int NGB = 3;                                      // geometry buffers (iteration % 3)
  static constexpr int RU = 32;                                      // floats per row of u
  static constexpr size_t O_UT = O_IN + 2 * IN_BUF;                  // per buffer: u as float [TE][RS]
  static constexpr size_t O_GEO = O_UT + NGB * (size_t)TE * RU * 4;  // per buffer: J^-1, |det J|, mu |det J| K [TE][24]
  static constexpr size_t O_W = O_GEO + NGB * (size_t)TE * 24 * 4;
  static constexpr size_t O_DPHI = O_W + round_up_sz((size_t)Q * 4, 16);  // [Q][RS]: dPhi_a^k at 3 a + k
  static constexpr size_t O_BAR = O_DPHI + (size_t)Q * RS * 4;
  static constexpr size_t SMEM = O_BAR + 256 + 128;  // + alignment of the base to 128 bytes
  static_assert(SMEM <= 232448, "shared memory per CTA");
  static_assert(O_IN % 16 == 0 && IN_BUF % 16 == 0 && (TE * 96) % 16 == 0, "bulk-copy alignment");
  static_assert(O_PW % 16 == 0 && (PW_E * 4) % 16 == 0 && O_PWK % 16 == 0 && O_UT % 16 == 0 && O_DPHI % 16 == 0,
                "vector alignment");
  static_assert(CLEN <= 32 && NS * 3 <= 32, "padded rows");
  static_assert(NS % 2 == 0, "node pairs");
  // rows of u and of dPhi at a point hold the nodes in pairs: entry 6 (a / 2) + 2 i + a % 2
  FEA_HD static constexpr int node_slot(int a, int i) { return 6 * (a >> 1) + 2 * i + (a & 1); }

  FEA_HD static int max_tile() { return TE; }
  FEA_HD static int pref_tile() { return TE; }
  FEA_HD static size_t smem(int, int) { return SMEM; }
};

struct NhTcBars {
  uint64_t in_full[2], geo_full[3], geo_empty[3], pw_full[3], pw_empty[3], h_full[2], h_empty[2], d_full[2],
      d_empty[2], done;
  uint32_t tbase;
};
// Tiles of the coming iterations (see the geometry role), in the barrier block's spare bytes.
constexpr int kNhTcRing = 16;
constexpr size_t kNhTcRingOff = 192;
static_assert(sizeof(NhTcBars) <= kNhTcRingOff && kNhTcRingOff + kNhTcRing * 4 <= 256, "tile ring");

// Elements EL0 .. EL0 + NEL - 1 of a half tile whose first element is e0 and
// whose accumulator columns start at dcol (of which the first nel exist: fewer
// in a ragged last tile): accumulator columns 9 EL0 .. -> hi + lo sum ->
// FP32 staging (both blocks of each pair, at this thread's nine offsets
// off[3 c + d]) -> coalesced stores, by the 128 threads of one epilogue set
// (named barrier `bar`); `release`, if given, is arrived on once the
// accumulator columns have been read.
template <int P, int EL0, int NEL>
__device__ __forceinline__ void nh_tc_epi_part(uint32_t dcol, int nel, bool writer, const int (&off)[9], float* stage,
                                               const Req& q, int64_t e0, int et, int bar, int lane, uint64_t* release) {
  using C = NhTc<P>;
  constexpr int C0 = 9 * EL0, C1 = 9 * (EL0 + NEL);
  if (nel > 0) {
#pragma unroll
    for (int ch = C0 / 16; ch < (C1 + 15) / 16; ++ch) {
      uint32_t r[16];
      tmem_ld16(dcol + 16u * (uint32_t)ch, r);
      tmem_wait_ld();
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int n = 16 * ch + j;
        if (n >= C0 && n < C1) {
          const float v = __uint_as_float(r[j]);
          const float sum = v + __shfl_xor_sync(0xffffffffu, v, 1);
          if (writer && n / 9 - EL0 < nel) stage[(n / 9 - EL0) * C::NN + off[n % 9]] = sum;
        }
      }
    }
  }
  if (release) {  // this set's last reads of the accumulator buffer: hand it back to the MMA
    tc_fence_before();
    __syncwarp();
    if (lane == 0) mbar_arrive(release);
  }
  named_sync(bar, 128);
  if (nel > 0) {
    const int64_t o = (e0 + EL0) * C::NN;  // a multiple of 4 entries
    const int cnt = nel * C::NN;
    if (q.out_f32) {
      const float4* s4 = reinterpret_cast<const float4*>(stage);
      float4* o4 = reinterpret_cast<float4*>(static_cast<float*>(q.out) + o);
#pragma unroll 2
      for (int k = et; k < cnt / 4; k += 128) __stcs(o4 + k, s4[k]);
    } else {
      const float4* s4 = reinterpret_cast<const float4*>(stage);
      double2* o2 = reinterpret_cast<double2*>(static_cast<double*>(q.out) + o);
#pragma unroll 1
      for (int k = et; k < cnt / 4; k += 128) {
        const float4 v = s4[k];
        __stcs(o2 + 2 * k, make_double2(f2d_ftz(v.x), f2d_ftz(v.y)));
        __stcs(o2 + 2 * k + 1, make_double2(f2d_ftz(v.z), f2d_ftz(v.w)));
      }
    }
  }
  named_sync(bar, 128);
}

// A packed pair (x, y) -> BF16 pair hi (x low) and the BF16 pair lo of the
// remainders (x - hi.x, y - hi.y, exact in FP32).
__device__ __forceinline__ void split_bf16_pair(float2 h, uint32_t& hi, uint32_t& lo) {
  const __nv_bfloat162 hb = __float22bfloat162_rn(h);
  const float2 r = __ffma2_rn(__bfloat1622float2(hb), make_float2(-1.f, -1.f), h);
  const __nv_bfloat162 lb = __float22bfloat162_rn(r);
  hi = *reinterpret_cast<const uint32_t*>(&hb);
  lo = *reinterpret_cast<const uint32_t*>(&lb);
}

// Point pairs 4 G .. 4 G + 3 of the H row (e, c, d): K columns 72 G .. 72 G + 71,
// two points at a time in packed FP32x2 arithmetic (the pair's values at one
// (k, l) are one packed BF16 pair), split into BF16 hi and lo parts; 9
// core-matrix columns of each, each stored as soon as its 4 pairs exist.
// rec: the element's pointwise record; pwk: its mu |det J| K.
template <int P>
__device__ __forceinline__ void nh_tc_build_group(int G, const float* rec, const float* pwk, int c, int d, float lam,
                                                  char* hhi, char* hlo) {
  using C = NhTc<P>;
  uint32_t whi[36], wlo[36];  // word 9 pl + kl: pair pl of the group at (k, l)
#pragma unroll
  for (int pl = 0; pl < 4; ++pl) {
    const int q0 = 2 * (4 * G + pl);  // the pair's first point
    float2 h[9];
    if (q0 < C::Q) {
      const float* pr = rec + 20 * (q0 >> 1);
      const float2 sa = *reinterpret_cast<const float2*>(pr);  // alpha_q, alpha_q+1
      const float2 sl = make_float2(lam, lam);
      float2 Mc[3], Md[3];  // rows c and d of M' = sqrt(s) M at both points
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        Mc[k] = *reinterpret_cast<const float2*>(pr + 2 + 6 * c + 2 * k);
        Md[k] = *reinterpret_cast<const float2*>(pr + 2 + 6 * d + 2 * k);
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float2 pd = __fmul2_rn(sa, Md[k]), lc = __fmul2_rn(sl, Mc[k]);
#pragma unroll
        for (int l = 0; l < 3; ++l) h[3 * k + l] = __ffma2_rn(pd, Mc[l], __fmul2_rn(lc, Md[l]));
      }
      if (q0 + 1 == C::Q) {  // the pair's second point is the point-summed term
#pragma unroll
        for (int kl = 0; kl < 9; ++kl) h[kl].y = c == d ? pwk[kl] : 0.f;
      }
    } else {
#pragma unroll
      for (int kl = 0; kl < 9; ++kl) h[kl] = make_float2(q0 == C::Q && c == d ? pwk[kl] : 0.f, 0.f);
    }
#pragma unroll
    for (int kl = 0; kl < 9; ++kl) split_bf16_pair(h[kl], whi[9 * pl + kl], wlo[9 * pl + kl]);
    // core-matrix columns complete after this pair: words 4 i .. 4 i + 3 < 9 (pl + 1)
#pragma unroll
    for (int i = (pl == 0 ? 0 : (9 * pl) / 4); i < (9 * (pl + 1)) / 4; ++i) {
      const int uidx = 9 * G + i;
      if (uidx < C::KU) {
        *reinterpret_cast<uint4*>(hhi + (size_t)uidx * C::LBO) = make_uint4(whi[4 * i], whi[4 * i + 1], whi[4 * i + 2], whi[4 * i + 3]);
        *reinterpret_cast<uint4*>(hlo + (size_t)uidx * C::LBO) = make_uint4(wlo[4 * i], wlo[4 * i + 1], wlo[4 * i + 2], wlo[4 * i + 3]);
      }
    }
  }
}

template <int P>
__global__ void __launch_bounds__(NhTc<P>::NTH, 1) nh_tc_kernel(Req q, unsigned* err) {
  using C = NhTc<P>;
  extern __shared__ __align__(16) char smem_raw[];
  if (C::SMEM > dynamic_smem_bytes()) {
    if (threadIdx.x == 0) flag_error(err, ERR_LAUNCH);
    return;
  }
  char* sm = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
  NhTcBars* bars = reinterpret_cast<NhTcBars*>(sm + C::O_BAR);
  volatile int* ring = reinterpret_cast<volatile int*>(sm + C::O_BAR + kNhTcRingOff);
  float* sW = reinterpret_cast<float*>(sm + C::O_W);
  float* sD = reinterpret_cast<float*>(sm + C::O_DPHI);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t ntiles = (q.E + C::TE - 1) / C::TE;
  const float* tab = static_cast<const float*>(q.tab);
  const TcTabLayout L = tc_tab_layout(C::Q, C::NS, C::K);
  const float mu_c = d2f(q.coeffs[q.E * C::CLEN]), lam_c = d2f(q.coeffs[q.E * C::CLEN + 1]);
  const float nan = __int_as_float(0x7fc00000);

  if (tid == 0) {
    for (int i = 0; i < 3; ++i) {
      mbar_init(&bars->geo_full[i], 1);
      mbar_init(&bars->geo_empty[i], 4);
      mbar_init(&bars->pw_full[i], 4);
      mbar_init(&bars->pw_empty[i], 8);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&bars->in_full[i], 1);
      mbar_init(&bars->h_full[i], 4);
      mbar_init(&bars->h_empty[i], 1);
      mbar_init(&bars->d_full[i], 1);
      mbar_init(&bars->d_empty[i], 8);
    }
    mbar_init(&bars->done, 1);
    fence_barrier_init();
  }
  for (int i = tid; i < C::Q; i += C::NTH) sW[i] = tab[L.offW + i];
  for (int i = tid; i < C::Q * C::RS; i += C::NTH) {
    const int qq = i / C::RS, j = i - qq * C::RS;
    if (j >= C::NS * 3) sD[i] = 0.f;
  }
  __syncthreads();
  for (int i = tid; i < C::Q * C::NS * 3; i += C::NTH) {  // dPhi_a^k at node_slot(a, k)
    const int qq = i / (C::NS * 3), r = i - qq * (C::NS * 3);
    sD[qq * C::RS + C::node_slot(r / 3, r % 3)] = tab[L.offDphi + i];
  }
  {
    uint4* z = reinterpret_cast<uint4*>(sm);
    for (int i = tid; i < 2 * C::HPART / 16; i += C::NTH) z[i] = make_uint4(0u, 0u, 0u, 0u);
    float* u = reinterpret_cast<float*>(sm + C::O_UT);
    for (int i = tid; i < C::NGB * C::TE * C::RU; i += C::NTH) u[i] = 0.f;
  }
  if (warp == 0) {
    tmem_alloc(&bars->tbase, C::TMEM_COLS);
    tmem_relinquish();
  }
  fence_proxy_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tb = bars->tbase;

  // reference tables into tensor memory (the first epilogue set covers the four lane quarters):
  // lane m = row m of R_stack, K / 2 packed columns
  if (warp >= C::W_EPI && warp < C::W_EPI + 4) {
    const int qd = warp & 3, m = 32 * qd + lane;
    const uint4* src = reinterpret_cast<const uint4*>(tab + L.offR) + (size_t)m * (C::K / 8);
    for (int c0 = 0; c0 < C::K / 2; c0 += 16) {
      uint32_t v[16];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const uint4 w = __ldg(src + c0 / 4 + j);
        v[4 * j] = w.x;
        v[4 * j + 1] = w.y;
        v[4 * j + 2] = w.z;
        v[4 * j + 3] = w.w;
      }
      tmem_st16(tb + ((uint32_t)(32 * qd) << 16) + C::COL_R + (uint32_t)c0, v);
    }
    tmem_wait_st();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();

  if (warp == 0) {
    // ------------------------------------------------------------- MMA issue
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_f16kind(1u, 128u, (uint32_t)C::NCOL);
      const uint32_t hhi = smem_addr(sm + C::O_HHI), hlo = smem_addr(sm + C::O_HLO);
      bool ok = true;
      for (int it = 0;; ++it) {
        const int buf = it & 1;
        ok = it < 2 || mbar_wait_sleep(&bars->d_empty[buf], (unsigned)(((it >> 1) - 1) & 1));
        if (ok) ok = mbar_wait_sleep(&bars->h_full[0], (unsigned)(it & 1));
        if (!ok) break;
        if (ring[it % kNhTcRing] < 0) {  // past the last tile: let the epilogue see it too
          tc_commit(&bars->d_full[buf]);
          break;
        }
        const uint32_t dt = tb + (uint32_t)buf * 128u;
        // the two halves of K, written by the two builder groups (K steps 0 .. KSA - 1, KSA .. KS - 1)
        for (int h = 0; h < 2 && ok; ++h) {
          if (h > 0) ok = mbar_wait_sleep(&bars->h_full[h], (unsigned)(it & 1));
          if (!ok) break;
          tc_fence_after();
          const int j0 = h == 0 ? 0 : C::KSA, j1 = h == 0 ? C::KSA : C::KS;
#pragma unroll 1
          for (int j = j0; j < j1; ++j) {
            const uint32_t at = tb + C::COL_R + 8u * (uint32_t)j;
            mma_f16_ts(dt, at, smem_desc_kmajor(hhi + 2u * C::LBO * j, C::LBO, C::SBO), idesc, j > 0 ? 1u : 0u);
            mma_f16_ts(dt, at, smem_desc_kmajor(hlo + 2u * C::LBO * j, C::LBO, C::SBO), idesc, 1u);
          }
          tc_commit(&bars->h_empty[h]);
        }
        if (!ok) break;
        tc_commit(&bars->d_full[buf]);
      }
      if (!ok) flag_error(err, ERR_TIMEOUT);
      tc_commit(&bars->done);
      if (!mbar_wait_sleep(&bars->done, 0u)) flag_error(err, ERR_TIMEOUT);
    }
    __syncwarp();
  } else if (warp < C::W_EPI) {
    // -------------------------------------------------------------- geometry
    const int gt = tid - 32 * C::W_GEO;  // 0 .. 95
    constexpr int NG_T = 32 * (C::W_EPI - C::W_GEO);
    auto issue_inputs = [&](int64_t t, int ib) -> bool {
      if (q.skip_copy == t + 1) return false;  // test hook: this tile's inputs never come
      const int64_t e0 = t * C::TE;
      const int ne = (int)(q.E - e0 < C::TE ? q.E - e0 : C::TE);
      char* inb = sm + C::O_IN + (size_t)ib * C::IN_BUF;
      mbar_expect_tx(&bars->in_full[ib], (unsigned)(ne * (12 + C::CLEN) * 8));
      bulk_g2s(inb, q.coords + e0 * 12, (unsigned)(ne * 96), &bars->in_full[ib]);
      bulk_g2s(inb + C::TE * 96, q.coeffs + e0 * C::CLEN, (unsigned)(ne * C::CLEN * 8), &bars->in_full[ib]);
      return true;
    };
    // leader: the tile of this CTA's next iteration, -1 past the last one (draws are monotonic)
    bool drawn_out = false;
    int64_t next_static = blockIdx.x;
    auto draw = [&]() -> int {
      if (drawn_out) return -1;
      const int64_t t = q.tile_ctr ? (int64_t)atomicAdd(q.tile_ctr, 1ull) : next_static;
      next_static += gridDim.x;
      if (t >= ntiles) {
        drawn_out = true;
        return -1;
      }
      return (int)t;
    };
    int pend0 = -1, pend1 = -1;  // iteration whose input copy is in flight, per buffer (leader thread)
    if (gt == 0) {
      const int t0 = draw();
      ring[0] = t0;
      if (t0 >= 0 && issue_inputs(t0, 0)) pend0 = 0;
      const int t1 = draw();
      ring[1] = t1;
      if (t1 >= 0 && issue_inputs(t1, 1)) pend1 = 1;
    }
    named_sync(C::BAR_GEO, NG_T);
    bool ok = true;
    for (int it = 0;; ++it) {
      const int64_t t = ring[it % kNhTcRing];
      const int b = it & 1, gb = it % 3;
      bool w = t < 0 || mbar_wait_sleep(&bars->in_full[b], (unsigned)((it >> 1) & 1));
      if (w && it >= 3) w = mbar_wait_sleep(&bars->geo_empty[gb], (unsigned)((it / 3 - 1) & 1));
      if (t < 0 && w && gt == 0) {
        // past the last tile: both kinematics groups learn it (this iteration and the next)
        mbar_arrive(&bars->geo_full[gb]);
        const int i1 = it + 1;
        w = i1 < 3 || mbar_wait_sleep(&bars->geo_empty[i1 % 3], (unsigned)((i1 / 3 - 1) & 1));
        ring[i1 % kNhTcRing] = -1;
        if (w) mbar_arrive(&bars->geo_full[i1 % 3]);
      }
      ok = named_and(C::BAR_GEO, NG_T, w);
      if (!ok || t < 0) break;
      const int64_t e0 = t * C::TE;
      const int ne = (int)(q.E - e0 < C::TE ? q.E - e0 : C::TE);
      if (gt == 0) (b ? pend1 : pend0) = -1;
      const double* xs = reinterpret_cast<const double*>(sm + C::O_IN + (size_t)b * C::IN_BUF);
      const double* us = xs + C::TE * 12;
      float* ut = reinterpret_cast<float*>(sm + C::O_UT) + gb * C::TE * C::RU;
      float* geo = reinterpret_cast<float*>(sm + C::O_GEO) + gb * C::TE * 24;
      for (int i = gt; i < ne * C::CLEN; i += NG_T) {
        const int e = i / C::CLEN;
        const int r = i - e * C::CLEN;  // displacement DOF u_a[c] at 3 a + c, to its node-pair slot
        ut[e * C::RU + C::node_slot(r / 3, r % 3)] = d2f_rz(us[i]);
      }
      if (gt < ne) {  // FP64 geometry of element gt
        double adj[9];
        const double det = geometry_fp64(xs + 12 * gt, adj);
        const uint64_t bits = (uint64_t)__double_as_longlong(det);
        const bool bad = ((bits << 1) == 0) || ((bits >> 52 & 0x7ff) == 0x7ff);
        if (bad) flag_error(err, ERR_DEGENERATE);
        const float df = d2f_rz(det), inv = 1.0f / df;
        float Ji[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) Ji[k] = d2f_rz(adj[k]) * inv;
        float* g = geo + 24 * gt;
#pragma unroll
        for (int k = 0; k < 9; ++k) g[k] = bad ? nan : Ji[k];
        g[9] = bad ? nan : fabsf(df);
        const float mdet = mu_c * fabsf(df);  // the point-summed term: mu |det J| J^-1 J^-T
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
          for (int l = 0; l < 3; ++l)
            g[12 + 3 * k + l] =
                bad ? nan : mdet * (Ji[3 * k] * Ji[3 * l] + Ji[3 * k + 1] * Ji[3 * l + 1] + Ji[3 * k + 2] * Ji[3 * l + 2]);
      }
      named_sync(C::BAR_GEO, NG_T);
      if (gt == 0) {
        // the input buffer has been read: draw the tile two iterations ahead and prefetch it into it
        const int t2 = draw();
        ring[(it + 2) % kNhTcRing] = t2;
        if (t2 >= 0) {
          fence_proxy_async();
          if (issue_inputs(t2, b)) (b ? pend1 : pend0) = it + 2;
        }
        mbar_arrive(&bars->geo_full[gb]);
      }
    }
    if (!ok) flag_error(err, ERR_TIMEOUT);
    // copies issued before giving up must land before the CTA leaves
    if (gt == 0) {
      if (pend0 >= 0) mbar_wait_sleep(&bars->in_full[0], (unsigned)((pend0 >> 1) & 1));
      if (pend1 >= 0) mbar_wait_sleep(&bars->in_full[1], (unsigned)((pend1 >> 1) & 1));
    }
  } else if (warp < C::W_KIN) {
    // -------------------------------------------------------------- epilogue
    const int set = (warp - C::W_EPI) >> 2;  // elements EH set .. EH set + EH - 1 of every tile
    const int et = tid - 32 * C::W_EPI - 128 * set;
    const int bar = C::BAR_EPI + set;
    const int qd = warp & 3, m = 32 * qd + lane, p = m >> 1, hx = m & 1;
    int a = 0, b = 0;
    if (p < C::NPAIR) sym_pair(p, C::NS, &a, &b);
    const bool writer = p < C::NPAIR && (hx == 0 || a != b);
    // even lane: entry (3a + c, 3b + d); odd lane: the mirrored entry (3b + d, 3a + c)
    const int base = hx == 0 ? 3 * a * C::N3 + 3 * b : 3 * b * C::N3 + 3 * a;
    const int sc = hx == 0 ? C::N3 : 1, sd = hx == 0 ? 1 : C::N3;
    int off[9];
#pragma unroll
    for (int cd = 0; cd < 9; ++cd) off[cd] = base + (cd / 3) * sc + (cd % 3) * sd;
    float* stage = reinterpret_cast<float*>(sm + C::O_STAGE + (size_t)set * round_up_sz((size_t)C::ES * C::NN * 4, 16));
    const uint32_t trow = tb + ((uint32_t)(32 * qd) << 16);
    bool ok = true;
    for (int it = 0;; ++it) {
      const int buf = it & 1;
      ok = named_and(bar, 128, mbar_wait_sleep(&bars->d_full[buf], (unsigned)((it >> 1) & 1)));
      if (!ok) break;
      const int64_t t = ring[it % kNhTcRing];
      if (t < 0) break;  // past the last tile
      const int64_t e0 = t * C::TE;
      const int ne = (int)(q.E - e0 < C::TE ? q.E - e0 : C::TE);
      tc_fence_after();
      const uint32_t dcol = trow + (uint32_t)buf * 128u;
      static_assert(C::EH == 7 && C::ES == 4 && 9 * C::EH < 64, "epilogue parts");
      const uint32_t dset = dcol + 64u * (uint32_t)set;
      const int64_t es = e0 + C::EH * set;
      const int ns = ne - C::EH * set;
      nh_tc_epi_part<P, 0, 4>(dset, min(4, ns), writer, off, stage, q, es, et, bar, lane, nullptr);
      nh_tc_epi_part<P, 4, 3>(dset, min(3, ns - 4), writer, off, stage, q, es, et, bar, lane, &bars->d_empty[buf]);
    }
    if (!ok) flag_error(err, ERR_TIMEOUT);
  } else if (warp < C::W_BLD) {
    // ------------------------------------------------------------ kinematics
    const int gk = (warp - C::W_KIN) >> 2;  // group gk takes the iterations gk, gk + 2, ...
    const int kt = tid - 32 * C::W_KIN - 128 * gk;
    const int bar_id = C::BAR_KIN + gk;
    bool ok = true;
    for (int it = gk;; it += 2) {
      const int gb = it % 3, slot = gb;  // geometry buffer and pointwise slot of this iteration
      const float* ut = reinterpret_cast<const float*>(sm + C::O_UT) + gb * C::TE * C::RU;
      float* pw = reinterpret_cast<float*>(sm + C::O_PW + (size_t)slot * C::PW_SLOT);
      float* pwk = reinterpret_cast<float*>(sm + C::O_PWK) + slot * C::TE * 9;
      const float* geo = reinterpret_cast<const float*>(sm + C::O_GEO) + gb * C::TE * 24;
      bool w = mbar_wait_sleep(&bars->geo_full[gb], (unsigned)((it / 3) & 1));
      if (w && it >= 3) w = mbar_wait_sleep(&bars->pw_empty[slot], (unsigned)((it / 3 - 1) & 1));
      ok = named_and(bar_id, 128, w);
      if (!ok) break;
      const int64_t t = ring[it % kNhTcRing];
      if (t < 0) {  // past the last tile: pass it on to the H builders
        if (lane == 0) mbar_arrive(&bars->pw_full[slot]);
        break;
      }
      const int64_t e0 = t * C::TE;
      const int ne = (int)(q.E - e0 < C::TE ? q.E - e0 : C::TE);
      if (kt < ne) {
#pragma unroll
        for (int k = 0; k < 9; ++k) pwk[9 * kt + k] = geo[24 * kt + 12 + k];
      }
      for (int w2 = kt; w2 < ne * C::Q; w2 += 128) {
        const int e = w2 / C::Q, qq = w2 - e * C::Q;
        float uv[32], dv[32];  // u_a[i] and dPhi_a^k at node_slot(a, i or k)
        {
          const float4* u4 = reinterpret_cast<const float4*>(ut + C::RU * e);
          const float4* d4 = reinterpret_cast<const float4*>(sD + C::RS * qq);
#pragma unroll
          for (int v = 0; v < 8; ++v) {
            const float4 uu = u4[v], dd = d4[v];
            uv[4 * v] = uu.x; uv[4 * v + 1] = uu.y; uv[4 * v + 2] = uu.z; uv[4 * v + 3] = uu.w;
            dv[4 * v] = dd.x; dv[4 * v + 1] = dd.y; dv[4 * v + 2] = dd.z; dv[4 * v + 3] = dd.w;
          }
        }
        // gr[3 i + k] = sum_a u_a[i] dPhi_a^k, two nodes at a time (packed), even and odd nodes summed last
        float2 acc[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) acc[k] = make_float2(0.f, 0.f);
#pragma unroll
        for (int np = 0; np < C::NS / 2; ++np)
#pragma unroll
          for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int k = 0; k < 3; ++k)
              acc[3 * i + k] = __ffma2_rn(make_float2(uv[6 * np + 2 * i], uv[6 * np + 2 * i + 1]),
                                          make_float2(dv[6 * np + 2 * k], dv[6 * np + 2 * k + 1]), acc[3 * i + k]);
        float gr[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) gr[k] = acc[k].x + acc[k].y;
        float J[12];
        {
          const float4* j4 = reinterpret_cast<const float4*>(geo + 24 * e);
          const float4 a0 = j4[0], a1 = j4[1], a2 = j4[2];
          J[0] = a0.x; J[1] = a0.y; J[2] = a0.z; J[3] = a0.w;
          J[4] = a1.x; J[5] = a1.y; J[6] = a1.z; J[7] = a1.w;
          J[8] = a2.x; J[9] = a2.y; J[10] = a2.z; J[11] = a2.w;
        }
        double F[9];  // F = I + grad u, grad u = gr J^-1 (FP32), widened exactly
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int x = 0; x < 3; ++x)
            F[3 * i + x] = f2d_normal(gr[3 * i] * J[x] + gr[3 * i + 1] * J[3 + x] + gr[3 * i + 2] * J[6 + x]);
        F[0] += 1.0;
        F[4] += 1.0;
        F[8] += 1.0;
        double cof[9];  // det(F) F^-1
        cof[0] = fma(F[4], F[8], -F[5] * F[7]);
        cof[1] = fma(F[2], F[7], -F[1] * F[8]);
        cof[2] = fma(F[1], F[5], -F[2] * F[4]);
        cof[3] = fma(F[5], F[6], -F[3] * F[8]);
        cof[4] = fma(F[0], F[8], -F[2] * F[6]);
        cof[5] = fma(F[2], F[3], -F[0] * F[5]);
        cof[6] = fma(F[3], F[7], -F[4] * F[6]);
        cof[7] = fma(F[1], F[6], -F[0] * F[7]);
        cof[8] = fma(F[0], F[4], -F[1] * F[3]);
        const double dF = fma(F[0], cof[0], fma(F[1], cof[3], F[2] * cof[6]));
        const uint32_t dhi = (uint32_t)__double2hiint(dF);
        const bool bad = (int)dhi <= 0 || (dhi >> 20) >= 0x7ffu;  // det F <= 0 (or tiny), inf or NaN
        if (bad) flag_error(err, ERR_DEGENERATE);
        // the cancellation-prone cofactors, det F and ln det F are FP64; F^-1 = cof / det F
        // is a well-conditioned scaling done after rounding to FP32
        // H = alpha M'_d M'_c + lam M'_c M'_d with M' = sqrt(s) M: sqrt(s) rides on 1 / det F
        const float rs = __fsqrt_rn(sW[qq] * J[9]);
        const float idF = __frcp_rn(d2f_rz(dF)) * rs;
        const float lnJ = d2f_rz(log_f64(dF));
        float Fi[9];  // Fi[3 I + c] = sqrt(s) (F^-1)[I][c]
#pragma unroll
        for (int k = 0; k < 9; ++k) Fi[k] = d2f_rz(cof[k]) * idF;
        const float al = mu_c - lam_c * lnJ;
        float* rec = pw + e * C::PW_E + 20 * (qq >> 1) + (qq & 1);  // this point's slots of its pair record
        rec[0] = bad ? nan : al;
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int k = 0; k < 3; ++k)  // M[c][k] = sum_I (F^-1)[I][c] (J^-1)[k][I]
            rec[2 + 6 * c + 2 * k] = bad ? nan : Fi[c] * J[3 * k] + Fi[3 + c] * J[3 * k + 1] + Fi[6 + c] * J[3 * k + 2];
      }
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&bars->pw_full[slot]);
        mbar_arrive(&bars->geo_empty[gb]);
      }
    }
    if (!ok) flag_error(err, ERR_TIMEOUT);
  } else {
    // ----------------------------------------------------------- H builders
    const int gb = (warp - C::W_BLD) >> 2;                // half of the point groups
    const int n = ((warp - C::W_BLD) & 3) * 32 + lane;   // H row = column of D
    const int nr = n & 63;                               // 64 columns per half tile, the last unused
    const int e = nr < 63 ? C::EH * (n >> 6) + nr / 9 : C::TE, cd = nr - 9 * (nr / 9), c = cd / 3, d = cd - 3 * (cd / 3);
    char* hhi = sm + C::O_HHI + (size_t)(n >> 3) * C::SBO + (size_t)(n & 7) * 16;
    char* hlo = sm + C::O_HLO + (size_t)(n >> 3) * C::SBO + (size_t)(n & 7) * 16;
    static_assert(C::NG == 4, "two point groups per builder half");
    bool ok = true;
    for (int it = 0;; ++it) {
      const int slot = it % 3;
      unsigned w = 1;
      if (lane == 0) {
        w = mbar_wait_sleep(&bars->pw_full[slot], (unsigned)((it / 3) & 1));
        // this group's half of H is free once the MMAs of the previous tile have read it
        if (w && it >= 1) w = mbar_wait_sleep(&bars->h_empty[gb], (unsigned)((it - 1) & 1));
      }
      ok = __shfl_sync(0xffffffffu, w, 0) != 0;
      if (!ok) break;
      const int64_t t = ring[it % kNhTcRing];
      if (t < 0) {  // past the last tile: pass it on to the MMA warp
        if (lane == 0) mbar_arrive(&bars->h_full[gb]);
        break;
      }
      const int64_t e0 = t * C::TE;
      const int ne = (int)(q.E - e0 < C::TE ? q.E - e0 : C::TE);
      if (e < ne) {
        const float* rec = reinterpret_cast<const float*>(sm + C::O_PW + (size_t)slot * C::PW_SLOT) + e * C::PW_E;
        const float* pwk = reinterpret_cast<const float*>(sm + C::O_PWK) + slot * C::TE * 9 + 9 * e;
#pragma unroll 1
        for (int G = 2 * gb; G < 2 * gb + 2; ++G) nh_tc_build_group<P>(G, rec, pwk, c, d, lam_c, hhi, hlo);
      }
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&bars->h_full[gb]);
        mbar_arrive(&bars->pw_empty[slot]);
      }
    }
    if (!ok) flag_error(err, ERR_TIMEOUT);
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tb, C::TMEM_COLS);
  }
}

}  // namespace fea
