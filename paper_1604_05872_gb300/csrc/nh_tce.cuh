// Neo-Hookean tangent stiffness on the tensor cores (tcgen05), one dense
// product per element; split-BF16 operands, FP32 accumulation.
//
// From P3 up the shared-operand form of nh_tc.cuh does not fit: the split
// reference tables of all basis pairs (2 x 210 rows x 9 (Q + 1) columns at P3)
// exceed both tensor and shared memory, and its product grows as n_s^2 x 9 Q.
// Here the contraction keeps the structure of the sharing-eliminated nest
// (Section 3.2, Algorithm 1) instead: with
//
//   M'_q = sqrt(s_q) F^-T J^-T (3 x 3 per point), s_q = w_q |det J|,
//   U[(a,x), q] = sum_k M'_q[x][k] dPhi_a^k(X_q)      (= sqrt(s_q) Y_a^x, Y = F^-T G)
//   S[(a,x),(b,y)] = sum_q U[(a,x),q] U[(b,y),q]
//   T[(a,x),(b,y)] = sum_q alpha_q U[(a,x),q] U[(b,y),q],  alpha = mu - lam ln det F
//
// the tangent is
//
//   A[(a,c),(b,d)] = T[(a,d),(b,c)] + lam S[(a,c),(b,d)] + delta_cd Mu[a][b],
//   Mu[a][b] = mu |det J| sum_{k,l} (J^-1 J^-T)[k][l] Rbar_ab^kl,
//   Rbar_ab^kl = sum_q w_q dPhi_a^k(X_q) dPhi_b^l(X_q)  (pre-evaluated, Section 3.3).
//
// S and T of one element are one MMA: D[128 x 64] = A_op[128 x Q] B_op[64 x Q]^T
// with A_op rows 0 .. 3 n_s - 1 = U, rows 64 .. 64 + 3 n_s - 1 = alpha U and
// B_op = U (the first 64 rows of A_op, the same shared memory), so D rows 0 ..
// hold S and rows 64 .. hold T.  U and alpha U are split into BF16 hi and lo
// parts; three chains A_hi B_hi + A_hi B_lo + A_lo B_hi accumulate into the same
// FP32 tensor-memory columns (the lo * lo term lies below the FP32 rounding of
// the sum).
//
// Roles (one CTA per SM, persistent over tiles of TE elements, 23 warps):
//   warp 0        allocates tensor memory; one lane issues the MMAs;
//   warp 1        geometry: tile inputs by bulk copy two tiles ahead, the
//                 displacement DOFs to FP32, per element J^-1, |det J| (FP64
//                 J, adj J, det J) and mu |det J| J^-1 J^-T;
//   warps 2-9     kinematics, two groups of four taking alternate tiles: per
//                 (element, point) grad u (packed FP32), F, its cofactors, det F
//                 and ln det F in FP64, alpha and M';
//   warps 10-14   operands: thread (a, point octet) keeps its dPhi_a in
//                 registers and writes the element's U and alpha U rows (hi and
//                 lo, 16-byte core-matrix rows); also the Mu tables;
//   warps 15-22   epilogue, two sets of four (elements 0, 1 and 2, 3 of a
//                 tile), each covering the four lane quarters of tensor memory:
//                 T rows scattered block-transposed into an FP32 staging
//                 matrix, then S rows (and Mu) added in place, then coalesced
//                 16-byte stores.
// Tiles are handed out by an atomic counter when the launch provides one (so a
// CTA on a faster SM takes more of them), else CTA c takes tiles c, c + grid, ...
// The geometry warp draws them, two iterations ahead, into a ring in shared
// memory; every role reads iteration i's tile there after the wait that hands it
// iteration i.  Past the last tile the ring holds -1: each role passes that mark
// on through the signal its consumer waits for, then leaves.
// Every mbarrier wait is bounded; a role that gives up sets the error word, the
// others then give up too, and the CTA waits for its copies and MMAs in flight
// before it frees the tensor memory and leaves.
#pragma once
#include "common.cuh"
#include "launch.cuh"
#include "log_f64.cuh"
#include "mbar.cuh"
#include "tc.cuh"

#include <cuda_bf16.h>

namespace fea {

template <int P>
struct NhTcE {
  static constexpr int NS = nbasis_c(P);
  static constexpr int N3 = 3 * NS;
  static constexpr int NN = N3 * N3;
  static constexpr int CLEN = 3 * NS;
  static constexpr int Q = (P + 1) * (P + 1) * (P + 1);  // collapsed rule, p + 1 points per direction
  static_assert(N3 <= 64 && Q % 16 == 0 && Q <= 64, "one 128 x 64 x Q product per element");
  static constexpr int K = Q;
  static constexpr int KC = K / 8;   // 16-byte core-matrix columns along K
  static constexpr int KS = K / 16;  // MMA steps per chain
  static constexpr uint32_t LBO = 128, SBO = KC * 128;
  static constexpr int OPB = 128 * K * 2;  // bytes of one split part of A_op
  static constexpr int OPSLOT = 2 * OPB;   // hi, then lo
  static constexpr int TE = 4;             // elements per tile: one operand slot each
  static constexpr int NCOL = 64;          // accumulator columns per element
  static constexpr int NOCT = Q / 8;       // point octets
  static constexpr int NBT = NS * NOCT;    // operand threads: (a, octet)
  static constexpr int NMU = NS * NS;
  static constexpr int MU_PER = (NMU + NBT - 1) / NBT;  // Mu entries per operand thread
  // pointwise record per element and octet: alpha[8], then M'[x][k][8]; 88 floats so that the
  // kinematics' stores of consecutive points fall on distinct banks across octets
  static constexpr int PW_O = 88, PW_E = NOCT * PW_O;
  static constexpr int NPW = 2;                         // slots: one per kinematics group
  static constexpr int PW_SLOT_F = TE * PW_E + TE * 8;  // + mu |det J| K (6, padded) per element
  static constexpr int LD = N3 + 2;                     // staging row stride (even: 8-byte pairs; rows spread over banks)
  static constexpr int RS = 68;                         // dPhi row per point: 16-byte loads on distinct banks
  static constexpr int RU = 64;                         // floats per element row of u
  static constexpr int NGB = 3;                         // geometry buffers (iteration % 3)
  static constexpr int W_GEO = 1, W_KIN = 2, W_BLD = 10, W_EPI = 15, NWARP = 23;
  static constexpr int NTH = 32 * NWARP;
  static_assert(32 * (W_EPI - W_BLD) == NBT, "one operand thread per (basis function, point octet)");
  static constexpr int BAR_KIN = 1, BAR_EPI = 3;  // kinematics groups 1, 2; epilogue sets 3, 4
  static constexpr uint32_t TMEM_COLS = 512;
  static_assert(2 * TE * NCOL <= (int)TMEM_COLS, "double-buffered accumulators");

  static constexpr size_t O_OP = 0;
  static constexpr size_t O_STAGE = O_OP + (size_t)TE * OPSLOT;
  static constexpr size_t STAGE_B = round_up_sz((size_t)N3 * LD * 4, 16);
  static constexpr size_t O_MU = O_STAGE + 2 * STAGE_B;  // [2 buffers][TE][NS][NS]
  static constexpr size_t O_PW = O_MU + 2 * (size_t)TE * NMU * 4;
  static constexpr size_t PW_SLOT = (size_t)PW_SLOT_F * 4;
  static constexpr size_t O_IN = O_PW + NPW * PW_SLOT;
  static constexpr size_t IN_BUF = (size_t)TE * (12 + CLEN) * 8;  // coords, then displacement DOFs
  static constexpr size_t O_UT = O_IN + 2 * IN_BUF;
  static constexpr size_t O_GEO = O_UT + NGB * (size_t)TE * RU * 4;  // per element J^-1, |det J|, mu|det J|K
  static constexpr size_t O_W = O_GEO + NGB * (size_t)TE * 24 * 4;
  static constexpr size_t O_DPHI = O_W + round_up_sz((size_t)Q * 4, 16);
  static constexpr size_t O_BAR = O_DPHI + (size_t)Q * RS * 4;
  static constexpr int NRING = 16;                    // tiles of the coming iterations (see the geometry role)
  static constexpr size_t O_RING = O_BAR + 256;
  static constexpr size_t SMEM = O_RING + NRING * 8 + 128;  // + alignment of the base to 128 bytes
  static_assert(SMEM <= 232448, "shared memory per CTA");
  static_assert(O_STAGE % 16 == 0 && O_MU % 16 == 0 && O_PW % 16 == 0 && O_IN % 16 == 0 && O_UT % 16 == 0 &&
                    O_GEO % 16 == 0 && O_DPHI % 16 == 0 && O_BAR % 16 == 0,
                "alignment");
  static_assert(IN_BUF % 16 == 0 && (TE * 96) % 16 == 0 && (CLEN * 8) % 16 == 0, "bulk-copy alignment");
  static_assert(NS % 2 == 0 && N3 <= RU && N3 <= RS && (N3 % 12) == 0, "node-pair rows");
  // rows of u and of dPhi at a point hold the nodes in pairs: entry 6 (a / 2) + 2 i + a % 2
  FEA_HD static constexpr int node_slot(int a, int i) { return 6 * (a >> 1) + 2 * i + (a & 1); }

  FEA_HD static int max_tile() { return TE; }
  FEA_HD static int pref_tile() { return TE; }
  FEA_HD static size_t smem(int, int) { return SMEM; }
};

// Device table of the kernel, in 32-bit words: W [Q], dphi [Q][ns][3], then
// the symmetric point-summed tables Rbar_s [ns * ns][6] (float).
struct TcETabLayout {
  int offW, offDphi, offRbar, total;
};
FEA_HD inline TcETabLayout tce_tab_layout(int Q, int ns) {
  TcETabLayout t{};
  t.offW = 0;
  t.offDphi = round_up(Q, 4);
  t.offRbar = t.offDphi + round_up(Q * ns * 3, 4);
  t.total = t.offRbar + ns * ns * 6;
  return t;
}

struct NhTcEBars {
  uint64_t in_full[2], geo_full[3], geo_empty[3], pw_full[2], pw_empty[2], op_full[4], op_empty[4], d_full[2],
      d_empty[2], mu_full[2], done;
  uint32_t tbase;
};

// D[d_tmem] (+)= A[a_desc] * B[b_desc]^T, both operands in shared memory, issued by one thread.
__device__ __forceinline__ void mma_f16_ss(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                           uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// A packed pair (x, y) -> BF16 pair hi (x low) and the BF16 pair lo of the
// remainders (x - hi.x, y - hi.y, exact in FP32).
__device__ __forceinline__ void split_bf16_pair_e(float2 h, uint32_t& hi, uint32_t& lo) {
  const __nv_bfloat162 hb = __float22bfloat162_rn(h);
  const float2 r = __ffma2_rn(__bfloat1622float2(hb), make_float2(-1.f, -1.f), h);
  const __nv_bfloat162 lb = __float22bfloat162_rn(r);
  hi = *reinterpret_cast<const uint32_t*>(&hb);
  lo = *reinterpret_cast<const uint32_t*>(&lb);
}

// One element's operand rows of operand thread (a, octet o): U[(a,x), 8 o ..] and
// alpha U, split into BF16 hi and lo parts, one 16-byte core-matrix row each.
// rec: the element's pointwise record of the octet; op: the element's operand slot.
template <int P>
__device__ __forceinline__ void nh_tce_build(const float4* __restrict__ r4, char* __restrict__ op,
                                             const float2 (&dp)[3][4], int a, int o) {
  using C = NhTcE<P>;
  float2 al[4];
  {
    const float4 x0 = r4[0], x1 = r4[1];
    al[0] = make_float2(x0.x, x0.y); al[1] = make_float2(x0.z, x0.w);
    al[2] = make_float2(x1.x, x1.y); al[3] = make_float2(x1.z, x1.w);
  }
#pragma unroll
  for (int x = 0; x < 3; ++x) {
    float2 u[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) u[j] = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float4 m0 = r4[2 + 2 * (3 * x + k)], m1 = r4[3 + 2 * (3 * x + k)];
      u[0] = __ffma2_rn(make_float2(m0.x, m0.y), dp[k][0], u[0]);
      u[1] = __ffma2_rn(make_float2(m0.z, m0.w), dp[k][1], u[1]);
      u[2] = __ffma2_rn(make_float2(m1.x, m1.y), dp[k][2], u[2]);
      u[3] = __ffma2_rn(make_float2(m1.z, m1.w), dp[k][3], u[3]);
    }
    uint32_t hi[4], lo[4], ahi[4], alo[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      split_bf16_pair_e(u[j], hi[j], lo[j]);
      split_bf16_pair_e(__fmul2_rn(al[j], u[j]), ahi[j], alo[j]);
    }
    const int row = 3 * a + x, rowa = 64 + row;
    const size_t off = (size_t)(row >> 3) * C::SBO + (size_t)o * C::LBO + (size_t)(row & 7) * 16;
    const size_t offa = (size_t)(rowa >> 3) * C::SBO + (size_t)o * C::LBO + (size_t)(rowa & 7) * 16;
    *reinterpret_cast<uint4*>(op + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
    *reinterpret_cast<uint4*>(op + C::OPB + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    *reinterpret_cast<uint4*>(op + offa) = make_uint4(ahi[0], ahi[1], ahi[2], ahi[3]);
    *reinterpret_cast<uint4*>(op + C::OPB + offa) = make_uint4(alo[0], alo[1], alo[2], alo[3]);
  }
}

// The Mu tables of a tile's ne elements, entries ab = bt, bt + NBT, ...:
// Mu[ab] = sum_i Kts_e[i] Rbar_s[ab][i] (Kts = mu |det J| J^-1 J^-T, 6 entries).
template <int P>
__device__ __forceinline__ void nh_tce_mu(const float* __restrict__ rbar, const float* __restrict__ pwk,
                                          float* __restrict__ mu_tab, int bt, int ne) {
  using C = NhTcE<P>;
  float rb[C::MU_PER][6];
#pragma unroll
  for (int j = 0; j < C::MU_PER; ++j)
#pragma unroll
    for (int i = 0; i < 6; ++i) rb[j][i] = bt + j * C::NBT < C::NMU ? __ldg(rbar + 6 * (bt + j * C::NBT) + i) : 0.f;
#pragma unroll 1
  for (int e = 0; e < ne; ++e) {
    float kk[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) kk[i] = pwk[8 * e + i];
#pragma unroll
    for (int j = 0; j < C::MU_PER; ++j) {
      float s = 0.f;
#pragma unroll
      for (int i = 0; i < 6; ++i) s = fmaf(kk[i], rb[j][i], s);
      if (bt + j * C::NBT < C::NMU) mu_tab[e * C::NMU + bt + j * C::NBT] = s;
    }
  }
}

template <int P>
__global__ void __launch_bounds__(NhTcE<P>::NTH, 1) nh_tce_kernel(Req q, unsigned* err) {
  using C = NhTcE<P>;
  extern __shared__ __align__(16) char smem_raw[];
  if (C::SMEM > dynamic_smem_bytes()) {
    if (threadIdx.x == 0) flag_error(err, ERR_LAUNCH);
    return;
  }
  char* sm = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
  NhTcEBars* bars = reinterpret_cast<NhTcEBars*>(sm + C::O_BAR);
  float* sW = reinterpret_cast<float*>(sm + C::O_W);
  float* sD = reinterpret_cast<float*>(sm + C::O_DPHI);
  volatile int64_t* ring = reinterpret_cast<volatile int64_t*>(sm + C::O_RING);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t ntiles = (q.E + C::TE - 1) / C::TE;
  const float* tab = static_cast<const float*>(q.tab);
  const TcETabLayout L = tce_tab_layout(C::Q, C::NS);
  const float mu_c = d2f(q.coeffs[q.E * C::CLEN]), lam_c = d2f(q.coeffs[q.E * C::CLEN + 1]);
  const float nan = __int_as_float(0x7fc00000);

  if (tid == 0) {
    for (int i = 0; i < 3; ++i) {
      mbar_init(&bars->geo_full[i], 1);
      mbar_init(&bars->geo_empty[i], 4);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&bars->in_full[i], 1);
      mbar_init(&bars->pw_full[i], 4);
      mbar_init(&bars->pw_empty[i], C::NBT / 32);
      mbar_init(&bars->d_full[i], 1);
      mbar_init(&bars->d_empty[i], 8);
      mbar_init(&bars->mu_full[i], C::NBT / 32);
    }
    for (int i = 0; i < C::TE; ++i) {
      mbar_init(&bars->op_full[i], C::NBT / 32);
      mbar_init(&bars->op_empty[i], 1);
    }
    mbar_init(&bars->done, 1);
    fence_barrier_init();
  }
  for (int i = tid; i < C::Q; i += C::NTH) sW[i] = tab[L.offW + i];
  for (int i = tid; i < C::Q * C::RS; i += C::NTH) {
    const int qq = i / C::RS, j = i - qq * C::RS;
    if (j >= C::N3) sD[i] = 0.f;
  }
  {
    // operands (their zero padding rows stay zero), staging and u rows
    uint4* z = reinterpret_cast<uint4*>(sm);
    for (int i = tid; i < (int)(C::O_MU / 16); i += C::NTH) z[i] = make_uint4(0u, 0u, 0u, 0u);
    float* u = reinterpret_cast<float*>(sm + C::O_UT);
    for (int i = tid; i < C::NGB * C::TE * C::RU; i += C::NTH) u[i] = 0.f;
  }
  __syncthreads();
  for (int i = tid; i < C::Q * C::N3; i += C::NTH) {  // dPhi_a^k at node_slot(a, k)
    const int qq = i / C::N3, r = i - qq * C::N3;
    sD[qq * C::RS + C::node_slot(r / 3, r % 3)] = tab[L.offDphi + i];
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

  if (warp == 0) {
    // ------------------------------------------------------------- MMA issue
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_f16kind(1u, 128u, (uint32_t)C::NCOL);
      const uint32_t op0 = smem_addr(sm + C::O_OP);
      bool ok = true;
      for (int it = 0;; ++it) {
        const int buf = it & 1;
        ok = it < 2 || mbar_wait_sleep(&bars->d_empty[buf], (unsigned)(((it >> 1) - 1) & 1));
        if (ok) ok = mbar_wait_sleep(&bars->op_full[0], (unsigned)(it & 1));
        if (!ok) break;
        if (ring[it % C::NRING] < 0) {  // past the last tile: let the epilogue see it too
          tc_commit(&bars->d_full[buf]);
          break;
        }
        for (int e = 0; e < C::TE && ok; ++e) {
          if (e > 0) ok = mbar_wait_sleep(&bars->op_full[e], (unsigned)(it & 1));
          if (!ok) break;
          tc_fence_after();
          const uint32_t dt = tb + (uint32_t)(buf * C::TE + e) * C::NCOL;
          const uint32_t ahi = op0 + (uint32_t)e * C::OPSLOT, alo = ahi + C::OPB;
#pragma unroll
          for (int j = 0; j < C::KS; ++j)
            mma_f16_ss(dt, smem_desc_kmajor(ahi + 256u * j, C::LBO, C::SBO), smem_desc_kmajor(ahi + 256u * j, C::LBO, C::SBO),
                       idesc, j > 0 ? 1u : 0u);
#pragma unroll
          for (int j = 0; j < C::KS; ++j)
            mma_f16_ss(dt, smem_desc_kmajor(ahi + 256u * j, C::LBO, C::SBO), smem_desc_kmajor(alo + 256u * j, C::LBO, C::SBO),
                       idesc, 1u);
#pragma unroll
          for (int j = 0; j < C::KS; ++j)
            mma_f16_ss(dt, smem_desc_kmajor(alo + 256u * j, C::LBO, C::SBO), smem_desc_kmajor(ahi + 256u * j, C::LBO, C::SBO),
                       idesc, 1u);
          tc_commit(&bars->op_empty[e]);
        }
        if (!ok) break;
        tc_commit(&bars->d_full[buf]);
      }
      if (!ok) flag_error(err, ERR_TIMEOUT);
      tc_commit(&bars->done);
      if (!mbar_wait_sleep(&bars->done, 0u)) flag_error(err, ERR_TIMEOUT);
    }
    __syncwarp();
  } else if (warp < C::W_KIN) {
    // -------------------------------------------------------------- geometry
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
    // lane 0: the tile of this CTA's next iteration, -1 past the last one (draws are monotonic)
    bool drawn_out = false;
    int64_t next_static = blockIdx.x;
    auto draw = [&]() -> int64_t {
      if (drawn_out) return -1;
      const int64_t t = q.tile_ctr ? (int64_t)atomicAdd(q.tile_ctr, 1ull) : next_static;
      next_static += gridDim.x;
      if (t >= ntiles) {
        drawn_out = true;
        return -1;
      }
      return t;
    };
    int pend0 = -1, pend1 = -1;  // iteration whose input copy is in flight, per buffer (lane 0)
    if (lane == 0) {
      const int64_t t0 = draw();
      ring[0] = t0;
      if (t0 >= 0 && issue_inputs(t0, 0)) pend0 = 0;
      const int64_t t1 = draw();
      ring[1] = t1;
      if (t1 >= 0 && issue_inputs(t1, 1)) pend1 = 1;
    }
    __syncwarp();
    bool ok = true;
    for (int it = 0;; ++it) {
      const int64_t t = ring[it % C::NRING];
      const int b = it & 1, gb = it % 3;
      unsigned w = 1;
      if (lane == 0) {
        if (t >= 0) w = mbar_wait_sleep(&bars->in_full[b], (unsigned)((it >> 1) & 1));
        if (w && it >= 3) w = mbar_wait_sleep(&bars->geo_empty[gb], (unsigned)((it / 3 - 1) & 1));
      }
      ok = __shfl_sync(0xffffffffu, w, 0) != 0;
      if (!ok) break;
      if (t < 0) {
        // past the last tile: both kinematics groups learn it (this iteration and the next)
        if (lane == 0) {
          mbar_arrive(&bars->geo_full[gb]);
          const int i1 = it + 1;
          w = i1 < 3 || mbar_wait_sleep(&bars->geo_empty[i1 % 3], (unsigned)((i1 / 3 - 1) & 1));
          ring[i1 % C::NRING] = -1;
          if (w) mbar_arrive(&bars->geo_full[i1 % 3]);
        }
        ok = __shfl_sync(0xffffffffu, w, 0) != 0;
        break;
      }
      const int64_t e0 = t * C::TE;
      const int ne = (int)(q.E - e0 < C::TE ? q.E - e0 : C::TE);
      if (lane == 0) (b ? pend1 : pend0) = -1;
      const double* xs = reinterpret_cast<const double*>(sm + C::O_IN + (size_t)b * C::IN_BUF);
      const double* us = xs + C::TE * 12;
      float* ut = reinterpret_cast<float*>(sm + C::O_UT) + gb * C::TE * C::RU;
      float* geo = reinterpret_cast<float*>(sm + C::O_GEO) + gb * C::TE * 24;
      for (int i = lane; i < ne * C::CLEN; i += 32) {
        const int e = i / C::CLEN;
        const int r = i - e * C::CLEN;  // displacement DOF u_a[c] at 3 a + c, to its node-pair slot
        ut[e * C::RU + C::node_slot(r / 3, r % 3)] = d2f_rz(us[i]);
      }
      if (lane < ne) {  // FP64 geometry of element `lane`
        double adj[9];
        const double det = geometry_fp64(xs + 12 * lane, adj);
        const uint64_t bits = (uint64_t)__double_as_longlong(det);
        const bool bad = ((bits << 1) == 0) || ((bits >> 52 & 0x7ff) == 0x7ff);
        if (bad) flag_error(err, ERR_DEGENERATE);
        const float df = d2f_rz(det), inv = 1.0f / df;
        float Ji[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) Ji[k] = d2f_rz(adj[k]) * inv;
        float* g = geo + 24 * lane;
#pragma unroll
        for (int k = 0; k < 9; ++k) g[k] = bad ? nan : Ji[k];
        g[9] = bad ? nan : fabsf(df);
        const float mdet = mu_c * fabsf(df);  // mu |det J| (J^-1 J^-T)[k][l], k <= l
        int i6 = 0;
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
          for (int l = k; l < 3; ++l, ++i6)
            g[12 + i6] = bad ? nan : mdet * (Ji[3 * k] * Ji[3 * l] + Ji[3 * k + 1] * Ji[3 * l + 1] + Ji[3 * k + 2] * Ji[3 * l + 2]);
      }
      __syncwarp();
      if (lane == 0) {
        // the input buffer has been read: draw the tile two iterations ahead and prefetch it into it
        const int64_t t2 = draw();
        ring[(it + 2) % C::NRING] = t2;
        if (t2 >= 0) {
          fence_proxy_async();
          if (issue_inputs(t2, b)) (b ? pend1 : pend0) = it + 2;
        }
        mbar_arrive(&bars->geo_full[gb]);
      }
      __syncwarp();
    }
    if (!ok) flag_error(err, ERR_TIMEOUT);
    // copies issued before giving up must land before the CTA leaves
    if (lane == 0) {
      if (pend0 >= 0) mbar_wait_sleep(&bars->in_full[0], (unsigned)((pend0 >> 1) & 1));
      if (pend1 >= 0) mbar_wait_sleep(&bars->in_full[1], (unsigned)((pend1 >> 1) & 1));
    }
  } else if (warp < C::W_BLD) {
    // ------------------------------------------------------------ kinematics
    const int gk = (warp - C::W_KIN) >> 2;  // group gk takes the iterations gk, gk + 2, ... (pointwise slot gk)
    const int kt = tid - 32 * C::W_KIN - 128 * gk;
    const int bar_id = C::BAR_KIN + gk;
    float* pw = reinterpret_cast<float*>(sm + C::O_PW + (size_t)gk * C::PW_SLOT);
    float* pwk = pw + C::TE * C::PW_E;
    bool ok = true;
    for (int it = gk;; it += 2) {
      const int gb = it % 3;
      const float* ut = reinterpret_cast<const float*>(sm + C::O_UT) + gb * C::TE * C::RU;
      const float* geo = reinterpret_cast<const float*>(sm + C::O_GEO) + gb * C::TE * 24;
      bool w = mbar_wait_sleep(&bars->geo_full[gb], (unsigned)((it / 3) & 1));
      if (w && it >= 2) w = mbar_wait_sleep(&bars->pw_empty[gk], (unsigned)(((it >> 1) - 1) & 1));
      ok = named_and(bar_id, 128, w);
      if (!ok) break;
      const int64_t t = ring[it % C::NRING];
      if (t < 0) {  // past the last tile: pass it on to the operand warps
        if (lane == 0) mbar_arrive(&bars->pw_full[gk]);
        break;
      }
      const int64_t e0 = t * C::TE;
      const int ne = (int)(q.E - e0 < C::TE ? q.E - e0 : C::TE);
      if (kt < ne * 6) pwk[8 * (kt / 6) + kt % 6] = geo[24 * (kt / 6) + 12 + kt % 6];
      for (int w2 = kt; w2 < ne * C::Q; w2 += 128) {
        const int e = w2 / C::Q, qq = w2 - e * C::Q;
        // gr[3 i + k] = sum_a u_a[i] dPhi_a^k, two nodes at a time (packed), even and odd nodes summed last
        float2 acc[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) acc[k] = make_float2(0.f, 0.f);
        const float4* u4 = reinterpret_cast<const float4*>(ut + C::RU * e);
        const float4* d4 = reinterpret_cast<const float4*>(sD + C::RS * qq);
#pragma unroll
        for (int v = 0; v < C::N3 / 12; ++v) {  // two node pairs: 12 floats of u and of dPhi
          float uv[12], dv[12];
#pragma unroll
          for (int j = 0; j < 3; ++j) {
            const float4 uu = u4[3 * v + j], dd = d4[3 * v + j];
            uv[4 * j] = uu.x; uv[4 * j + 1] = uu.y; uv[4 * j + 2] = uu.z; uv[4 * j + 3] = uu.w;
            dv[4 * j] = dd.x; dv[4 * j + 1] = dd.y; dv[4 * j + 2] = dd.z; dv[4 * j + 3] = dd.w;
          }
#pragma unroll
          for (int np = 0; np < 2; ++np)
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
              for (int k = 0; k < 3; ++k)
                acc[3 * i + k] = __ffma2_rn(make_float2(uv[6 * np + 2 * i], uv[6 * np + 2 * i + 1]),
                                            make_float2(dv[6 * np + 2 * k], dv[6 * np + 2 * k + 1]), acc[3 * i + k]);
        }
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
        // is a well-conditioned scaling done after rounding to FP32; sqrt(s) rides on 1 / det F
        const float rs = __fsqrt_rn(sW[qq] * J[9]);
        const float idF = __frcp_rn(d2f_rz(dF)) * rs;
        const float lnJ = d2f_rz(log_f64(dF));
        float Fi[9];  // Fi[3 I + c] = sqrt(s) (F^-1)[I][c]
#pragma unroll
        for (int k = 0; k < 9; ++k) Fi[k] = d2f_rz(cof[k]) * idF;
        const float al = mu_c - lam_c * lnJ;
        float* rec = pw + e * C::PW_E + (qq >> 3) * C::PW_O + (qq & 7);
        rec[0] = bad ? nan : al;
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int k = 0; k < 3; ++k)  // M'[c][k] = sum_I sqrt(s) (F^-1)[I][c] (J^-1)[k][I]
            rec[8 + 8 * (3 * c + k)] = bad ? nan : Fi[c] * J[3 * k] + Fi[3 + c] * J[3 * k + 1] + Fi[6 + c] * J[3 * k + 2];
      }
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&bars->pw_full[gk]);
        mbar_arrive(&bars->geo_empty[gb]);
      }
    }
    if (!ok) flag_error(err, ERR_TIMEOUT);
  } else if (warp < C::W_EPI) {
    // -------------------------------------------------------------- operands
    const int bt = tid - 32 * C::W_BLD;        // 0 .. NBT - 1
    const int a = bt % C::NS, o = bt / C::NS;  // basis function a, points 8 o .. 8 o + 7
    float2 dp[3][4];                           // dPhi_a^k at the octet's points, in pairs
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int j = 0; j < 4; ++j)
        dp[k][j] = make_float2(sD[(8 * o + 2 * j) * C::RS + C::node_slot(a, k)],
                               sD[(8 * o + 2 * j + 1) * C::RS + C::node_slot(a, k)]);
    float* mu_tab = reinterpret_cast<float*>(sm + C::O_MU);
    bool ok = true;
    for (int it = 0;; ++it) {
      const int slot = it & 1, buf = it & 1;
      unsigned w = 1;
      if (lane == 0) w = mbar_wait_sleep(&bars->pw_full[slot], (unsigned)((it >> 1) & 1));
      ok = __shfl_sync(0xffffffffu, w, 0) != 0;
      if (!ok) break;
      const int64_t t = ring[it % C::NRING];
      if (t < 0) {
        // past the last tile: pass it on to the MMA warp (operand slot 0) and to the epilogue
        // (Mu table), each after the wait that keeps the barrier phases in step
        if (lane == 0) {
          w = it < 1 || mbar_wait_sleep(&bars->op_empty[0], (unsigned)((it - 1) & 1));
          if (w) mbar_arrive(&bars->op_full[0]);
          if (w) w = it < 2 || mbar_wait_sleep(&bars->d_empty[buf], (unsigned)(((it >> 1) - 1) & 1));
          if (w) mbar_arrive(&bars->mu_full[buf]);
        }
        ok = __shfl_sync(0xffffffffu, w, 0) != 0;
        break;
      }
      const int64_t e0 = t * C::TE;
      const int ne = (int)(q.E - e0 < C::TE ? q.E - e0 : C::TE);
      const float* pw = reinterpret_cast<const float*>(sm + C::O_PW + (size_t)slot * C::PW_SLOT);
      for (int e = 0; e < C::TE; ++e) {
        if (lane == 0 && it >= 1) w = mbar_wait_sleep(&bars->op_empty[e], (unsigned)((it - 1) & 1));
        ok = __shfl_sync(0xffffffffu, w, 0) != 0;
        if (!ok) break;
        if (e < ne)
          nh_tce_build<P>(reinterpret_cast<const float4*>(pw + e * C::PW_E + o * C::PW_O),
                          sm + C::O_OP + (size_t)e * C::OPSLOT, dp, a, o);
        fence_proxy_async();
        __syncwarp();
        if (lane == 0) mbar_arrive(&bars->op_full[e]);
      }
      if (!ok) break;
      // the Mu table of this accumulator buffer is free once the epilogue of two tiles ago is done
      if (lane == 0 && it >= 2) w = mbar_wait_sleep(&bars->d_empty[buf], (unsigned)(((it >> 1) - 1) & 1));
      ok = __shfl_sync(0xffffffffu, w, 0) != 0;
      if (!ok) break;
      nh_tce_mu<P>(tab + L.offRbar, pw + C::TE * C::PW_E, mu_tab + buf * C::TE * C::NMU, bt, ne);
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&bars->mu_full[buf]);
        mbar_arrive(&bars->pw_empty[slot]);
      }
    }
    if (!ok) flag_error(err, ERR_TIMEOUT);
  } else {
    // -------------------------------------------------------------- epilogue
    const int set = (warp - C::W_EPI) >> 2;  // elements 2 set, 2 set + 1 of every tile
    const int et = tid - 32 * C::W_EPI - 128 * set;
    const int bar = C::BAR_EPI + set;
    const int qd = warp & 3, m = 32 * qd + lane;
    const bool srow = m < C::N3, trow = m >= 64 && m < 64 + C::N3;
    const int r = srow ? m : (trow ? m - 64 : 0), ra = r / 3, rx = r - 3 * ra;
    float* stage = reinterpret_cast<float*>(sm + C::O_STAGE + (size_t)set * C::STAGE_B);
    const float* mu_tab = reinterpret_cast<const float*>(sm + C::O_MU);
    const uint32_t tlane = tb + ((uint32_t)(32 * qd) << 16);
    // this thread's pairs of output entries k = et + 128 m: staging offset of the first; each
    // next one lies 128 pairs = 4 rows + 16 entries further on
    constexpr int NP = C::NN / 2, NM = (NP + 127) / 128, HM = (NM + 1) / 2;
    static_assert(C::N3 == 60, "pair stepping of the output loop");
    const int soff0 = (et / 30) * C::LD + 2 * (et % 30);
    bool ok = true;
    for (int it = 0;; ++it) {
      const int buf = it & 1;
      bool w = mbar_wait_sleep(&bars->d_full[buf], (unsigned)((it >> 1) & 1));
      if (w) w = mbar_wait_sleep(&bars->mu_full[buf], (unsigned)((it >> 1) & 1));
      ok = named_and(bar, 128, w);
      if (!ok) break;
      const int64_t t = ring[it % C::NRING];
      if (t < 0) break;  // past the last tile
      const int64_t e0 = t * C::TE;
      const int ne = (int)(q.E - e0 < C::TE ? q.E - e0 : C::TE);
      tc_fence_after();
#pragma unroll 1
      for (int j = 0; j < 2; ++j) {
        const int el = 2 * set + j;
        const uint32_t dcol = tlane + (uint32_t)(buf * C::TE + el) * C::NCOL;
        // (1) T rows: T[(a,x),(b,y)] -> A[(a,y),(b,x)], a bijection of the staging entries
        if (el < ne && qd >= 2) {
#pragma unroll
          for (int ch = 0; ch < (C::N3 + 15) / 16; ++ch) {
            uint32_t v[16];
            tmem_ld16(dcol + 16u * ch, v);
            tmem_wait_ld();
            if (trow) {
#pragma unroll
              for (int jj = 0; jj < 16; ++jj) {
                const int n = 16 * ch + jj;
                if (n < C::N3) stage[(3 * ra + n % 3) * C::LD + 3 * (n / 3) + rx] = __uint_as_float(v[jj]);
              }
            }
          }
        }
        named_sync(bar, 128);
        // (2) S rows: A[(a,c),(b,d)] += lam S[(a,c),(b,d)] + delta_cd Mu[a][b]; a chunk's staging
        // entries and Mu values are loaded before any of its stores
        if (el < ne && qd < 2) {
          const float* mu = mu_tab + (buf * C::TE + el) * C::NMU + ra * C::NS;
          float* srow_p = stage + r * C::LD;
#pragma unroll
          for (int ch = 0; ch < (C::N3 + 15) / 16; ++ch) {
            uint32_t v[16];
            tmem_ld16(dcol + 16u * ch, v);
            float sv[16], mv[6];
            if (srow) {
#pragma unroll
              for (int jj = 0; jj < 16; ++jj)
                if (16 * ch + jj < C::N3) sv[jj] = srow_p[16 * ch + jj];
#pragma unroll
              for (int bb = 0; bb < 6; ++bb) {
                const int b = (16 * ch) / 3 + bb;
                mv[bb] = b < C::NS ? mu[b] : 0.f;
              }
            }
            tmem_wait_ld();
            if (srow) {
#pragma unroll
              for (int jj = 0; jj < 16; ++jj) {
                const int n = 16 * ch + jj;
                if (n < C::N3)
                  srow_p[n] = sv[jj] + fmaf(lam_c, __uint_as_float(v[jj]), n % 3 == rx ? mv[n / 3 - (16 * ch) / 3] : 0.f);
              }
            }
          }
        }
        if (j == 1) {  // this set's last reads of the accumulator buffer: hand it back
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&bars->d_empty[buf]);
        }
        named_sync(bar, 128);
        // (3) coalesced stores of the element matrix: all of this thread's pairs loaded first
        if (el < ne) {
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            float2 v[HM];
            int so = soff0, jc = 2 * (et % 30);
#pragma unroll
            for (int mm = 0; mm < NM; ++mm) {
              if (mm >= h * HM && mm < (h + 1) * HM && et + 128 * mm < NP)
                v[mm - h * HM] = *reinterpret_cast<const float2*>(stage + so);
              so += 4 * C::LD + 16;
              jc += 16;
              if (jc >= C::N3) {
                jc -= C::N3;
                so += C::LD - C::N3;
              }
            }
            if (q.out_f32) {
              float2* o2 = reinterpret_cast<float2*>(static_cast<float*>(q.out) + (e0 + el) * C::NN) + et;
#pragma unroll
              for (int mm = h * HM; mm < (h + 1) * HM && mm < NM; ++mm)
                if (et + 128 * mm < NP) __stcs(o2 + 128 * mm, v[mm - h * HM]);
            } else {
              double2* o2 = reinterpret_cast<double2*>(static_cast<double*>(q.out) + (e0 + el) * C::NN) + et;
#pragma unroll
              for (int mm = h * HM; mm < (h + 1) * HM && mm < NM; ++mm)
                if (et + 128 * mm < NP) __stcs(o2 + 128 * mm, make_double2(f2d_ftz(v[mm - h * HM].x), f2d_ftz(v[mm - h * HM].y)));
            }
          }
        }
        named_sync(bar, 128);
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
