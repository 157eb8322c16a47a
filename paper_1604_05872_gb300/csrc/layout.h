// Constants and layouts shared by the host planner and the device kernels.
#pragma once
#include <cstddef>
#include <cstdint>

#ifdef __CUDACC__
#define FEA_HD __host__ __device__
#else
#define FEA_HD
#endif

namespace fea {

constexpr int NT = 256;  // threads per CTA of every tile function

FEA_HD constexpr int nbasis_c(int p) { return (p + 1) * (p + 2) * (p + 3) / 6; }
FEA_HD constexpr int ncomp_c(int form) { return (form == 2 || form == 3) ? 3 : 1; }
FEA_HD constexpr int coeff_len_c(int form, int p) {
  return form == 0 ? 0 : form == 1 ? nbasis_c(p) : form == 2 ? 8 : 3 * nbasis_c(p);
}
FEA_HD constexpr int pre_terms_c(int form, int p) {
  return form == 0 ? 1 : form == 1 ? 6 + nbasis_c(p) : form == 2 ? 36 : 0;
}
FEA_HD constexpr int round_up(int x, int m) { return (x + m - 1) / m * m; }
FEA_HD constexpr size_t round_up_sz(size_t x, size_t m) { return (x + m - 1) / m * m; }

// Device table of one (form, degree, precision): W [Q], phi [Q][ns],
// dphi [Q][ns][3], phi1 [Q][4], R [r][ns][ns]; every section starts on a
// multiple of 4 entries (16 bytes for float, 32 for double).
struct TabLayout {
  int Q, ns, r;
  int offW, offPhi, offDphi, offPhi1, offR, total;
};
FEA_HD inline TabLayout tab_layout(int Q, int ns, int r) {
  TabLayout t{};
  t.Q = Q;
  t.ns = ns;
  t.r = r;
  t.offW = 0;
  t.offPhi = round_up(Q, 4);
  t.offDphi = t.offPhi + round_up(Q * ns, 4);
  t.offPhi1 = t.offDphi + round_up(Q * ns * 3, 4);
  t.offR = t.offPhi1 + round_up(Q * 4, 4);
  t.total = t.offR + round_up(r * ns * ns, 4);
  return t;
}

// Pair p of the upper triangle a <= b of an n x n grid of blocks, row by row:
// (0,0), (0,1), ..., (0,n-1), (1,1), ...
FEA_HD inline void sym_pair(int p, int n, int* a, int* b) {
  int aa = 0;
  while (aa < n && p >= n - aa) {
    p -= n - aa;
    ++aa;
  }
  *a = aa;
  *b = aa + p;
}

// Device table of the tensor-core Neo-Hookean kernel, in 32-bit words: W [Q],
// dphi [Q][ns][3] (float), then the split reference tables R_stack [128][K / 2]
// (packed 16-bit pairs; row 2p = hi, 2p + 1 = lo part of the pair p = (a, b)).
struct TcTabLayout {
  int offW, offDphi, offR, total;
};
FEA_HD inline TcTabLayout tc_tab_layout(int Q, int ns, int K) {
  TcTabLayout t{};
  t.offW = 0;
  t.offDphi = round_up(Q, 4);
  t.offR = t.offDphi + round_up(Q * ns * 3, 4);
  t.total = t.offR + 128 * (K / 2);
  return t;
}

// One assembly request as the kernels see it.
struct Req {
  const double* coords;
  const double* coeffs;
  void* out;
  const void* tab;   // device table, float or double
  int64_t E;
  int form, p, Q;
  int tile;          // elements per tile (even)
  int out_f32;
  int kind;          // kernel kind (batch dispatch)
  int64_t tile0;     // first global tile of this request (batch)
  int64_t skip_copy; // test hook: 1 + the global tile whose input copy is skipped (0: none)
  unsigned long long* tile_ctr;  // tiles handed out by an atomic counter zeroed before the launch
                                 // (kernels that support it), or null: tiles blockIdx.x + k gridDim.x
};

// Global assembly target of the one-pass kernel: the CSR values of the global
// matrix and, per element entry (e, i, j), its position in them (int32 or int64).
struct ScatterArgs {
  const void* map;
  int64_t nnz;
  double* values;
};

enum Variant { V_NAIVE = 0, V_SE = 1, V_PRE = 2 };

}  // namespace fea
