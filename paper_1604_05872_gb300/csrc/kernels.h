// Registry of compiled tile kernels (host side).
#pragma once
#include <cstddef>
#include <cstdint>

#include "layout.h"

namespace fea {

struct KernelInfo {
  const void* fn;                     // __global__ void (Req, unsigned*)
  int variant, form, p, prec;         // prec: 0 = FP64, 1 = FP32
  int max_tile;                       // upper bound on elements per tile
  size_t (*smem)(int TE, int Q);      // dynamic shared memory for a tile of TE
  int pref_tile;                      // tile the thread layout is built for (0: none)
  int threads = 0;                    // threads per CTA (0: NT)
  bool dyn_tiles = false;             // takes its tiles from Req::tile_ctr when one is given
};

// Registered by the kernel translation units.
extern const KernelInfo kPreKernels[];
extern const int kNumPreKernels;
extern const KernelInfo kSeKernels[];
extern const int kNumSeKernels;
extern const KernelInfo kNaiveKernels[];
extern const int kNumNaiveKernels;

// Tensor-core kernels (split-operand precisions): Neo-Hookean P2.
extern const KernelInfo kTcKernels[];
extern const int kNumTcKernels;

extern const KernelInfo kPreTileF32[];
extern const int kNumPreTileF32;

// The first registered kernel of (variant, form, degree, precision) whose
// one-element tile fits `budget` bytes of shared memory (any, if none does or
// budget is 0).
const KernelInfo* find_kernel(int variant, int form, int p, int prec, size_t budget = 0, int Q = 0);
// Tile functions of the batched persistent kernel (FP32): PreTile / SeTile.
const KernelInfo* find_batch_kernel(int variant, int form, int p);
// Element-vector kernels (linear forms): Helmholtz load vector, Neo-Hookean residual.
const KernelInfo* find_vec_kernel(int form, int p, int prec);
// The fused local + global assembly form of the streaming kernel `plain`
// (mass and Helmholtz P1-P3), with an int32 or int64 position map; nullptr if none.
const void* find_scatter_kernel(const void* plain, int map_i64);
// Combined global assembly target (pre_combine.cuh): the plan built by
// fea_csr_combine_plan (32-bit words; header magic kCombineMagic) and the CSR values.
constexpr int32_t kCombineMagic = 0x46435031;  // "FCP1"
struct CombineArgs {
  const int32_t* plan;
  int64_t plan_words;
  int64_t nnz;
  double* values;
};
// Elements per tile of the combining plan for local dimension n (min(128, 3200 / n^2), even).
int combine_tile(int n);
// The one-pass kernel with tile-combined atomics for (form, degree), and its
// shared memory at the combining tile; nullptr if none.
const void* find_combine_kernel(int form, int p, size_t* smem);

}  // namespace fea
