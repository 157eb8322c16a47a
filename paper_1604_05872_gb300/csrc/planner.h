// Host planner: operation counts of the loop-nest variants, the transformation
// algorithm's choice between sharing elimination and pre-evaluation, tile
// selection, and tuned overrides.
#pragma once
#include <cstddef>
#include <cstdint>

#include "kernels.h"

namespace fea {

struct Plan {
  const KernelInfo* k = nullptr;
  int variant = 0, prec = 1, tile = 0, Q = 0;
  size_t smem = 0;
  // the tile came from the planner's rule for a kernel whose thread layout does
  // not depend on it: a launch with fewer elements than SMs x tile may use a
  // smaller one, so that every SM gets work and a tile's latency chain shortens
  bool shrink_small = false;
};

// A launch resolved on the host (kernel, persistent grid, shared memory, request).
struct DevState;
struct PreparedLaunch {
  const void* fn = nullptr;
  unsigned grid = 0;
  int threads = NT;
  size_t smem = 0;
  Req q{};
  unsigned* err = nullptr;
  bool dyn = false;         // the kernel takes a tile counter (zeroed on the launch stream first)
  DevState* st = nullptr;   // owner of the per-stream tile counters
};

// Per-element operation counts (adds and products; an FMA counts 2) of the
// three loop nests as the kernels execute them.  pre = -1 when the form has no
// pre-evaluated form.
struct OpCounts {
  int64_t naive, se, pre;
};
OpCounts op_counts(int form, int p);

// Algorithm 3 (Section 4.1) on the form's monomials with the memory threshold
// T_H = `budget` bytes of shared memory: returns FEA_VARIANT_SE or _PRE.
// Tuned choices installed with set_tuned() take precedence.
int choose_variant(int form, int p, int prec, size_t budget, bool use_tuned = true);
int default_tile(int variant, int form, int p, int prec, int max_tile, size_t budget, int Q,
                 size_t (*smem)(int, int), bool use_tuned = true, int pref_tile = 0);

// Tuned overrides (autotuner / learned cost model), keyed by (form, p, prec).
void set_tuned(int form, int p, int prec, int variant, int tile);
bool get_tuned(int form, int p, int prec, int* variant, int* tile);
void clear_tuned();
int tuned_generation();  // changes whenever a tuned choice is installed or cleared

struct BatchState;
void free_batch_state(BatchState* b);

}  // namespace fea
