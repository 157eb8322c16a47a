// C ABI of the library (include/fea.h): argument checking, plans, device
// tables, launches, the host-buffer pipeline and the batched persistent launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/fea.h"
#include "host_model.h"
#include "kernels.h"
#include "planner.h"

namespace fea {

// The split-BF16 kernel of the pre-evaluated scalar forms (kernels_pretc.cu).
const KernelInfo* find_pretc_kernel(int form, int p);
bool is_pretc_kernel(const void* fn);
bool pretc_table_words(int form, int p, std::vector<uint32_t>* words);

bool tc_table_words(int form, int p, std::vector<uint32_t>* words);
bool bernstein_table_words(int form, int p, std::vector<uint32_t>* words);
const KernelInfo* find_tc_kernel(int form, int p);

static thread_local std::string g_last_error;
// test hook (fea_test_skip_input_copy): 1 + the tile whose input copy the next launch skips
static std::atomic<int64_t> g_skip_copy{0};
static int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}
#define CUDA_TRY(x)                                                                        \
  do {                                                                                     \
    cudaError_t e_ = (x);                                                                  \
    if (e_ != cudaSuccess) return fail(FEA_ECUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
  } while (0)

struct TableEntry {
  void* dev = nullptr;
  TabLayout lay{};
};

struct DevState {
  int dev = -1;
  int sms = 0;
  size_t smem_optin = 0;
  unsigned* err = nullptr;  // device error word
  std::map<std::tuple<int, int, int>, TableEntry> tables;
  // host-buffer pipeline workspace
  cudaStream_t hs[2] = {nullptr, nullptr};
  void* ws[2][3] = {{nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr}};
  size_t ws_bytes[2][3] = {{0, 0, 0}, {0, 0, 0}};
  // batch
  BatchState* batch = nullptr;
  // tile counters of the kernels that hand out tiles dynamically: one per stream that
  // launches them (launches on one stream run in order, so its counter is reset before
  // each and never shared with a launch in flight on another stream)
  static constexpr int kCounters = 64;
  unsigned long long* ctr = nullptr;
  std::map<cudaStream_t, int> ctr_slot;
};

static std::mutex g_mu;
static std::map<int, std::unique_ptr<DevState>> g_dev;

static int get_dev(DevState** out) {
  int dev = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_dev.find(dev);
  if (it == g_dev.end()) {
    auto st = std::make_unique<DevState>();
    st->dev = dev;
    cudaDeviceProp prop;
    CUDA_TRY(cudaGetDeviceProperties(&prop, dev));
    st->sms = prop.multiProcessorCount;
    st->smem_optin = prop.sharedMemPerBlockOptin;
    CUDA_TRY(cudaMalloc(&st->err, sizeof(unsigned)));
    CUDA_TRY(cudaMemset(st->err, 0, sizeof(unsigned)));
    CUDA_TRY(cudaMalloc(&st->ctr, DevState::kCounters * sizeof(unsigned long long)));
    CUDA_TRY(cudaMemset(st->ctr, 0, DevState::kCounters * sizeof(unsigned long long)));
    it = g_dev.emplace(dev, std::move(st)).first;
  }
  *out = it->second.get();
  return FEA_OK;
}

unsigned* device_error_word(DevState* st) { return st->err; }
int device_sms(DevState* st) { return st->sms; }
size_t device_smem_optin(DevState* st) { return st->smem_optin; }
int device_index(DevState* st) { return st->dev; }
int get_dev_state(DevState** out) { return get_dev(out); }
BatchState*& dev_batch(DevState* st) { return st->batch; }
int set_error(int code, const char* msg) { return fail(code, msg); }

// Device tables of (form, degree, precision), built and uploaded once.
int get_tables(DevState* st, int form, int p, int prec, TableEntry** out) {
  std::lock_guard<std::mutex> lk(g_mu);
  auto key = std::make_tuple(form, p, prec);
  auto it = st->tables.find(key);
  if (it == st->tables.end() && (prec == 2 || prec == 3)) {
    // 32-bit word tables: the tensor-core kernels (2) and the Bernstein variant (3)
    std::vector<uint32_t> words;
    if (prec == 2 && !tc_table_words(form, p, &words) && !pretc_table_words(form, p, &words))
      return fail(FEA_EINVAL, "no tensor-core table for this form/degree");
    if (prec == 3 && !bernstein_table_words(form, p, &words)) return fail(FEA_EINVAL, "no Bernstein table for this form/degree");
    TableEntry te;
    te.lay.total = (int)words.size();
    const size_t bytes = words.size() * 4;
    if (cudaMalloc(&te.dev, bytes) != cudaSuccess) return fail(FEA_ENOMEM, "table allocation failed");
    const cudaError_t e = cudaMemcpy(te.dev, words.data(), bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(FEA_ECUDA, std::string("table upload: ") + cudaGetErrorString(e));
    it = st->tables.emplace(key, te).first;
  }
  if (it == st->tables.end()) {
    Tables t = make_tables(form, p);
    TableEntry te;
    te.lay = tab_layout(t.Q, t.ns, t.r);
    std::vector<double> h(te.lay.total, 0.0);
    for (int q = 0; q < t.Q; ++q) h[te.lay.offW + q] = t.W[q];
    for (size_t k = 0; k < t.phi.size(); ++k) h[te.lay.offPhi + k] = t.phi[k];
    for (size_t k = 0; k < t.dphi.size(); ++k) h[te.lay.offDphi + k] = t.dphi[k];
    for (size_t k = 0; k < t.phi1.size(); ++k) h[te.lay.offPhi1 + k] = t.phi1[k];
    for (size_t k = 0; k < t.R.size(); ++k) h[te.lay.offR + k] = t.R[k];
    size_t bytes = (size_t)te.lay.total * (prec == 0 ? 8 : 4);
    if (cudaMalloc(&te.dev, bytes) != cudaSuccess) return fail(FEA_ENOMEM, "table allocation failed");
    cudaError_t e;
    if (prec == 0) {
      e = cudaMemcpy(te.dev, h.data(), bytes, cudaMemcpyHostToDevice);
    } else {
      std::vector<float> hf(h.begin(), h.end());
      e = cudaMemcpy(te.dev, hf.data(), bytes, cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) return fail(FEA_ECUDA, std::string("table upload: ") + cudaGetErrorString(e));
    it = st->tables.emplace(key, te).first;
  }
  *out = &it->second;
  return FEA_OK;
}

// Lookups that never create anything: the device state and the FP32 tables of
// (form, p) if an earlier call on the current device made them, else NULL.
DevState* existing_dev_state() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_dev.find(dev);
  return it == g_dev.end() ? nullptr : it->second.get();
}
const void* existing_table(DevState* st, int form, int p, int prec) {
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = st->tables.find(std::make_tuple(form, p, prec));
  return it == st->tables.end() ? nullptr : it->second.dev;
}

const void* table_ptr(DevState* st, int form, int p, int prec, int* rc) {
  TableEntry* te = nullptr;
  *rc = get_tables(st, form, p, prec, &te);
  return *rc ? nullptr : te->dev;
}

static fea_options default_options() {
  fea_options o;
  o.precision = FEA_PREC_FP32;
  o.out_f32 = 0;
  o.variant = FEA_VARIANT_AUTO;
  o.tile = 0;
  o.smem_budget = 0;
  return o;
}

static bool valid_fd(int form, int p) { return form >= 0 && form <= 3 && p >= 1 && p <= 4; }

// Resolve variant, kernel and tile for a request.  Plans are cached: planning
// runs Algorithm 3 (expression rewriting and counting), far too slow to repeat
// on every launch.
static int make_plan_uncached(DevState* st, int form, int p, const fea_options& o, Plan* pl, bool batch,
                              bool use_tuned);

int make_plan(DevState* st, int form, int p, const fea_options& o, Plan* pl, bool batch, bool use_tuned);
int make_plan(DevState* st, int form, int p, const fea_options& o, Plan* pl, bool batch) {
  return make_plan(st, form, p, o, pl, batch, true);
}

int make_plan(DevState* st, int form, int p, const fea_options& o, Plan* pl, bool batch, bool use_tuned) {
  static std::mutex mu;
  static std::map<std::vector<int64_t>, Plan> cache;
  const std::vector<int64_t> key = {form, p, o.precision, o.out_f32, o.variant, o.tile, (int64_t)o.smem_budget,
                                    batch ? 1 : 0, st ? (int64_t)st->smem_optin : -1,
                                    use_tuned ? tuned_generation() : -1};
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(key);
    if (it != cache.end()) {
      *pl = it->second;
      return FEA_OK;
    }
  }
  int rc = make_plan_uncached(st, form, p, o, pl, batch, use_tuned);
  if (rc == FEA_OK) {
    std::lock_guard<std::mutex> lk(mu);
    cache[key] = *pl;
  }
  return rc;
}

static int make_plan_uncached(DevState* st, int form, int p, const fea_options& o, Plan* pl, bool batch,
                              bool use_tuned) {
  if (!valid_fd(form, p)) return fail(FEA_EINVAL, "unsupported form/degree");
  if (o.precision != FEA_PREC_FP64 && o.precision != FEA_PREC_FP32 && o.precision != FEA_PREC_BF16X2)
    return fail(FEA_EINVAL, "unsupported precision");
  // split-BF16 tensor-core contraction where a kernel exists and the contraction is
  // compute-bound: the Neo-Hookean tangent, and the pre-evaluated scalar forms with
  // FP32 output (with FP64 output they are bound by HBM); the rest run the FP32 contraction
  const bool scalar = form == FEA_MASS || form == FEA_HELMHOLTZ;
  const KernelInfo* tc = nullptr;
  if (o.precision == FEA_PREC_BF16X2 && !batch)
    tc = scalar ? (o.out_f32 == 1 ? find_pretc_kernel(form, p) : nullptr) : find_tc_kernel(form, p);
  const int prec = o.precision == FEA_PREC_FP64 ? 0 : 1;
  const size_t limit = st ? st->smem_optin : 232448;
  const size_t budget = o.smem_budget ? std::min(o.smem_budget, limit) : limit;
  int variant = o.variant;
  if (variant == FEA_VARIANT_AUTO) variant = choose_variant(form, p, prec, budget, use_tuned);
  if (variant == FEA_VARIANT_NAIVE && prec != 0) return fail(FEA_EINVAL, "the plain variant is FP64 only");
  if (variant == FEA_VARIANT_PRE && pre_terms(form, p) == 0)
    return fail(FEA_EINVAL, "pre-evaluation does not apply to this form (integrand not polynomial)");
  const int Q = rule_points(rule_index(form, p));
  const KernelInfo* k = batch ? find_batch_kernel(variant, form, p) : find_kernel(variant, form, p, prec, budget, Q);
  if (tc && variant == tc->variant) k = tc;
  if (!k) return fail(FEA_EINVAL, "no kernel for this variant/form/degree/precision");
  int TE = o.tile;
  if (TE < 0) return fail(FEA_EINVAL, "negative tile");
  // tuned tiles were measured on the standalone kernels; the batch keeps its own rule
  if (k == tc) {
    // the tensor-core kernel's layout fixes its tile (its accumulator columns per element)
    if (TE != 0 && TE != tc->pref_tile)
      return fail(FEA_EINVAL, "the tensor-core kernel runs tiles of exactly " + std::to_string(tc->pref_tile) + " elements");
    TE = tc->pref_tile;
  }
  if (TE == 0) TE = default_tile(variant, form, p, prec, k->max_tile, budget, Q, k->smem, use_tuned && !batch, k->pref_tile);
  if (TE < 1 || TE > k->max_tile) return fail(FEA_EINVAL, "tile out of range for this kernel");
  const size_t smem = k->smem(TE, Q);
  if (smem > budget) return fail(FEA_EINVAL, "tile does not fit the shared-memory budget (Constraint 2)");
  pl->k = k;
  pl->variant = variant;
  pl->prec = k->prec;
  pl->tile = TE;
  pl->Q = Q;
  pl->smem = smem;
  pl->shrink_small = o.tile == 0 && !batch && k->pref_tile == 0;
  return FEA_OK;
}

int check_device_ptr(const void* p, const char* what, bool allow_null) {
  if (!p) return allow_null ? FEA_OK : fail(FEA_EINVAL, std::string(what) + " is NULL");
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(FEA_EINVAL, std::string(what) + " is not a device pointer");
  }
  if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
    return fail(FEA_EINVAL, std::string(what) + " is a host pointer (device memory required; no CPU fallback)");
  int dev = 0;
  cudaGetDevice(&dev);
  if (a.type == cudaMemoryTypeDevice && a.device != dev)
    return fail(FEA_EINVAL, std::string(what) + " belongs to another device");
  if (reinterpret_cast<uintptr_t>(p) & 15) return fail(FEA_EINVAL, std::string(what) + " is not 16-byte aligned");
  return FEA_OK;
}

// Everything a launch of plan `pl` needs, resolved on the host: tables resident,
// the kernel's shared-memory ceiling raised, the persistent grid sized from
// its occupancy.  No stream work (usable before a graph capture).
int prepare_launch(DevState* st, const Plan& pl, int form, int p, int64_t E, const double* coords,
                   const double* coeffs, void* out, int out_f32, PreparedLaunch* L) {
  TableEntry* te = nullptr;
  int rc = get_tables(st, form, p, pl.prec, &te);
  if (rc) return rc;
  int tile = pl.tile;
  size_t smem_bytes = pl.smem;
  if (pl.shrink_small && st->sms > 0) {
    // fewer elements than one tile per SM: whole-warp tiles of about E / SMs elements
    const int64_t per_sm = (E + st->sms - 1) / st->sms;
    const int64_t t = std::max<int64_t>(32, (per_sm + 31) / 32 * 32);
    if (t < tile) {
      tile = (int)t;
      smem_bytes = pl.k->smem(tile, pl.Q);
    }
  }
  Req q;
  q.coords = coords;
  q.coeffs = coeffs;
  q.out = out;
  q.tab = te->dev;
  q.E = E;
  q.form = form;
  q.p = p;
  q.Q = pl.Q;
  q.tile = tile;
  q.out_f32 = out_f32;
  q.kind = 0;
  q.tile0 = 0;
  q.skip_copy = g_skip_copy.exchange(0);  // test hook, one launch only
  q.tile_ctr = nullptr;                   // set per launch (issue_launch_raw)
  const int64_t ntiles = (E + tile - 1) / tile;
  int per_sm = 0;
  {
    // the opt-in shared-memory ceiling is raised once per kernel and device (it only
    // permits; each launch still asks for its own size), occupancy once per size
    static std::mutex mu;
    static std::map<std::tuple<const void*, size_t, int>, int> occ;
    std::lock_guard<std::mutex> lk(mu);
    auto key = std::make_tuple(pl.k->fn, smem_bytes, st->dev);
    auto it = occ.find(key);
    if (it == occ.end()) {
      cudaFuncAttributes fa;
      CUDA_TRY(cudaFuncGetAttributes(&fa, pl.k->fn));
      const int ceiling = (int)st->smem_optin - (int)fa.sharedSizeBytes;  // minus the kernel's static shared memory
      if ((int)smem_bytes > ceiling) return fail(FEA_EINVAL, "tile does not fit the device's shared memory");
      CUDA_TRY(cudaFuncSetAttribute(pl.k->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, ceiling));
      // the tensor-core kernels size their residency by shared memory (their tensor-memory
      // columns must fit): ask for the largest shared-memory carveout, or the occupancy
      // query counts one CTA per SM where two fit
      if (pl.k->prec == 2)
        CUDA_TRY(cudaFuncSetAttribute(pl.k->fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      (int)cudaSharedmemCarveoutMaxShared));
      CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pl.k->fn, pl.k->threads ? pl.k->threads : NT,
                                                             smem_bytes));
      if (is_pretc_kernel(pl.k->fn) && per_sm == 1) per_sm = 2;  // two fit by shared memory and tensor memory
      occ[key] = per_sm;
    } else {
      per_sm = it->second;
    }
  }
  if (per_sm < 1) return fail(FEA_EINVAL, "kernel cannot be resident with this tile");
  L->fn = pl.k->fn;
  L->threads = pl.k->threads ? pl.k->threads : NT;
  L->grid = (unsigned)std::min<int64_t>(ntiles, (int64_t)st->sms * per_sm);
  L->smem = smem_bytes;
  L->q = q;
  L->err = st->err;
  L->dyn = pl.k->dyn_tiles;
  L->st = st;
  return FEA_OK;
}

// The tile counter of `stream` (assigned on first use, no allocation), or null
// once every counter has a stream: the kernel then runs its static schedule.
static unsigned long long* tile_counter(DevState* st, cudaStream_t stream) {
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = st->ctr_slot.find(stream);
  if (it == st->ctr_slot.end()) {
    if ((int)st->ctr_slot.size() >= DevState::kCounters) return nullptr;
    it = st->ctr_slot.emplace(stream, (int)st->ctr_slot.size()).first;
  }
  return st->ctr + it->second;
}

// Launch a prepared kernel on `stream`; a kernel that hands out its tiles
// dynamically gets its stream's counter, zeroed on the stream just before.
cudaError_t issue_launch_raw(PreparedLaunch& L, cudaStream_t stream) {
  Req q = L.q;
  q.tile_ctr = nullptr;
  if (L.dyn && L.st) {
    q.tile_ctr = tile_counter(L.st, stream);
    if (q.tile_ctr) {
      const cudaError_t e = cudaMemsetAsync(q.tile_ctr, 0, sizeof(unsigned long long), stream);
      if (e != cudaSuccess) return e;
    }
  }
  void* args[] = {&q, &L.err};
  return cudaLaunchKernel(L.fn, dim3(L.grid), dim3(L.threads), args, L.smem, stream);
}

int issue_launch(PreparedLaunch& L, cudaStream_t stream) {
  CUDA_TRY(issue_launch_raw(L, stream));
  return FEA_OK;
}

int launch_plan(DevState* st, const Plan& pl, int form, int p, int64_t E, const double* coords, const double* coeffs,
                void* out, int out_f32, cudaStream_t stream) {
  PreparedLaunch L;
  int rc = prepare_launch(st, pl, form, p, E, coords, coeffs, out, out_f32, &L);
  if (rc) return rc;
  return issue_launch(L, stream);
}

int assemble_impl(int form, int degree, int64_t E, const double* coords, const double* coeffs, void* out,
                  const fea_options* opt, void* stream) {
  if (!valid_fd(form, degree)) return fail(FEA_EINVAL, "unsupported form/degree");
  if (E < 0) return fail(FEA_EINVAL, "negative element count");
  const fea_options o = opt ? *opt : default_options();
  if (o.out_f32 != 0 && o.out_f32 != 1) return fail(FEA_EINVAL, "out_f32 must be 0 or 1");
  const int n = local_dim(form, degree);
  if (E > (int64_t)(INT64_MAX / ((int64_t)n * n * 8))) return fail(FEA_EINVAL, "size overflow");
  DevState* st = nullptr;
  int rc = get_dev(&st);
  if (rc) return rc;
  Plan pl;
  rc = make_plan(st, form, degree, o, &pl, false);
  if (rc) return rc;
  if (E == 0) return FEA_OK;
  if ((rc = check_device_ptr(coords, "coords", false))) return rc;
  if ((rc = check_device_ptr(coeffs, "coeffs", form == FEA_MASS))) return rc;
  if ((rc = check_device_ptr(out, "out", false))) return rc;
  return launch_plan(st, pl, form, degree, E, coords, coeffs, out, o.out_f32, (cudaStream_t)stream);
}

// Local and global assembly in one pass: the streaming pre-evaluated kernel
// adds each element matrix into the CSR values at its precomputed positions
// instead of storing it (mass and Helmholtz P1-P3, FP32 contraction).
int assemble_csr_impl(int form, int degree, int64_t E, const double* coords, const double* coeffs, const void* map,
                      int map_i64, int64_t nnz, double* values, void* stream) {
  if (!valid_fd(form, degree)) return fail(FEA_EINVAL, "unsupported form/degree");
  if ((form != FEA_MASS && form != FEA_HELMHOLTZ) || degree > 3)
    return fail(FEA_EINVAL, "one-pass global assembly covers mass and Helmholtz P1-P3 "
                            "(other forms: fea_assemble, then fea_scatter_add_csr_mapped)");
  if (E < 0 || nnz < 0) return fail(FEA_EINVAL, "negative size");
  if (map_i64 != 0 && map_i64 != 1) return fail(FEA_EINVAL, "map_i64 must be 0 or 1");
  if (!map_i64 && nnz > 2147483647) return fail(FEA_EINVAL, "nnz >= 2^31 needs an int64 map");
  const int n = local_dim(form, degree);
  if (E > (int64_t)(INT64_MAX / ((int64_t)n * n * 8))) return fail(FEA_EINVAL, "size overflow");
  DevState* st = nullptr;
  int rc = get_dev(&st);
  if (rc) return rc;
  fea_options o = default_options();
  o.variant = FEA_VARIANT_PRE;
  Plan pl;
  if ((rc = make_plan(st, form, degree, o, &pl, false))) return rc;
  const void* fn = find_scatter_kernel(pl.k->fn, map_i64);
  if (!fn) return fail(FEA_EINVAL, "no one-pass kernel for this plan");
  if (E == 0) return FEA_OK;
  if ((rc = check_device_ptr(coords, "coords", false))) return rc;
  if ((rc = check_device_ptr(coeffs, "coeffs", form == FEA_MASS))) return rc;
  if ((rc = check_device_ptr(map, "map", false))) return rc;
  if ((rc = check_device_ptr(values, "values", nnz == 0))) return rc;
  PreparedLaunch L;
  if ((rc = prepare_launch(st, pl, form, degree, E, coords, coeffs, nullptr, 0, &L))) return rc;
  int per_sm = 0;
  {
    static std::mutex mu;
    static std::map<std::tuple<const void*, size_t, int>, int> occ;
    std::lock_guard<std::mutex> lk(mu);
    auto key = std::make_tuple(fn, L.smem, st->dev);
    auto it = occ.find(key);
    if (it == occ.end()) {
      cudaFuncAttributes fa;
      CUDA_TRY(cudaFuncGetAttributes(&fa, fn));
      CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)st->smem_optin - (int)fa.sharedSizeBytes));
      CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, NT, L.smem));
      occ[key] = per_sm;
    } else {
      per_sm = it->second;
    }
  }
  if (per_sm < 1) return fail(FEA_EINVAL, "kernel cannot be resident with this tile");
  const int64_t ntiles = (E + L.q.tile - 1) / L.q.tile;
  const unsigned grid = (unsigned)std::min<int64_t>(ntiles, (int64_t)st->sms * per_sm);
  ScatterArgs sc{map, nnz, values};
  void* args[] = {&L.q, &sc, &L.err};
  CUDA_TRY(cudaLaunchKernel(fn, dim3(grid), dim3(NT), args, L.smem, (cudaStream_t)stream));
  return FEA_OK;
}

// The same with the entries of each tile combined per CSR position (plan from
// fea_csr_combine_plan): one FP64 atomic per distinct position of a tile.
int assemble_csr_combined_impl(int form, int degree, int64_t E, const double* coords, const double* coeffs,
                               const int32_t* plan, int64_t plan_words, int64_t nnz, double* values, void* stream) {
  if (!valid_fd(form, degree)) return fail(FEA_EINVAL, "unsupported form/degree");
  size_t smem = 0;
  const void* fn = find_combine_kernel(form, degree, &smem);
  if (!fn) return fail(FEA_EINVAL, "combined global assembly covers mass and Helmholtz P1-P3");
  if (E < 0 || nnz < 0 || plan_words < 0) return fail(FEA_EINVAL, "negative size");
  const int n = local_dim(form, degree);
  if (E > (int64_t)(INT64_MAX / ((int64_t)n * n * 8))) return fail(FEA_EINVAL, "size overflow");
  const int T = combine_tile(n);
  const int64_t ntiles = (E + T - 1) / T;
  if (plan_words < 4 + 2 * (ntiles + 1)) return fail(FEA_EINVAL, "plan too short for E elements");
  if (reinterpret_cast<uintptr_t>(plan) % 16) return fail(FEA_EINVAL, "plan must be 16-byte aligned");
  DevState* st = nullptr;
  int rc = get_dev(&st);
  if (rc) return rc;
  fea_options o = default_options();
  o.variant = FEA_VARIANT_PRE;
  Plan pl;
  if ((rc = make_plan(st, form, degree, o, &pl, false))) return rc;
  if (!find_scatter_kernel(pl.k->fn, 0)) return fail(FEA_EINVAL, "no one-pass kernel for this plan");
  if (E == 0) return FEA_OK;
  if ((rc = check_device_ptr(coords, "coords", false))) return rc;
  if ((rc = check_device_ptr(coeffs, "coeffs", form == FEA_MASS))) return rc;
  if ((rc = check_device_ptr(plan, "plan", false))) return rc;
  if ((rc = check_device_ptr(values, "values", nnz == 0))) return rc;
  PreparedLaunch L;
  if ((rc = prepare_launch(st, pl, form, degree, E, coords, coeffs, nullptr, 0, &L))) return rc;
  L.q.tile = T;  // the plan's tile, whatever the planner chose
  int per_sm = 0;
  {
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, int> occ;
    std::lock_guard<std::mutex> lk(mu);
    auto key = std::make_pair(fn, st->dev);
    auto it = occ.find(key);
    if (it == occ.end()) {
      cudaFuncAttributes fa;
      CUDA_TRY(cudaFuncGetAttributes(&fa, fn));
      CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)st->smem_optin - (int)fa.sharedSizeBytes));
      CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, NT, smem));
      occ[key] = per_sm;
    } else {
      per_sm = it->second;
    }
  }
  if (per_sm < 1) return fail(FEA_EINVAL, "kernel cannot be resident with the combining tile");
  const unsigned grid = (unsigned)std::min<int64_t>(ntiles, (int64_t)st->sms * per_sm);
  CombineArgs cb{plan, plan_words, nnz, values};
  void* args[] = {&L.q, &cb, &L.err};
  CUDA_TRY(cudaLaunchKernel(fn, dim3(grid), dim3(NT), args, smem, (cudaStream_t)stream));
  return FEA_OK;
}

// Element vectors (linear forms): Helmholtz load vector, Neo-Hookean residual.
int assemble_vector_impl(int form, int degree, int64_t E, const double* coords, const double* coeffs, void* out,
                         const fea_options* opt, void* stream) {
  if (!valid_fd(form, degree)) return fail(FEA_EINVAL, "unsupported form/degree");
  if (form != FEA_HELMHOLTZ && form != FEA_NEOHOOKEAN)
    return fail(FEA_EINVAL, "element vectors exist for the Helmholtz load vector and the Neo-Hookean residual only");
  if (E < 0) return fail(FEA_EINVAL, "negative element count");
  const fea_options o = opt ? *opt : default_options();
  if (o.out_f32 != 0 && o.out_f32 != 1) return fail(FEA_EINVAL, "out_f32 must be 0 or 1");
  if (o.precision != FEA_PREC_FP64 && o.precision != FEA_PREC_FP32) return fail(FEA_EINVAL, "unsupported precision");
  if (o.variant != FEA_VARIANT_AUTO) return fail(FEA_EINVAL, "element vectors have one variant (AUTO)");
  DevState* st = nullptr;
  int rc = get_dev(&st);
  if (rc) return rc;
  const int prec = o.precision == FEA_PREC_FP64 ? 0 : 1;
  // the load vector reads the mass form's pre-evaluated table (int phi_i phi_k)
  const int table_form = form == FEA_HELMHOLTZ ? FEA_MASS : form;
  Plan pl;
  pl.k = find_vec_kernel(form, degree, prec);
  if (!pl.k) return fail(FEA_EINVAL, "no element-vector kernel for this form/degree/precision");
  pl.variant = pl.k->variant;
  pl.prec = prec;
  pl.Q = rule_points(rule_index(table_form, degree));
  const size_t limit = st->smem_optin;
  const size_t budget = o.smem_budget ? std::min(o.smem_budget, limit) : limit;
  pl.tile = o.tile ? o.tile : pl.k->pref_tile;
  if (pl.tile < 1 || pl.tile > pl.k->max_tile) return fail(FEA_EINVAL, "tile out of range for this kernel");
  while (o.tile == 0 && pl.tile > 1 && pl.k->smem(pl.tile, pl.Q) > budget) --pl.tile;
  pl.smem = pl.k->smem(pl.tile, pl.Q);
  if (pl.smem > budget) return fail(FEA_EINVAL, "tile does not fit the shared-memory budget (Constraint 2)");
  if (E == 0) return FEA_OK;
  if ((rc = check_device_ptr(coords, "coords", false))) return rc;
  if ((rc = check_device_ptr(coeffs, "coeffs", false))) return rc;
  if ((rc = check_device_ptr(out, "out", false))) return rc;
  return launch_plan(st, pl, table_form, degree, E, coords, coeffs, out, o.out_f32, (cudaStream_t)stream);
}

// ------------------------------------------------------------------ host API
static int ensure_ws(DevState* st, int b, int k, size_t bytes) {
  if (st->ws_bytes[b][k] >= bytes) return FEA_OK;
  if (st->ws[b][k]) cudaFree(st->ws[b][k]);
  st->ws[b][k] = nullptr;
  st->ws_bytes[b][k] = 0;
  if (cudaMalloc(&st->ws[b][k], bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(FEA_ENOMEM, "workspace allocation failed");
  }
  st->ws_bytes[b][k] = bytes;
  return FEA_OK;
}

int assemble_host_impl(int form, int degree, int64_t E, const double* coords, const double* coeffs, void* out,
                       const fea_options* opt, void* stream) {
  if (!valid_fd(form, degree)) return fail(FEA_EINVAL, "unsupported form/degree");
  if (E < 0) return fail(FEA_EINVAL, "negative element count");
  const fea_options o = opt ? *opt : default_options();
  DevState* st = nullptr;
  int rc = get_dev(&st);
  if (rc) return rc;
  Plan pl;
  rc = make_plan(st, form, degree, o, &pl, false);
  if (rc) return rc;
  if (E == 0) return FEA_OK;
  if (!coords || !out || (!coeffs && form != FEA_MASS)) return fail(FEA_EINVAL, "NULL host buffer");
  const int n = local_dim(form, degree);
  const int clen = coeff_len(form, degree);
  const size_t osz = o.out_f32 ? 4 : 8;
  for (int b = 0; b < 2; ++b)
    if (!st->hs[b]) CUDA_TRY(cudaStreamCreateWithFlags(&st->hs[b], cudaStreamNonBlocking));
  // chunks: at least 4 for overlap, tile-aligned, at most 64 MiB of output each
  int64_t chunk = std::max<int64_t>(pl.tile, (int64_t)((64ull << 20) / ((size_t)n * n * osz)));
  chunk = std::min<int64_t>(chunk, (E + 3) / 4);
  chunk = std::max<int64_t>(1, (chunk + pl.tile - 1) / pl.tile * pl.tile);
  const size_t cbytes = (size_t)chunk * 12 * 8;
  const size_t fbytes = ((size_t)chunk * clen + (form == FEA_NEOHOOKEAN ? 2 : 0)) * 8;
  const size_t obytes = (size_t)chunk * n * n * osz;
  for (int b = 0; b < 2; ++b) {
    if ((rc = ensure_ws(st, b, 0, cbytes))) return rc;
    if (fbytes && (rc = ensure_ws(st, b, 1, fbytes))) return rc;
    if ((rc = ensure_ws(st, b, 2, obytes))) return rc;
  }
  cudaStream_t us = (cudaStream_t)stream;
  cudaEvent_t ev;
  CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  CUDA_TRY(cudaEventRecord(ev, us));
  for (int b = 0; b < 2; ++b) CUDA_TRY(cudaStreamWaitEvent(st->hs[b], ev, 0));
  int k = 0;
  for (int64_t e0 = 0; e0 < E; e0 += chunk, ++k) {
    const int b = k & 1;
    cudaStream_t s = st->hs[b];
    const int64_t ne = std::min<int64_t>(chunk, E - e0);
    double* dc = (double*)st->ws[b][0];
    double* df = (double*)st->ws[b][1];
    CUDA_TRY(cudaMemcpyAsync(dc, coords + e0 * 12, (size_t)ne * 96, cudaMemcpyHostToDevice, s));
    if (clen) CUDA_TRY(cudaMemcpyAsync(df, coeffs + e0 * clen, (size_t)ne * clen * 8, cudaMemcpyHostToDevice, s));
    if (form == FEA_NEOHOOKEAN)
      CUDA_TRY(cudaMemcpyAsync(df + ne * clen, coeffs + E * clen, 16, cudaMemcpyHostToDevice, s));
    rc = launch_plan(st, pl, form, degree, ne, dc, clen ? df : nullptr, st->ws[b][2], o.out_f32, s);
    if (rc) return rc;
    CUDA_TRY(cudaMemcpyAsync((char*)out + (size_t)e0 * n * n * osz, st->ws[b][2], (size_t)ne * n * n * osz,
                             cudaMemcpyDeviceToHost, s));
  }
  for (int b = 0; b < 2; ++b) CUDA_TRY(cudaStreamSynchronize(st->hs[b]));
  cudaEventDestroy(ev);
  return FEA_OK;
}

int sync_impl(void* stream) {
  DevState* st = nullptr;
  int rc = get_dev(&st);
  if (rc) return rc;
  CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
  unsigned h = 0;
  CUDA_TRY(cudaMemcpy(&h, st->err, sizeof(unsigned), cudaMemcpyDeviceToHost));
  if (h) {
    CUDA_TRY(cudaMemset(st->err, 0, sizeof(unsigned)));
    if (h & 4u) return fail(FEA_EINVAL, "a kernel refused a tile larger than its shared memory");
    if (h & 8u) return fail(FEA_EINVAL, "global assembly: a DOF, row segment or column is outside the CSR pattern");
    if (h & 2u) return fail(FEA_ETIMEOUT, "a bounded wait for a tile's input copy gave up");
    return fail(FEA_EDEGENERATE, "degenerate element (det J == 0 or det F <= 0); NaN written for it");
  }
  return FEA_OK;
}

void finalize_impl() {
  std::lock_guard<std::mutex> lk(g_mu);
  int cur = 0;
  cudaGetDevice(&cur);
  for (auto& kv : g_dev) {
    DevState* st = kv.second.get();
    cudaSetDevice(st->dev);
    for (auto& t : st->tables) cudaFree(t.second.dev);
    for (int b = 0; b < 2; ++b) {
      for (int k = 0; k < 3; ++k)
        if (st->ws[b][k]) cudaFree(st->ws[b][k]);
      if (st->hs[b]) cudaStreamDestroy(st->hs[b]);
    }
    free_batch_state(st->batch);
    cudaFree(st->err);
    cudaFree(st->ctr);
  }
  g_dev.clear();
  cudaSetDevice(cur);
}

int batch_impl(const fea_request* reqs, int nreq, const fea_options* opt, void* stream);
int batch_fused_impl(const fea_request* reqs, int nreq, const fea_options* opt, void* stream);
int batch_noalloc_impl(const fea_request* reqs, int nreq, const fea_options* opt, void* stream);

}  // namespace fea

using namespace fea;

extern "C" {

int fea_local_dim(int form, int degree) { return valid_fd(form, degree) ? local_dim(form, degree) : -1; }
int fea_coeff_len(int form, int degree) { return valid_fd(form, degree) ? coeff_len(form, degree) : -1; }
int64_t fea_coeffs_size(int form, int degree, int64_t E) {
  if (!valid_fd(form, degree) || E < 0) return -1;
  return (int64_t)coeff_len(form, degree) * E + (form == FEA_NEOHOOKEAN ? 2 : 0);
}
int fea_quad_points(int form, int degree) {
  return valid_fd(form, degree) ? rule_points(rule_index(form, degree)) : -1;
}

int fea_assemble(int form, int degree, int64_t E, const double* coords, const double* coeffs, void* out, void* stream) {
  return assemble_impl(form, degree, E, coords, coeffs, out, nullptr, stream);
}
int fea_assemble_ex(int form, int degree, int64_t E, const double* coords, const double* coeffs, void* out,
                    const fea_options* opt, void* stream) {
  return assemble_impl(form, degree, E, coords, coeffs, out, opt, stream);
}
int fea_assemble_host(int form, int degree, int64_t E, const double* coords_host, const double* coeffs_host,
                      void* out_host, const fea_options* opt, void* stream) {
  return assemble_host_impl(form, degree, E, coords_host, coeffs_host, out_host, opt, stream);
}
int fea_assemble_batch(const fea_request* reqs, int nreq, const fea_options* opt, void* stream) {
  return batch_impl(reqs, nreq, opt, stream);
}
int fea_assemble_vector(int form, int degree, int64_t E, const double* coords, const double* coeffs, void* out,
                        const fea_options* opt, void* stream) {
  return assemble_vector_impl(form, degree, E, coords, coeffs, out, opt, stream);
}
int fea_assemble_batch_fused(const fea_request* reqs, int nreq, const fea_options* opt, void* stream) {
  return batch_fused_impl(reqs, nreq, opt, stream);
}
int fea_assemble_csr(int form, int degree, int64_t E, const double* coords, const double* coeffs, const void* map,
                     int map_i64, int64_t nnz, double* values, void* stream) {
  return assemble_csr_impl(form, degree, E, coords, coeffs, map, map_i64, nnz, values, stream);
}

int fea_assemble_csr_combined(int form, int degree, int64_t E, const double* coords, const double* coeffs,
                              const int32_t* plan, int64_t plan_words, int64_t nnz, double* values, void* stream) {
  return assemble_csr_combined_impl(form, degree, E, coords, coeffs, plan, plan_words, nnz, values, stream);
}
int fea_assemble_batch_noalloc(const fea_request* reqs, int nreq, const fea_options* opt, void* stream) {
  return batch_noalloc_impl(reqs, nreq, opt, stream);
}
int fea_sync(void* stream) { return sync_impl(stream); }
int fea_test_skip_input_copy(int64_t tile) {
  if (tile < -1) return fail(FEA_EINVAL, "tile must be >= -1");
  g_skip_copy.store(tile + 1);
  return FEA_OK;
}

static int plan_impl(int form, int degree, const fea_options* opt, fea_plan_info* info, bool use_tuned) {
  if (!info) return fail(FEA_EINVAL, "info is NULL");
  const fea_options o = opt ? *opt : default_options();
  DevState* st = nullptr;
  int dev_count = 0;
  if (cudaGetDeviceCount(&dev_count) == cudaSuccess && dev_count > 0) {
    int rc = get_dev(&st);
    if (rc) return rc;
  } else {
    cudaGetLastError();
  }
  Plan pl;
  int rc = make_plan(st, form, degree, o, &pl, false, use_tuned);
  if (rc) return rc;
  OpCounts oc = op_counts(form, degree);
  info->variant = pl.variant;
  info->tile = pl.tile;
  info->threads = pl.k->threads ? pl.k->threads : NT;
  info->quad_points = pl.Q;
  info->ref_terms = pre_terms(form, degree);
  info->smem_bytes = pl.smem;
  info->flops_naive = oc.naive;
  info->flops_se = oc.se;
  info->flops_pre = oc.pre;
  info->flops_run = pl.variant == FEA_VARIANT_PRE ? oc.pre : pl.variant == FEA_VARIANT_SE ? oc.se : oc.naive;
  const int n = local_dim(form, degree);
  info->bytes = 96 + 8 * (int64_t)coeff_len(form, degree) + (int64_t)n * n * (o.out_f32 ? 4 : 8);
  return FEA_OK;
}

int fea_plan(int form, int degree, const fea_options* opt, fea_plan_info* info) {
  return plan_impl(form, degree, opt, info, true);
}

int fea_plan_flop(int form, int degree, const fea_options* opt, fea_plan_info* info) {
  return plan_impl(form, degree, opt, info, false);
}

int fea_op_count(int form, int degree, int variant, int64_t* naive_flops, int64_t* opt_flops) {
  if (!valid_fd(form, degree)) return fail(FEA_EINVAL, "unsupported form/degree");
  OpCounts oc = op_counts(form, degree);
  if (variant == FEA_VARIANT_AUTO) variant = choose_variant(form, degree, 1, 232448);
  int64_t v = variant == FEA_VARIANT_PRE ? oc.pre : variant == FEA_VARIANT_SE ? oc.se : oc.naive;
  if (v < 0) return fail(FEA_EINVAL, "variant not applicable");
  if (naive_flops) *naive_flops = oc.naive;
  if (opt_flops) *opt_flops = v;
  return FEA_OK;
}

const char* fea_last_error(void) { return g_last_error.c_str(); }
void fea_finalize(void) { finalize_impl(); }

}  // extern "C"
