// Uneven batches in one persistent launch.
//
// Every request is cut into tiles of its own size; the tiles of all requests
// form one work list (request r owns global tiles [tile0_r, tile0_r + nt_r)).
// A persistent CTA pulls the next tile with an atomic counter, finds its
// request by binary search and dispatches on (variant, form, degree) to the
// same tile functions the standalone kernels run.  Pulling never waits on
// another CTA, so there is no spin loop.  The counter reset and the launch are
// captured once into a CUDA graph per distinct batch and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/fea.h"
#include "host_model.h"
#include "launch.cuh"
#include "planner.h"
#include "pre.cuh"
#include "se.cuh"
#include "se_vec.cuh"
#include "pre_vec.cuh"

namespace fea {

int kind_of(int variant, int form, int p) { return (variant == FEA_VARIANT_PRE ? 16 : 0) + form * 4 + (p - 1); }

template <class K>
__device__ __forceinline__ void run_one(const Req& q, int64_t t, char* sm, unsigned* err, unsigned dyn) {
  if (K::smem(q.tile, q.Q) > dyn) {  // a tile larger than the launch's shared memory is refused
    if (threadIdx.x == 0) flag_error(err, ERR_LAUNCH);
    return;
  }
  const int64_t e0 = t * q.tile;
  const int64_t left = q.E - e0;
  K::tile(q, e0, (int)(left < q.tile ? left : q.tile), sm, err);
}

__global__ void __launch_bounds__(NT, 2) batch_kernel(const Req* __restrict__ reqs, int nreq, long long total,
                                                   unsigned long long* counter, unsigned* err) {
  extern __shared__ __align__(16) char smem_raw[];
  __shared__ long long s_w;
  __shared__ int s_r;
  for (;;) {
    if (threadIdx.x == 0) s_w = (long long)atomicAdd(counter, 1ull);
    __syncthreads();
    const long long w = s_w;
    if (w >= total) break;
    if (threadIdx.x == 0) {
      int lo = 0, hi = nreq - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (reqs[mid].tile0 <= w) lo = mid;
        else hi = mid - 1;
      }
      s_r = lo;
    }
    __syncthreads();
    const Req q = reqs[s_r];
    const int64_t t = w - q.tile0;
    const unsigned dyn = dynamic_smem_bytes();
    switch (q.kind) {
#define SEK(F, P) case (F) * 4 + (P) - 1: run_one<SeTile<F, P, float>>(q, t, smem_raw, err, dyn); break;
#define SEVK(F, P) case (F) * 4 + (P) - 1: run_one<SeVecTile<F, P, float>>(q, t, smem_raw, err, dyn); break;
#define PREK(F, P) case 16 + (F) * 4 + (P) - 1: run_one<PreTile<F, P, float>>(q, t, smem_raw, err, dyn); break;
      SEK(0, 1) SEK(0, 2) SEK(0, 3) SEK(0, 4)
      SEK(1, 1) SEK(1, 2) SEK(1, 3) SEK(1, 4)
      SEVK(2, 1) SEVK(2, 2) SEVK(2, 3) SEVK(2, 4)
      SEVK(3, 1) SEVK(3, 2) SEVK(3, 3) SEVK(3, 4)
      PREK(0, 1) PREK(0, 2) PREK(0, 3) PREK(0, 4)
      PREK(1, 1) PREK(1, 2) PREK(1, 3) PREK(1, 4)
      case 16 + 2 * 4 + 0: run_one<PreVecTile<1, float>>(q, t, smem_raw, err, dyn); break;
      case 16 + 2 * 4 + 1: run_one<PreVecTile<2, float>>(q, t, smem_raw, err, dyn); break;
      case 16 + 2 * 4 + 2: run_one<PreVecTile<3, float>>(q, t, smem_raw, err, dyn); break;
      case 16 + 2 * 4 + 3: run_one<PreVecTile<4, float>>(q, t, smem_raw, err, dyn); break;
#undef SEK
#undef SEVK
#undef PREK
      default: break;
    }
    __syncthreads();
  }
}

constexpr int kBranches = 4;  // concurrent branches of the per-request graph

struct BatchState {
  // one fused persistent kernel (fea_assemble_batch_fused)
  std::vector<Req> sig;  // requests of the captured graph
  size_t smem = 0;
  int grid = 0;
  Req* dreqs = nullptr;
  size_t dcap = 0;
  unsigned long long* counter = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  // one persistent kernel per request in concurrent graph branches (fea_assemble_batch)
  std::vector<PreparedLaunch> gsig;
  cudaGraph_t ggraph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  cudaStream_t br[kBranches] = {};
  cudaEvent_t ev[kBranches + 1] = {};
};

void free_batch_state(BatchState* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->ggraph) cudaGraphDestroy(b->ggraph);
  for (auto& x : b->br) if (x) cudaStreamDestroy(x);
  for (auto& x : b->ev) if (x) cudaEventDestroy(x);
  if (b->dreqs) cudaFree(b->dreqs);
  if (b->counter) cudaFree(b->counter);
  delete b;
}

// from fea_api.cu
struct DevState;
struct TableEntry;
int get_dev_state(DevState** out);
BatchState*& dev_batch(DevState* st);
unsigned* device_error_word(DevState* st);
int device_sms(DevState* st);
size_t device_smem_optin(DevState* st);
int device_index(DevState* st);
const void* table_ptr(DevState* st, int form, int p, int prec, int* rc);
int make_plan(DevState* st, int form, int p, const fea_options& o, Plan* pl, bool batch);
int set_error(int code, const char* msg);
int check_device_ptr(const void* p, const char* what, bool allow_null);
cudaError_t issue_launch_raw(PreparedLaunch& L, cudaStream_t stream);
int prepare_launch(DevState* st, const Plan& pl, int form, int p, int64_t E, const double* coords,
                   const double* coeffs, void* out, int out_f32, PreparedLaunch* L);

// The batched kernel's dynamic shared-memory ceiling, raised once per device to
// the device limit (a ceiling only permits; each launch asks for its own
// size), so that no launch path lowers it under another path's cached graph.
static int batch_kernel_smem_ceiling(DevState* st) {
  static std::mutex mu;
  static bool done[64] = {};
  const int dev = device_index(st);
  if (dev < 0 || dev >= 64) return set_error(FEA_EINVAL, "device index out of range");
  std::lock_guard<std::mutex> lk(mu);
  if (done[dev]) return FEA_OK;
  const void* fn = reinterpret_cast<const void*>(&batch_kernel);
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, fn);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)device_smem_optin(st) - (int)fa.sharedSizeBytes);
  if (e != cudaSuccess) return set_error(FEA_ECUDA, cudaGetErrorString(e));
  done[dev] = true;
  return FEA_OK;
}

static bool same_sig(const std::vector<Req>& a, const std::vector<Req>& b) {
  if (a.size() != b.size()) return false;
  return a.empty() || std::memcmp(a.data(), b.data(), a.size() * sizeof(Req)) == 0;
}

int batch_fused_impl(const fea_request* reqs, int nreq, const fea_options* opt, void* stream) {
  if (nreq < 0 || (nreq > 0 && !reqs)) return set_error(FEA_EINVAL, "bad request list");
  if (nreq == 0) return FEA_OK;
  fea_options o;
  if (opt) o = *opt;
  else { o.precision = FEA_PREC_FP32; o.out_f32 = 0; o.variant = FEA_VARIANT_AUTO; o.tile = 0; o.smem_budget = 0; }
  if (o.precision != FEA_PREC_FP32) return set_error(FEA_EINVAL, "the batched launch runs the FP32 contraction");
  DevState* st = nullptr;
  int rc = get_dev_state(&st);
  if (rc) return rc;
  std::vector<Req> R;
  R.reserve(nreq);
  size_t smem = 0;
  long long tiles = 0;
  for (int i = 0; i < nreq; ++i) {
    const fea_request& r = reqs[i];
    if (r.form < 0 || r.form > 3 || r.degree < 1 || r.degree > 4 || r.E < 0)
      return set_error(FEA_EINVAL, "bad request");
    if (r.E == 0) continue;
    if ((rc = check_device_ptr(r.coords, "coords", false))) return rc;
    if ((rc = check_device_ptr(r.coeffs, "coeffs", r.form == FEA_MASS))) return rc;
    if ((rc = check_device_ptr(r.out, "out", false))) return rc;
    fea_options oi = o;
    Plan pl;
    if ((rc = make_plan(st, r.form, r.degree, oi, &pl, true))) return rc;
    if (pl.variant == FEA_VARIANT_NAIVE) return set_error(FEA_EINVAL, "the batched launch has no plain variant");
    Req q;
    std::memset(&q, 0, sizeof(q));
    q.coords = r.coords;
    q.coeffs = r.coeffs;
    q.out = r.out;
    q.tab = table_ptr(st, r.form, r.degree, 1, &rc);
    if (rc) return rc;
    q.E = r.E;
    q.form = r.form;
    q.p = r.degree;
    q.Q = pl.Q;
    q.tile = pl.tile;
    q.out_f32 = o.out_f32;
    q.kind = kind_of(pl.variant, r.form, r.degree);
    q.tile0 = tiles;
    tiles += (r.E + pl.tile - 1) / pl.tile;
    smem = std::max(smem, pl.smem);
    R.push_back(q);
  }
  if (R.empty()) return FEA_OK;
  BatchState*& bs = dev_batch(st);
  if (!bs) bs = new BatchState();
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  if (!bs->exec || !same_sig(bs->sig, R)) {
    if (bs->exec) { cudaGraphExecDestroy(bs->exec); bs->exec = nullptr; }
    if (bs->graph) { cudaGraphDestroy(bs->graph); bs->graph = nullptr; }
    if (bs->dcap < R.size()) {
      if (bs->dreqs) cudaFree(bs->dreqs);
      bs->dreqs = nullptr;
      if (cudaMalloc(&bs->dreqs, R.size() * sizeof(Req)) != cudaSuccess) return set_error(FEA_ENOMEM, "batch list");
      bs->dcap = R.size();
    }
    if (!bs->counter && cudaMalloc(&bs->counter, sizeof(unsigned long long)) != cudaSuccess)
      return set_error(FEA_ENOMEM, "batch counter");
    if ((e = cudaMemcpy(bs->dreqs, R.data(), R.size() * sizeof(Req), cudaMemcpyHostToDevice)) != cudaSuccess)
      return set_error(FEA_ECUDA, cudaGetErrorString(e));
    const void* fn = reinterpret_cast<const void*>(&batch_kernel);
    if ((rc = batch_kernel_smem_ceiling(st))) return rc;
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, NT, smem)) != cudaSuccess || per_sm < 1)
      return set_error(FEA_ECUDA, "batch kernel occupancy");
    bs->grid = (int)std::min<long long>(tiles, (long long)device_sms(st) * per_sm);
    bs->smem = smem;
    // capture: counter reset + persistent launch
    cudaStream_t cap;
    if ((e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking)) != cudaSuccess)
      return set_error(FEA_ECUDA, cudaGetErrorString(e));
    unsigned* err = device_error_word(st);
    int nr = (int)R.size();
    long long total = tiles;
    Req* dr = bs->dreqs;
    unsigned long long* ctr = bs->counter;
    void* args[] = {&dr, &nr, &total, &ctr, &err};
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) e = cudaMemsetAsync(bs->counter, 0, sizeof(unsigned long long), cap);
    if (e == cudaSuccess) e = cudaLaunchKernel(fn, dim3(bs->grid), dim3(NT), args, smem, cap);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(cap, &g);
    cudaStreamDestroy(cap);
    if (e != cudaSuccess || e2 != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return set_error(FEA_ECUDA, cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    bs->graph = g;
    if ((e = cudaGraphInstantiate(&bs->exec, g, 0)) != cudaSuccess) return set_error(FEA_ECUDA, cudaGetErrorString(e));
    bs->sig = R;
  }
  if ((e = cudaGraphLaunch(bs->exec, s)) != cudaSuccess) return set_error(FEA_ECUDA, cudaGetErrorString(e));
  return FEA_OK;
}

// ------------------------------------------------------------------------
// The default batch schedule: one CUDA graph whose nodes are the requests' own
// standalone persistent kernels (each with its own tile, registers and shared
// memory), spread over concurrent branches, largest requests first.  Captured
// once per distinct batch and replayed.
// ------------------------------------------------------------------------
static bool same_launches(const std::vector<PreparedLaunch>& a, const std::vector<PreparedLaunch>& b) {
  if (a.size() != b.size()) return false;
  for (size_t i = 0; i < a.size(); ++i)
    if (a[i].fn != b[i].fn || a[i].grid != b[i].grid || a[i].threads != b[i].threads || a[i].smem != b[i].smem ||
        a[i].err != b[i].err ||
        std::memcmp(&a[i].q, &b[i].q, sizeof(Req)) != 0)
      return false;
  return true;
}

int batch_impl(const fea_request* reqs, int nreq, const fea_options* opt, void* stream) {
  if (nreq < 0 || (nreq > 0 && !reqs)) return set_error(FEA_EINVAL, "bad request list");
  if (nreq == 0) return FEA_OK;
  fea_options o;
  if (opt) o = *opt;
  else { o.precision = FEA_PREC_FP32; o.out_f32 = 0; o.variant = FEA_VARIANT_AUTO; o.tile = 0; o.smem_budget = 0; }
  if (o.precision != FEA_PREC_FP32 && o.precision != FEA_PREC_BF16X2)
    return set_error(FEA_EINVAL, "the batched launch runs the FP32 or split-BF16 contraction");
  DevState* st = nullptr;
  int rc = get_dev_state(&st);
  if (rc) return rc;
  std::vector<std::pair<double, PreparedLaunch>> work;
  work.reserve(nreq);
  for (int i = 0; i < nreq; ++i) {
    const fea_request& r = reqs[i];
    if (r.form < 0 || r.form > 3 || r.degree < 1 || r.degree > 4 || r.E < 0)
      return set_error(FEA_EINVAL, "bad request");
    if (r.E == 0) continue;
    if ((rc = check_device_ptr(r.coords, "coords", false))) return rc;
    if ((rc = check_device_ptr(r.coeffs, "coeffs", r.form == FEA_MASS))) return rc;
    if ((rc = check_device_ptr(r.out, "out", false))) return rc;
    Plan pl;
    if ((rc = make_plan(st, r.form, r.degree, o, &pl, false))) return rc;
    if (pl.variant == FEA_VARIANT_NAIVE) return set_error(FEA_EINVAL, "the batched launch has no plain variant");
    PreparedLaunch L;
    if ((rc = prepare_launch(st, pl, r.form, r.degree, r.E, r.coords, r.coeffs, r.out, o.out_f32, &L))) return rc;
    const int n = (r.form >= 2 ? 3 : 1) * (r.degree + 1) * (r.degree + 2) * (r.degree + 3) / 6;
    work.emplace_back((double)r.E * n * n, L);  // output size: the larger requests first
  }
  if (work.empty()) return FEA_OK;
  std::stable_sort(work.begin(), work.end(), [](const auto& a, const auto& b) { return a.first > b.first; });
  std::vector<PreparedLaunch> L;
  L.reserve(work.size());
  for (auto& w : work) L.push_back(w.second);
  BatchState*& bs = dev_batch(st);
  if (!bs) bs = new BatchState();
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  if (!bs->gexec || !same_launches(bs->gsig, L)) {
    if (bs->gexec) { cudaGraphExecDestroy(bs->gexec); bs->gexec = nullptr; }
    if (bs->ggraph) { cudaGraphDestroy(bs->ggraph); bs->ggraph = nullptr; }
    for (auto& x : bs->br)
      if (!x && (e = cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking)) != cudaSuccess)
        return set_error(FEA_ECUDA, cudaGetErrorString(e));
    for (auto& x : bs->ev)
      if (!x && (e = cudaEventCreateWithFlags(&x, cudaEventDisableTiming)) != cudaSuccess)
        return set_error(FEA_ECUDA, cudaGetErrorString(e));
    // capture: fork from branch 0 into the others, one kernel per request on the
    // least-loaded branch, join back into branch 0
    double load[kBranches] = {};
    e = cudaStreamBeginCapture(bs->br[0], cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) e = cudaEventRecord(bs->ev[kBranches], bs->br[0]);
    for (int k = 1; k < kBranches && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(bs->br[k], bs->ev[kBranches], 0);
    for (size_t i = 0; i < L.size() && e == cudaSuccess; ++i) {
      int k = 0;
      for (int b = 1; b < kBranches; ++b)
        if (load[b] < load[k]) k = b;
      load[k] += work[i].first;
      e = issue_launch_raw(L[i], bs->br[k]);
    }
    for (int k = 1; k < kBranches && e == cudaSuccess; ++k) {
      e = cudaEventRecord(bs->ev[k], bs->br[k]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(bs->br[0], bs->ev[k], 0);
    }
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(bs->br[0], &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return set_error(FEA_ECUDA, cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    bs->ggraph = g;
    if ((e = cudaGraphInstantiate(&bs->gexec, g, 0)) != cudaSuccess) return set_error(FEA_ECUDA, cudaGetErrorString(e));
    bs->gsig = L;
  }
  if ((e = cudaGraphLaunch(bs->gexec, s)) != cudaSuccess) return set_error(FEA_ECUDA, cudaGetErrorString(e));
  return FEA_OK;
}

// ------------------------------------------------------------------------
// The batched launch without any device allocation.
//
// Some callers cannot call cudaMalloc at the moment they assemble: code that
// lives inside another framework's memory pool and may not allocate outside
// it, or a latency-critical loop where an allocation may block, fail or cost
// more than the assembly.  fea_assemble_batch_noalloc serves them: the
// work-list counter and the request list that the batched kernel needs sit in
// the file-scope device array below instead of in library allocations; the
// request list is handed over as kernel parameters (by value) to a small copy
// kernel, and the batched kernel is launched directly.  Limits: at most
// kNoAllocMaxRequests requests per call; the device state and the tables of
// every (form, degree) in the batch must already exist on the current device
// (made by any earlier allocating call there), otherwise the call is
// rejected.  Every call shares the array, so calls whose kernels overlap on
// the GPU race.
// ------------------------------------------------------------------------
constexpr int kNoAllocMaxRequests = 512;
constexpr size_t kNoAllocReqOffset = 256;  // counter in the first 256 bytes
constexpr size_t kNoAllocBytes = kNoAllocReqOffset + (size_t)kNoAllocMaxRequests * sizeof(Req);
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

DevState* existing_dev_state();
const void* existing_table(DevState* st, int form, int p, int prec);

namespace {
constexpr int kMaxDevices = 64;
unsigned char* g_noalloc_ptr[kMaxDevices];  // device address of g_noalloc_scratch, per device
std::mutex g_noalloc_mu;

// Requests handed to the copy kernel by value, a few dozen at a time (well
// inside the kernel-parameter limit).
constexpr int kUploadChunk = 48;
struct ReqChunk {
  Req r[kUploadChunk];
};
}  // namespace

// dst[0 .. n) = chunk; the first chunk also restarts the work-list counter (the
// array keeps the previous call's contents).
__global__ void noalloc_upload(ReqChunk chunk, int n, Req* dst, unsigned long long* counter, int reset) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = chunk.r[i];
  if (reset && threadIdx.x == 0) *counter = 0ull;
}

int batch_noalloc_impl(const fea_request* reqs, int nreq, const fea_options* opt, void* stream) {
  if (nreq < 0 || (nreq > 0 && !reqs)) return set_error(FEA_EINVAL, "bad request list");
  if (nreq > kNoAllocMaxRequests)
    return set_error(FEA_EINVAL, "fea_assemble_batch_noalloc takes at most 512 requests per call");
  if (nreq == 0) return FEA_OK;
  fea_options o;
  if (opt) o = *opt;
  else { o.precision = FEA_PREC_FP32; o.out_f32 = 0; o.variant = FEA_VARIANT_AUTO; o.tile = 0; o.smem_budget = 0; }
  if (o.precision != FEA_PREC_FP32) return set_error(FEA_EINVAL, "the batched launch runs the FP32 contraction");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_error(FEA_ECUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return set_error(FEA_EINVAL, "device index out of range");
  DevState* st = existing_dev_state();
  if (!st) return set_error(FEA_EINVAL, "no library state on this device yet: make one allocating call first");
  unsigned char* scratch = nullptr;
  {
    // set-up, once per device, with that device current
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess) return set_error(FEA_ECUDA, cudaGetErrorString(e));
      g_noalloc_ptr[dev] = static_cast<unsigned char*>(p);
    }
    scratch = g_noalloc_ptr[dev];
  }
  cudaStream_t s = (cudaStream_t)stream;
  unsigned long long* ctr = reinterpret_cast<unsigned long long*>(scratch);
  Req* dr = reinterpret_cast<Req*>(scratch + kNoAllocReqOffset);
  // requests go to the device array a chunk at a time, as kernel parameters of the copy kernel
  ReqChunk chunk;
  int nc = 0;   // requests in `chunk`
  int nr = 0;   // requests uploaded or in `chunk`
  auto flush = [&]() -> int {
    if (nc == 0) return FEA_OK;
    noalloc_upload<<<1, 64, 0, s>>>(chunk, nc, dr + (nr - nc), ctr, nr == nc ? 1 : 0);
    const cudaError_t ce = cudaGetLastError();
    nc = 0;
    return ce == cudaSuccess ? FEA_OK : set_error(FEA_ECUDA, cudaGetErrorString(ce));
  };
  size_t smem = 0;
  long long tiles = 0;
  int rc;
  for (int i = 0; i < nreq; ++i) {
    const fea_request& r = reqs[i];
    if (r.form < 0 || r.form > 3 || r.degree < 1 || r.degree > 4 || r.E < 0)
      return set_error(FEA_EINVAL, "bad request");
    if (r.E == 0) continue;
    if ((rc = check_device_ptr(r.coords, "coords", false))) return rc;
    if ((rc = check_device_ptr(r.coeffs, "coeffs", r.form == FEA_MASS))) return rc;
    if ((rc = check_device_ptr(r.out, "out", false))) return rc;
    Plan pl;
    if ((rc = make_plan(st, r.form, r.degree, o, &pl, true))) return rc;
    if (pl.variant == FEA_VARIANT_NAIVE) return set_error(FEA_EINVAL, "the batched launch has no plain variant");
    const void* tab = existing_table(st, r.form, r.degree, 1);
    if (!tab) return set_error(FEA_EINVAL, "tables of a requested form/degree are not resident: make one allocating call first");
    Req& q = chunk.r[nc++];
    ++nr;
    std::memset(&q, 0, sizeof(q));
    q.coords = r.coords;
    q.coeffs = r.coeffs;
    q.out = r.out;
    q.tab = tab;
    q.E = r.E;
    q.form = r.form;
    q.p = r.degree;
    q.Q = pl.Q;
    q.tile = pl.tile;
    q.out_f32 = o.out_f32;
    q.kind = kind_of(pl.variant, r.form, r.degree);
    q.tile0 = tiles;
    tiles += (r.E + pl.tile - 1) / pl.tile;
    smem = std::max(smem, pl.smem);
    if (nc == kUploadChunk && (rc = flush())) return rc;
  }
  if (nr == 0) return FEA_OK;
  if ((rc = flush())) return rc;
  const void* fn = reinterpret_cast<const void*>(&batch_kernel);
  if ((rc = batch_kernel_smem_ceiling(st))) return rc;
  int per_sm = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, NT, smem)) != cudaSuccess || per_sm < 1)
    return set_error(FEA_ECUDA, "batch kernel occupancy");
  const int grid = (int)std::min<long long>(tiles, (long long)device_sms(st) * per_sm);
  unsigned* err = device_error_word(st);
  long long total = tiles;
  void* args[] = {&dr, &nr, &total, &ctr, &err};
  if ((e = cudaLaunchKernel(fn, dim3(grid), dim3(NT), args, smem, s)) != cudaSuccess)
    return set_error(FEA_ECUDA, cudaGetErrorString(e));
  return FEA_OK;
}

}  // namespace fea
