// Global assembly (the step after local assembly, Section 2: A = sum_K of the
// element matrices at their global degrees of freedom): the CSR sparsity
// pattern of a mesh's element-to-DOF map, built on the host, and the GPU
// scatter-add of element matrices into the CSR values.
//
// Symmetric storage: with `upper` set, the pattern holds the upper triangle
// (column >= row) only; the position map marks the lower entries of an element
// matrix with kSkipPos, which the scatters pass over without an error.
//
// Scatter: one thread per (element, local row i); the row's CSR segment is the
// same for every local column j, each column is found by binary search in the
// sorted segment and added with an FP64 atomic.  A column missing from the
// pattern, a DOF outside [0, nrows) or a row segment outside [0, nnz) is
// skipped and flagged (the next fea_sync returns FEA_EINVAL): every access
// stays inside the arrays' declared sizes.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <string>
#include <thread>
#include <vector>

#include "../../include/fea.h"
#include "common.cuh"
#include "kernels.h"

namespace fea {

constexpr int64_t kSkipPos = -2;  // map entry of a lower-triangle entry under symmetric storage

template <typename TE>
__global__ void __launch_bounds__(256) scatter_csr_kernel(int64_t E, int n, const int32_t* __restrict__ dofs,
                                                          const TE* __restrict__ elem, int64_t nrows,
                                                          const int64_t* __restrict__ row_ptr,
                                                          const int32_t* __restrict__ col_idx, int64_t nnz,
                                                          double* values, unsigned* err) {
  const int64_t rows = E * n;
  for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < rows; w += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = w / n;
    const int i = (int)(w - e * n);
    const int32_t* de = dofs + e * n;
    const int32_t r = __ldg(de + i);
    if (r < 0 || r >= nrows) {
      flag_error(err, ERR_PATTERN);
      continue;
    }
    const int64_t lo0 = __ldg(row_ptr + r), hi0 = __ldg(row_ptr + r + 1);
    if (lo0 < 0 || hi0 < lo0 || hi0 > nnz) {
      flag_error(err, ERR_PATTERN);
      continue;
    }
    const TE* a = elem + (e * n + i) * (int64_t)n;
    for (int j = 0; j < n; ++j) {
      const int32_t c = __ldg(de + j);
      int64_t lo = lo0, hi = hi0;  // first position with col_idx >= c
      while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (__ldg(col_idx + mid) < c) lo = mid + 1;
        else hi = mid;
      }
      if (lo < hi0 && __ldg(col_idx + lo) == c) atomicAdd(values + lo, (double)__ldg(a + j));
      else flag_error(err, ERR_PATTERN);
    }
  }
}

// The CSR position of every (element, i, j): the same search as the scatter,
// done once; -1 (and the error flag) where the pattern has no such entry.
// TM is int32_t (patterns with nnz < 2^31) or int64_t.
template <typename TM>
__global__ void __launch_bounds__(256) scatter_map_kernel(int64_t E, int n, const int32_t* __restrict__ dofs,
                                                          int64_t nrows, const int64_t* __restrict__ row_ptr,
                                                          const int32_t* __restrict__ col_idx, int64_t nnz,
                                                          int upper, TM* map, unsigned* err) {
  const int64_t rows = E * n;
  for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < rows; w += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = w / n;
    const int32_t* de = dofs + e * n;
    const int32_t r = __ldg(de + (w - e * n));
    TM* m = map + w * n;
    int64_t lo0 = 0, hi0 = 0;
    const bool row_ok = r >= 0 && r < nrows;
    if (row_ok) {
      lo0 = __ldg(row_ptr + r);
      hi0 = __ldg(row_ptr + r + 1);
    }
    const bool seg_ok = row_ok && lo0 >= 0 && hi0 >= lo0 && hi0 <= nnz;
    for (int j = 0; j < n; ++j) {
      int64_t pos = -1;
      if (seg_ok && upper && __ldg(de + j) < r) {
        pos = kSkipPos;
      } else if (seg_ok) {
        const int32_t c = __ldg(de + j);
        int64_t lo = lo0, hi = hi0;
        while (lo < hi) {
          const int64_t mid = (lo + hi) >> 1;
          if (__ldg(col_idx + mid) < c) lo = mid + 1;
          else hi = mid;
        }
        if (lo < hi0 && __ldg(col_idx + lo) == c) pos = lo;
      }
      if (pos == -1) flag_error(err, ERR_PATTERN);
      m[j] = (TM)pos;
    }
  }
}

// values[map[k]] += elem[k] over all E n^2 entries: coalesced reads of the map
// and the element matrices, one FP64 atomic per entry.
template <typename TE, typename TM>
__global__ void __launch_bounds__(256) scatter_mapped_kernel(int64_t total, const TM* __restrict__ map,
                                                             const TE* __restrict__ elem, int64_t nnz, double* values,
                                                             unsigned* err) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pos = __ldg(map + k);
    if (pos >= 0 && pos < nnz) atomicAdd(values + pos, (double)__ldg(elem + k));
    else if (pos != kSkipPos) flag_error(err, ERR_PATTERN);
  }
}

int set_error(int code, const char* msg);
int check_device_ptr(const void* p, const char* what, bool allow_null);
struct DevState;
int get_dev_state(DevState** out);
unsigned* device_error_word(DevState* st);
int device_sms(DevState* st);

int scatter_impl(int64_t E, int n, const int32_t* dofs, const void* elem, int elem_f32, int64_t nrows,
                 const int64_t* row_ptr, const int32_t* col_idx, int64_t nnz, double* values, void* stream) {
  if (E < 0 || n < 1 || nrows < 0 || nnz < 0) return set_error(FEA_EINVAL, "negative size or empty local dimension");
  if (elem_f32 != 0 && elem_f32 != 1) return set_error(FEA_EINVAL, "elem_f32 must be 0 or 1");
  if (E == 0) return FEA_OK;
  DevState* st = nullptr;
  int rc = get_dev_state(&st);
  if (rc) return rc;
  if ((rc = check_device_ptr(dofs, "dofs", false))) return rc;
  if ((rc = check_device_ptr(elem, "elem", false))) return rc;
  if ((rc = check_device_ptr(row_ptr, "row_ptr", false))) return rc;
  if ((rc = check_device_ptr(col_idx, "col_idx", nnz == 0))) return rc;
  if ((rc = check_device_ptr(values, "values", nnz == 0))) return rc;
  const int64_t rows = E * n;
  const int64_t grid = std::min<int64_t>((rows + 255) / 256, (int64_t)device_sms(st) * 8);
  cudaStream_t s = (cudaStream_t)stream;
  unsigned* err = device_error_word(st);
  if (elem_f32)
    scatter_csr_kernel<float><<<(unsigned)grid, 256, 0, s>>>(E, n, dofs, static_cast<const float*>(elem), nrows, row_ptr,
                                                            col_idx, nnz, values, err);
  else
    scatter_csr_kernel<double><<<(unsigned)grid, 256, 0, s>>>(E, n, dofs, static_cast<const double*>(elem), nrows, row_ptr,
                                                             col_idx, nnz, values, err);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(FEA_ECUDA, cudaGetErrorString(e));
  return FEA_OK;
}

constexpr int64_t kMaxMap32 = 2147483647;  // largest position an int32 map holds

int scatter_map_impl(int64_t E, int n, const int32_t* dofs, int64_t nrows, const int64_t* row_ptr,
                     const int32_t* col_idx, int64_t nnz, int upper, void* map, int map_i64, void* stream) {
  if (E < 0 || n < 1 || nrows < 0 || nnz < 0) return set_error(FEA_EINVAL, "negative size or empty local dimension");
  if (map_i64 != 0 && map_i64 != 1) return set_error(FEA_EINVAL, "map_i64 must be 0 or 1");
  if (upper != 0 && upper != 1) return set_error(FEA_EINVAL, "upper must be 0 or 1");
  if (!map_i64 && nnz > kMaxMap32) return set_error(FEA_EINVAL, "nnz >= 2^31 needs an int64 map");
  if (E == 0) return FEA_OK;
  DevState* st = nullptr;
  int rc = get_dev_state(&st);
  if (rc) return rc;
  if ((rc = check_device_ptr(dofs, "dofs", false))) return rc;
  if ((rc = check_device_ptr(row_ptr, "row_ptr", false))) return rc;
  if ((rc = check_device_ptr(col_idx, "col_idx", nnz == 0))) return rc;
  if ((rc = check_device_ptr(map, "map", false))) return rc;
  const int64_t rows = E * n;
  const int64_t grid = std::min<int64_t>((rows + 255) / 256, (int64_t)device_sms(st) * 8);
  cudaStream_t s = (cudaStream_t)stream;
  unsigned* err = device_error_word(st);
  if (map_i64)
    scatter_map_kernel<int64_t><<<(unsigned)grid, 256, 0, s>>>(E, n, dofs, nrows, row_ptr, col_idx, nnz, upper,
                                                               static_cast<int64_t*>(map), err);
  else
    scatter_map_kernel<int32_t><<<(unsigned)grid, 256, 0, s>>>(E, n, dofs, nrows, row_ptr, col_idx, nnz, upper,
                                                               static_cast<int32_t*>(map), err);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(FEA_ECUDA, cudaGetErrorString(e));
  return FEA_OK;
}

template <typename TM>
void launch_mapped(unsigned grid, cudaStream_t s, int64_t total, const TM* map, const void* elem, int elem_f32,
                   int64_t nnz, double* values, unsigned* err) {
  if (elem_f32)
    scatter_mapped_kernel<float, TM><<<grid, 256, 0, s>>>(total, map, static_cast<const float*>(elem), nnz, values, err);
  else
    scatter_mapped_kernel<double, TM><<<grid, 256, 0, s>>>(total, map, static_cast<const double*>(elem), nnz, values, err);
}

int scatter_mapped_impl(int64_t E, int n, const void* map, int map_i64, const void* elem, int elem_f32, int64_t nnz,
                        double* values, void* stream) {
  if (E < 0 || n < 1 || nnz < 0) return set_error(FEA_EINVAL, "negative size or empty local dimension");
  if (elem_f32 != 0 && elem_f32 != 1) return set_error(FEA_EINVAL, "elem_f32 must be 0 or 1");
  if (map_i64 != 0 && map_i64 != 1) return set_error(FEA_EINVAL, "map_i64 must be 0 or 1");
  if (E == 0) return FEA_OK;
  DevState* st = nullptr;
  int rc = get_dev_state(&st);
  if (rc) return rc;
  if ((rc = check_device_ptr(map, "map", false))) return rc;
  if ((rc = check_device_ptr(elem, "elem", false))) return rc;
  if ((rc = check_device_ptr(values, "values", nnz == 0))) return rc;
  const int64_t total = E * n * n;
  const int64_t grid = std::min<int64_t>((total + 255) / 256, (int64_t)device_sms(st) * 8);
  cudaStream_t s = (cudaStream_t)stream;
  unsigned* err = device_error_word(st);
  if (map_i64)
    launch_mapped<int64_t>((unsigned)grid, s, total, static_cast<const int64_t*>(map), elem, elem_f32, nnz, values, err);
  else
    launch_mapped<int32_t>((unsigned)grid, s, total, static_cast<const int32_t*>(map), elem, elem_f32, nnz, values, err);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(FEA_ECUDA, cudaGetErrorString(e));
  return FEA_OK;
}

// Record of one tile of the combining plan (layout in pre_combine.cuh), or only
// its size in words when out is null; -1 for a position outside [0, nnz).
template <typename TM>
int64_t combine_tile_record(const TM* map, int64_t e0, int ne, int nn, int64_t nnz, std::vector<uint64_t>& keys,
                            std::vector<int32_t>& slot_start, std::vector<int32_t>& slot_order, int32_t* out) {
  keys.clear();
  const TM* m = map + e0 * nn;
  for (int k = 0; k < ne * nn; ++k) {
    const int64_t pos = (int64_t)m[k];
    if (pos == kSkipPos) continue;
    if (pos < 0 || pos >= nnz) return -1;
    keys.push_back((uint64_t)pos << 16 | (uint64_t)k);  // k < 2^16: n^2 T <= 65536
  }
  std::sort(keys.begin(), keys.end());
  slot_start.clear();
  for (size_t i = 0; i < keys.size(); ++i)
    if (i == 0 || (keys[i] >> 16) != (keys[i - 1] >> 16)) slot_start.push_back((int32_t)i);
  const int U = (int)slot_start.size(), L = (int)keys.size();
  slot_start.push_back(L);
  // positions by number of entries, largest first; ascending position among equals
  slot_order.resize((size_t)U);
  for (int s = 0; s < U; ++s) slot_order[(size_t)s] = s;
  auto mult = [&](int32_t s) { return slot_start[(size_t)s + 1] - slot_start[(size_t)s]; };
  std::stable_sort(slot_order.begin(), slot_order.end(), [&](int32_t a, int32_t b) { return mult(a) > mult(b); });
  const int R = U ? mult(slot_order[0]) : 0;
  const int64_t cw = (R + 3) & ~3, pw = (U + 3) & ~3, iw = ((L + 1) / 2 + 3) & ~3;
  const int64_t words = 4 + cw + pw + iw;
  if (!out) return words;
  std::fill(out, out + words, 0);
  out[0] = U;
  out[1] = R;
  out[2] = L;
  int32_t* cnt = out + 4;
  int32_t* pos = cnt + cw;
  uint16_t* idx = reinterpret_cast<uint16_t*>(pos + pw);
  for (int s = 0; s < U; ++s) {
    const int32_t so = slot_order[(size_t)s];
    pos[s] = (int32_t)(keys[(size_t)slot_start[(size_t)so]] >> 16);
    for (int r = 0; r < mult(so); ++r) ++cnt[r];  // positions with more than r entries
  }
  int64_t off = 0;
  for (int r = 0; r < R; ++r) {
    for (int s = 0; s < cnt[r]; ++s)
      idx[off + s] = (uint16_t)(keys[(size_t)slot_start[(size_t)slot_order[(size_t)s]] + r] & 0xffff);
    off += cnt[r];
  }
  return words;
}

// The combining plan of a position map (host): tile records built in parallel.
int csr_combine_plan_impl(int64_t E, int n, const void* map, int map_i64, int64_t nnz, int32_t* plan,
                          int64_t* plan_words) {
  if (E < 0 || n < 1 || nnz < 0 || !plan_words) return set_error(FEA_EINVAL, "bad combining-plan arguments");
  if (map_i64 != 0 && map_i64 != 1) return set_error(FEA_EINVAL, "map_i64 must be 0 or 1");
  if (E > 0 && !map) return set_error(FEA_EINVAL, "map is null");
  if (nnz > kMaxMap32) return set_error(FEA_EINVAL, "the plan holds 32-bit positions: nnz must be below 2^31");
  const int T = combine_tile(n);
  const int nn = n * n;
  if ((int64_t)nn * T > 65536) return set_error(FEA_EINVAL, "local dimension too large for 16-bit tile entries");
  const int64_t ntiles = (E + T - 1) / T;
  const int64_t hdr = (4 + 2 * (ntiles + 1) + 3) & ~3ll;
  std::vector<int64_t> off((size_t)ntiles + 1, 0);
  std::atomic<bool> bad{false};
  const int64_t hw = std::max<int64_t>(1, (int64_t)std::thread::hardware_concurrency());
  const int nth = (int)std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(hw, 64), (ntiles + 15) / 16));
  // pass 1: sizes (out == nullptr); pass 2: the records, into the plan
  auto run = [&](bool fill) {
    std::vector<std::thread> pool;
    for (int w = 0; w < nth; ++w)
      pool.emplace_back([&, w, fill] {
        std::vector<uint64_t> keys;
        std::vector<int32_t> start, order;
        keys.reserve((size_t)nn * T);
        for (int64_t t = w; t < ntiles && !bad.load(std::memory_order_relaxed); t += nth) {
          const int64_t e0 = t * T;
          const int ne = (int)std::min<int64_t>(T, E - e0);
          int32_t* out = fill ? plan + off[(size_t)t] : nullptr;
          const int64_t words =
              map_i64 ? combine_tile_record(static_cast<const int64_t*>(map), e0, ne, nn, nnz, keys, start, order, out)
                      : combine_tile_record(static_cast<const int32_t*>(map), e0, ne, nn, nnz, keys, start, order, out);
          if (words < 0) bad = true;
          else if (!fill) off[(size_t)t + 1] = words;
        }
      });
    for (auto& th : pool) th.join();
  };
  run(false);
  if (bad) return set_error(FEA_EINVAL, "a map position is outside [0, nnz) (and not -2)");
  off[0] = hdr;
  for (int64_t t = 0; t < ntiles; ++t) off[(size_t)t + 1] += off[(size_t)t];
  const int64_t total = off[(size_t)ntiles];
  if (plan) {
    if (*plan_words < total) return set_error(FEA_EINVAL, "plan is smaller than needed (query plan_words first)");
    std::fill(plan, plan + hdr, 0);
    plan[0] = kCombineMagic;
    plan[1] = n;
    plan[2] = T;
    std::copy(off.begin(), off.end(), reinterpret_cast<int64_t*>(plan + 4));
    run(true);
  }
  *plan_words = total;
  return FEA_OK;
}

// CSR pattern of sum_K (dofs_K x dofs_K): sorted unique columns per row.
int csr_pattern_impl(int64_t E, int n, const int32_t* dofs, int64_t nrows, int upper, int64_t* row_ptr,
                     int32_t* col_idx, int64_t* nnz) {
  if (E < 0 || n < 1 || nrows < 0 || !nnz || (E > 0 && !dofs)) return set_error(FEA_EINVAL, "bad pattern arguments");
  if (upper != 0 && upper != 1) return set_error(FEA_EINVAL, "upper must be 0 or 1");
  std::vector<std::vector<int32_t>> cols((size_t)nrows);
  for (int64_t e = 0; e < E; ++e) {
    const int32_t* d = dofs + e * n;
    for (int i = 0; i < n; ++i) {
      if (d[i] < 0 || d[i] >= nrows) return set_error(FEA_EINVAL, "a DOF index is outside [0, nrows)");
      for (int j = 0; j < n; ++j)
        if (!upper || d[j] >= d[i]) cols[(size_t)d[i]].push_back(d[j]);
    }
  }
  int64_t total = 0;
  for (auto& c : cols) {
    std::sort(c.begin(), c.end());
    c.erase(std::unique(c.begin(), c.end()), c.end());
    total += (int64_t)c.size();
  }
  if (col_idx && *nnz < total) return set_error(FEA_EINVAL, "col_idx is smaller than the pattern (query nnz first)");
  *nnz = total;
  if (row_ptr) {
    int64_t k = 0;
    for (int64_t r = 0; r < nrows; ++r) {
      row_ptr[r] = k;
      if (col_idx) std::copy(cols[(size_t)r].begin(), cols[(size_t)r].end(), col_idx + k);
      k += (int64_t)cols[(size_t)r].size();
    }
    row_ptr[nrows] = k;
  }
  return FEA_OK;
}

}  // namespace fea

extern "C" int fea_scatter_add_csr(int64_t E, int n, const int32_t* dofs, const void* elem, int elem_f32, int64_t nrows,
                                   const int64_t* row_ptr, const int32_t* col_idx, int64_t nnz, double* values,
                                   void* stream) {
  return fea::scatter_impl(E, n, dofs, elem, elem_f32, nrows, row_ptr, col_idx, nnz, values, stream);
}

extern "C" int fea_csr_pattern(int64_t E, int n, const int32_t* dofs, int64_t nrows, int upper, int64_t* row_ptr,
                               int32_t* col_idx, int64_t* nnz) {
  return fea::csr_pattern_impl(E, n, dofs, nrows, upper, row_ptr, col_idx, nnz);
}

extern "C" int fea_csr_scatter_map(int64_t E, int n, const int32_t* dofs, int64_t nrows, const int64_t* row_ptr,
                                   const int32_t* col_idx, int64_t nnz, int upper, void* map, int map_i64,
                                   void* stream) {
  return fea::scatter_map_impl(E, n, dofs, nrows, row_ptr, col_idx, nnz, upper, map, map_i64, stream);
}

extern "C" int fea_scatter_add_csr_mapped(int64_t E, int n, const void* map, int map_i64, const void* elem,
                                          int elem_f32, int64_t nnz, double* values, void* stream) {
  return fea::scatter_mapped_impl(E, n, map, map_i64, elem, elem_f32, nnz, values, stream);
}

extern "C" int fea_csr_combine_plan(int64_t E, int n, const void* map, int map_i64, int64_t nnz, int32_t* plan,
                                    int64_t* plan_words) {
  return fea::csr_combine_plan_impl(E, n, map, map_i64, nnz, plan, plan_words);
}
