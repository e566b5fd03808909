// decode.h -- internal launchers of the decode kernels (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "../../include/bp128.h"
#include "format.h"

namespace bp {

// The lists of one call: a device array (batch calls) or a single descriptor
// passed by value (single-list calls, which have no device array).
struct ListSrc {
  const bp_list *lists;  // device array, or nullptr to use `one`
  uint32_t count;
  bp_list one;
#ifdef __CUDACC__
  __device__ __forceinline__ bp_list get(uint32_t i) const { return lists ? lists[i] : one; }
  __device__ __forceinline__ uint64_t unit_base(uint32_t i) const {
    return lists ? lists[i].unit_base : one.unit_base;
  }
  // list owning global unit u: largest i with unit_base(i) <= u
  __device__ __forceinline__ uint32_t find(uint64_t u) const {
    uint32_t lo = 0, hi = count - 1;
    while (lo < hi) {
      const uint32_t mid = (lo + hi + 1) >> 1;
      if (unit_base(mid) <= u) lo = mid;
      else hi = mid - 1;
    }
    return lo;
  }
#endif
};

inline ListSrc single_list(size_t enc_bytes, size_t n, int layout) {
  ListSrc s;
  s.lists = nullptr;
  s.count = 1;
  s.one = bp_list{0, enc_bytes, 0, 0, (uint32_t)n, (uint32_t)layout, 0};
  return s;
}

int device_sm_count();

// GL layout.  sums == nullptr: store into out; else sums[i] += sum of list i.
// GP (S4-FastPFOR) lists: one warp per page of 32 blocks, unpack, patch,
// prefix (decode_pfor.cu).
int launch_gp_decode(const uint8_t *data, const ListSrc &src, uint64_t total_units,
                     uint32_t *out, uint64_t out_cap, uint64_t *sums, uint32_t *status,
                     cudaStream_t s);

// bp_decode_ablation: GL lists decoded by one list-major kernel with the
// prefix integrated (mode 0) or as a separate pass over a block buffer in
// shared memory (1).
int launch_gl_ablation(const uint8_t *data, const bp_list *lists, uint32_t count, uint32_t *out,
                       uint64_t out_cap, uint32_t *status, int mode, cudaStream_t s);

int launch_gl_decode(const uint8_t *data, const ListSrc &src, uint64_t total_units,
                     uint32_t *out, uint64_t out_cap, uint64_t *sums, uint32_t *status,
                     cudaStream_t s);

// Paper layout (needs scratch: pl_scratch_bytes).
size_t pl_scratch_bytes(uint64_t total_units, uint32_t count);
int launch_pl_decode(const uint8_t *data, const ListSrc &src, uint64_t total_units,
                     uint32_t *out, uint64_t out_cap, uint64_t *sums, void *scratch,
                     size_t scratch_bytes, uint32_t *status, cudaStream_t s);

// Pairwise intersection (intersect.cu).
size_t intersect_scratch_bytes(size_t na, size_t nb, int layout, int mode);
int launch_intersect_pair(const uint8_t *da, size_t a_bytes, size_t na, const uint8_t *db,
                          size_t b_bytes, size_t nb, int layout, int mode, uint32_t *out,
                          size_t out_cap, uint32_t *count, void *scratch, size_t scratch_bytes,
                          uint32_t *status, cudaStream_t s);

// Conjunctive queries (query.cu).
size_t query_batch_scratch_bytes(const bp_list *h_lists, uint32_t n_terms, const uint32_t *h_terms,
                                 const uint64_t *h_term_off, uint32_t nq, uint64_t out_cap);
int launch_query_batch(const uint8_t *data, const bp_list *lists, uint32_t n_terms,
                       const uint32_t *terms, const uint64_t *term_off, uint64_t total_terms,
                       uint32_t nq, uint32_t *out, uint64_t out_cap, uint64_t *out_off,
                       uint32_t *counts, void *scratch, size_t scratch_bytes, uint32_t *status,
                       cudaStream_t s);
// Work items of a query whose shortest list has nmin integers, and the
// scratch of a batch from its totals (incremental forms of the above).
uint64_t query_items_of(const bp_list &driver);  // driver: first list in Set-vs-Set order
size_t query_batch_scratch_for(uint64_t total_terms, uint32_t nq, uint64_t out_cap,
                               uint64_t items);
size_t query_one_scratch_bytes(const bp_list *h_lists, const uint32_t *h_terms, uint32_t k);
int launch_query_one(const uint8_t *data, const bp_list *h_lists, const uint32_t *h_terms,
                     uint32_t k, uint32_t *out, uint64_t out_cap, uint32_t *count, void *scratch,
                     size_t scratch_bytes, uint32_t *status, cudaStream_t s);

}  // namespace bp
