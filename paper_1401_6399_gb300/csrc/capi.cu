// capi.cu -- extern "C" entry points of the device-side decode calls.
#include <algorithm>
#include <mutex>

#include "decode.h"

namespace bp {

int device_sm_count() {
  // cached per device: the SM count never changes for a device
  static std::mutex mu;
  static int cache[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
  std::lock_guard<std::mutex> g(mu);
  if (!cache[dev]) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1)
      n = 1;
    cache[dev] = n;
  }
  return cache[dev];
}

}  // namespace bp

using bp::ListSrc;

namespace {

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

int decode_common(const uint8_t *d_enc, size_t enc_bytes, int layout, size_t n, uint32_t *d_out,
                  size_t out_cap, uint64_t *d_sum, void *d_scratch, size_t scratch_bytes,
                  uint32_t *d_status, void *stream) {
  if (!d_enc || !d_status || !aligned16(d_enc)) return BP_ERR_ARG;
  if (layout != BP_LAYOUT_PAPER && layout != BP_LAYOUT_GPU) return BP_ERR_ARG;
  if (n > bp_fmt::kMaxList) return BP_ERR_ARG;
  if (!d_sum) {
    if (!d_out && n) return BP_ERR_ARG;
    if (out_cap < n) return BP_ERR_CAPACITY;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const ListSrc src = bp::single_list(enc_bytes, n, layout);
  const uint64_t units = bp_fmt::units_of(n, layout);
  if (layout == BP_LAYOUT_GPU)
    return bp::launch_gl_decode(d_enc, src, units, d_out, n, d_sum, d_status, s);
  return bp::launch_pl_decode(d_enc, src, units, d_out, n, d_sum, d_scratch, scratch_bytes,
                              d_status, s);
}

}  // namespace

extern "C" {

size_t bp_decode_scratch_bytes(size_t n, int layout) {
  if (layout != BP_LAYOUT_PAPER) return 0;
  return bp::pl_scratch_bytes(bp_fmt::units_of(n, layout), 1);
}

int bp_decode(const uint8_t *d_enc, size_t enc_bytes, int layout, size_t n, uint32_t *d_out,
              size_t out_cap, void *d_scratch, size_t scratch_bytes, uint32_t *d_status,
              void *stream) {
  return decode_common(d_enc, enc_bytes, layout, n, d_out, out_cap, nullptr, d_scratch,
                       scratch_bytes, d_status, stream);
}

int bp_decode_sum(const uint8_t *d_enc, size_t enc_bytes, int layout, size_t n, uint64_t *d_sum,
                  void *d_scratch, size_t scratch_bytes, uint32_t *d_status, void *stream) {
  if (!d_sum) return BP_ERR_ARG;
  return decode_common(d_enc, enc_bytes, layout, n, nullptr, 0, d_sum, d_scratch, scratch_bytes,
                       d_status, stream);
}

size_t bp_decode_batch_scratch_bytes(const bp_list *lists, uint32_t count) {
  if (!lists || count == 0 || lists[0].layout != BP_LAYOUT_PAPER) return 0;
  uint64_t units = 0;
  for (uint32_t i = 0; i < count; i++) units += bp_fmt::units_of(lists[i].n, BP_LAYOUT_PAPER);
  return bp::pl_scratch_bytes(units, count);
}

int bp_decode_batch(const uint8_t *d_data, const bp_list *d_lists, uint32_t count,
                    uint64_t total_units, int layout, uint32_t *d_out, uint64_t out_cap,
                    uint64_t *d_sums, void *d_scratch, size_t scratch_bytes, uint32_t *d_status,
                    void *stream) {
  if (!d_data || !d_lists || !d_status || count == 0 || !aligned16(d_data)) return BP_ERR_ARG;
  if (layout != BP_LAYOUT_PAPER && layout != BP_LAYOUT_GPU) return BP_ERR_ARG;
  if (!d_sums && !d_out) return BP_ERR_ARG;
  ListSrc src;
  src.lists = d_lists;
  src.count = count;
  src.one = bp_list{};
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (layout == BP_LAYOUT_GPU)
    return bp::launch_gl_decode(d_data, src, total_units, d_out, out_cap, d_sums, d_status, s);
  return bp::launch_pl_decode(d_data, src, total_units, d_out, out_cap, d_sums, d_scratch,
                              scratch_bytes, d_status, s);
}

int bp_decode_batch_host(const uint8_t *h_data, size_t data_bytes, const bp_list *h_lists,
                         uint32_t count, uint64_t total_units, int layout, uint8_t *d_data,
                         bp_list *d_lists, uint32_t *d_out, uint64_t out_cap, uint32_t *h_out,
                         void *d_scratch, size_t scratch_bytes, uint32_t *d_status,
                         uint32_t *h_status, void *stream) {
  if (!h_data || !h_lists || !d_data || !d_lists || !d_out || !h_out || !d_status || !h_status ||
      count == 0)
    return BP_ERR_ARG;
  uint64_t total_n = 0;
  for (uint32_t i = 0; i < count; i++) {
    if (h_lists[i].enc_offset + h_lists[i].enc_bytes > data_bytes) return BP_ERR_ARG;
    total_n = std::max<uint64_t>(total_n, h_lists[i].out_offset + h_lists[i].n);
  }
  if (total_n > out_cap) return BP_ERR_CAPACITY;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaMemcpyAsync(d_data, h_data, data_bytes, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(d_lists, h_lists, sizeof(bp_list) * count, cudaMemcpyHostToDevice, s) !=
          cudaSuccess ||
      cudaMemsetAsync(d_status, 0, sizeof(uint32_t), s) != cudaSuccess)
    return BP_ERR_CUDA;
  int rc = bp_decode_batch(d_data, d_lists, count, total_units, layout, d_out, out_cap, nullptr,
                           d_scratch, scratch_bytes, d_status, stream);
  if (rc != BP_OK) return rc;
  if (cudaMemcpyAsync(h_out, d_out, 4ull * total_n, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(h_status, d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s) !=
          cudaSuccess)
    return BP_ERR_CUDA;
  return BP_OK;
}

size_t bp_intersect_scratch_bytes(size_t n_a, size_t n_b, int layout, int mode) {
  if (mode == BP_MODE_AUTO) mode = layout == BP_LAYOUT_GPU ? BP_MODE_FUSED : BP_MODE_UNFUSED;
  return bp::intersect_scratch_bytes(n_a, n_b, layout, mode);
}

int bp_intersect_pair(const uint8_t *d_a, size_t a_bytes, size_t n_a, const uint8_t *d_b,
                      size_t b_bytes, size_t n_b, int layout, int mode, uint32_t *d_out,
                      size_t out_cap, uint32_t *d_count, void *d_scratch, size_t scratch_bytes,
                      uint32_t *d_status, void *stream) {
  if (!d_a || !d_b || !d_count || !d_status || !d_scratch) return BP_ERR_ARG;
  if (!aligned16(d_a) || !aligned16(d_b)) return BP_ERR_ARG;
  if (layout != BP_LAYOUT_PAPER && layout != BP_LAYOUT_GPU) return BP_ERR_ARG;
  if (n_a > bp_fmt::kMaxList || n_b > bp_fmt::kMaxList) return BP_ERR_ARG;
  if (mode == BP_MODE_AUTO) mode = layout == BP_LAYOUT_GPU ? BP_MODE_FUSED : BP_MODE_UNFUSED;
  if (mode != BP_MODE_FUSED && mode != BP_MODE_UNFUSED) return BP_ERR_ARG;
  if (mode == BP_MODE_FUSED && layout != BP_LAYOUT_GPU) return BP_ERR_ARG;
  if (!d_out && out_cap) return BP_ERR_ARG;
  if (scratch_bytes < bp::intersect_scratch_bytes(n_a, n_b, layout, mode)) return BP_ERR_SCRATCH;
  return bp::launch_intersect_pair(d_a, a_bytes, n_a, d_b, b_bytes, n_b, layout, mode, d_out,
                                   out_cap, d_count, d_scratch, scratch_bytes, d_status,
                                   static_cast<cudaStream_t>(stream));
}

size_t bp_query_batch_scratch_bytes(const bp_list *h_lists, uint32_t n_terms,
                                    const uint32_t *h_terms, const uint64_t *h_term_off,
                                    uint32_t n_queries, uint64_t out_cap) {
  if (!h_term_off || (n_terms && !h_lists)) return 0;
  return bp::query_batch_scratch_bytes(h_lists, n_terms, h_terms, h_term_off, n_queries, out_cap);
}

int bp_query_batch(const uint8_t *d_data, const bp_list *d_lists, uint32_t n_terms,
                   const uint32_t *d_terms, const uint64_t *d_term_off, uint64_t total_terms,
                   uint32_t n_queries, uint32_t *d_out, uint64_t out_cap, uint64_t *d_out_off,
                   uint32_t *d_counts, void *d_scratch, size_t scratch_bytes, uint32_t *d_status,
                   void *stream) {
  if (!d_data || !d_lists || !d_term_off || !d_out_off || !d_counts || !d_status || !d_scratch)
    return BP_ERR_ARG;
  if ((total_terms && !d_terms) || (out_cap && !d_out) || !aligned16(d_data)) return BP_ERR_ARG;
  return bp::launch_query_batch(d_data, d_lists, n_terms, d_terms, d_term_off, total_terms,
                                n_queries, d_out, out_cap, d_out_off, d_counts, d_scratch,
                                scratch_bytes, d_status, static_cast<cudaStream_t>(stream));
}

size_t bp_query_one_scratch_bytes(const bp_list *h_lists, uint32_t n_terms,
                                  const uint32_t *h_terms, uint32_t k) {
  if (!h_lists || (k && !h_terms)) return 0;
  for (uint32_t i = 0; i < k; i++)
    if (h_terms[i] >= n_terms) return 0;
  return bp::query_one_scratch_bytes(h_lists, h_terms, k);
}

int bp_query_one(const uint8_t *d_data, const bp_list *h_lists, uint32_t n_terms,
                 const uint32_t *h_terms, uint32_t k, uint32_t *d_out, size_t out_cap,
                 uint32_t *d_count, void *d_scratch, size_t scratch_bytes, uint32_t *d_status,
                 void *stream) {
  if (!d_data || !h_lists || !d_count || !d_status || !d_scratch || (k && !h_terms))
    return BP_ERR_ARG;
  if (!aligned16(d_data) || k > 64) return BP_ERR_ARG;
  for (uint32_t i = 0; i < k; i++)
    if (h_terms[i] >= n_terms) return BP_ERR_ARG;
  return bp::launch_query_one(d_data, h_lists, h_terms, k, d_out, out_cap, d_count, d_scratch,
                              scratch_bytes, d_status, static_cast<cudaStream_t>(stream));
}

}  // extern "C"
