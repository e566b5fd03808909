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
  if (layout != BP_LAYOUT_PAPER && layout != BP_LAYOUT_GPU && layout != BP_LAYOUT_PFOR)
    return BP_ERR_ARG;
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
  if (layout == BP_LAYOUT_PFOR)
    return bp::launch_gp_decode(d_enc, src, units, d_out, n, d_sum, d_status, s);
  return bp::launch_pl_decode(d_enc, src, units, d_out, n, d_sum, d_scratch, scratch_bytes,
                              d_status, s);
}

// ---- bp_decode_batch_host as a pipeline over groups of lists ---------------------------------
//
// Copy-in of group g+1, decode of group g and copy-out of group g-1 overlap on
// three library streams (the host link carries both directions at once);
// they are forked from the caller's stream by an event and joined back into
// it, so the call keeps the order of the work on that stream.

constexpr int kPipeGroups = 32;  // small groups: the first copy-in (before any copy-out) is short
constexpr int kNotPipelined = -1;

struct HostPipe {
  bool ready = false, failed = false;
  cudaStream_t h2d = nullptr, dec = nullptr, d2h = nullptr;
  cudaEvent_t start = nullptr, done = nullptr;
  cudaEvent_t in[kPipeGroups] = {}, decoded[kPipeGroups] = {};
};

std::mutex g_pipe_mu;

// The device's pipeline resources, created once (g_pipe_mu held); nullptr
// if they cannot be created.
HostPipe *host_pipe() {
  static HostPipe pipes[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  HostPipe &p = pipes[dev];
  if (p.failed) return nullptr;
  if (!p.ready) {
    bool ok = cudaStreamCreateWithFlags(&p.h2d, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&p.dec, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&p.d2h, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&p.start, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&p.done, cudaEventDisableTiming) == cudaSuccess;
    for (int g = 0; ok && g < kPipeGroups; g++)
      ok = cudaEventCreateWithFlags(&p.in[g], cudaEventDisableTiming) == cudaSuccess &&
           cudaEventCreateWithFlags(&p.decoded[g], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
      p.failed = true;
      return nullptr;
    }
    p.ready = true;
  }
  return &p;
}

__global__ void rebase_units_kernel(bp_list *lists, uint32_t count, uint64_t base) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) lists[i].unit_base -= base;
}

// kNotPipelined unless the lists are laid out in order (streams and outputs
// ascending and disjoint, units consecutive from 0) and there are at least two.
int decode_host_pipelined(const uint8_t *h_data, const bp_list *h_lists, uint32_t count,
                          uint64_t total_units, int layout, uint8_t *d_data, bp_list *d_lists,
                          uint32_t *d_out, uint64_t out_cap, uint32_t *h_out, void *d_scratch,
                          size_t scratch_bytes, uint32_t *d_status, uint32_t *h_status,
                          cudaStream_t s) {
  if (count < 2) return kNotPipelined;
  uint64_t units = 0, total_n = 0;
  for (uint32_t i = 0; i < count; i++) {
    const bp_list &L = h_lists[i];
    if (L.unit_base != units || L.layout != (uint32_t)layout) return kNotPipelined;
    if (i && (L.enc_offset < h_lists[i - 1].enc_offset + h_lists[i - 1].enc_bytes ||
              L.out_offset < h_lists[i - 1].out_offset + h_lists[i - 1].n))
      return kNotPipelined;
    units += bp_fmt::units_of(L.n, layout);
    total_n += L.n;
  }
  if (units != total_units) return kNotPipelined;
  // groups of consecutive lists with about equal output
  uint32_t first[kPipeGroups + 1];
  int ng = 0;
  {
    uint64_t acc = 0;
    first[ng++] = 0;
    for (uint32_t i = 0; i + 1 < count && ng < kPipeGroups; i++) {
      acc += h_lists[i].n;
      if (acc * kPipeGroups >= total_n * (uint64_t)ng) first[ng++] = i + 1;
    }
    first[ng] = count;
  }
  std::lock_guard<std::mutex> lock(g_pipe_mu);
  HostPipe *p = host_pipe();
  if (!p) return kNotPipelined;
  int rc = BP_OK;
  auto ck = [&rc](cudaError_t e) {
    if (e != cudaSuccess && rc == BP_OK) rc = BP_ERR_CUDA;
  };
  ck(cudaMemsetAsync(d_status, 0, sizeof(uint32_t), s));
  ck(cudaEventRecord(p->start, s));
  ck(cudaStreamWaitEvent(p->h2d, p->start, 0));
  ck(cudaMemcpyAsync(d_lists, h_lists, sizeof(bp_list) * count, cudaMemcpyHostToDevice, p->h2d));
  for (int g = 0; g < ng; g++) {
    const bp_list &A = h_lists[first[g]], &B = h_lists[first[g + 1] - 1];
    const uint64_t lo = A.enc_offset, hi = B.enc_offset + B.enc_bytes;
    ck(cudaMemcpyAsync(d_data + lo, h_data + lo, hi - lo, cudaMemcpyHostToDevice, p->h2d));
    ck(cudaEventRecord(p->in[g], p->h2d));
  }
  for (int g = 0; g < ng; g++) {
    const uint32_t a = first[g], cnt = first[g + 1] - a;
    const bp_list &B = h_lists[first[g + 1] - 1];
    const uint64_t ubase = h_lists[a].unit_base;
    const uint64_t gunits = B.unit_base + bp_fmt::units_of(B.n, layout) - ubase;
    ck(cudaStreamWaitEvent(p->dec, p->in[g], 0));
    rebase_units_kernel<<<(cnt + 255) / 256, 256, 0, p->dec>>>(d_lists + a, cnt, ubase);
    ck(cudaPeekAtLastError());
    if (rc == BP_OK) {
      const int r = bp_decode_batch(d_data, d_lists + a, cnt, gunits, layout, d_out, out_cap,
                                    nullptr, d_scratch, scratch_bytes, d_status, p->dec);
      if (r != BP_OK) rc = r;
    }
    ck(cudaEventRecord(p->decoded[g], p->dec));
  }
  for (int g = 0; g < ng; g++) {
    const bp_list &A = h_lists[first[g]], &B = h_lists[first[g + 1] - 1];
    const uint64_t lo = A.out_offset, hi = B.out_offset + B.n;
    ck(cudaStreamWaitEvent(p->d2h, p->decoded[g], 0));
    if (hi > lo)
      ck(cudaMemcpyAsync(h_out + lo, d_out + lo, 4ull * (hi - lo), cudaMemcpyDeviceToHost, p->d2h));
  }
  // join: the caller's stream waits for everything above (also after an error)
  ck(cudaEventRecord(p->done, p->d2h));
  ck(cudaStreamWaitEvent(s, p->done, 0));
  ck(cudaMemcpyAsync(h_status, d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  return rc;
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
  if (layout != BP_LAYOUT_PAPER && layout != BP_LAYOUT_GPU && layout != BP_LAYOUT_PFOR)
    return BP_ERR_ARG;
  if (!d_sums && !d_out) return BP_ERR_ARG;
  ListSrc src;
  src.lists = d_lists;
  src.count = count;
  src.one = bp_list{};
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (layout == BP_LAYOUT_GPU)
    return bp::launch_gl_decode(d_data, src, total_units, d_out, out_cap, d_sums, d_status, s);
  if (layout == BP_LAYOUT_PFOR)
    return bp::launch_gp_decode(d_data, src, total_units, d_out, out_cap, d_sums, d_status, s);
  return bp::launch_pl_decode(d_data, src, total_units, d_out, out_cap, d_sums, d_scratch,
                              scratch_bytes, d_status, s);
}

int bp_decode_ablation(const uint8_t *d_data, const bp_list *d_lists, uint32_t count,
                       uint32_t *d_out, uint64_t out_cap, uint32_t *d_status, int two_pass,
                       void *stream) {
  if (!d_data || !d_lists || !d_out || !d_status || count == 0 || !aligned16(d_data))
    return BP_ERR_ARG;
  if (two_pass != 0 && two_pass != 1) return BP_ERR_ARG;
  return bp::launch_gl_ablation(d_data, d_lists, count, d_out, out_cap, d_status, two_pass,
                                static_cast<cudaStream_t>(stream));
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
  const int piped = decode_host_pipelined(h_data, h_lists, count, total_units, layout, d_data,
                                          d_lists, d_out, out_cap, h_out, d_scratch,
                                          scratch_bytes, d_status, h_status, s);
  if (piped != kNotPipelined) return piped;
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
