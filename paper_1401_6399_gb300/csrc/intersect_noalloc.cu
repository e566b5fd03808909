// intersect_noalloc.cu -- bp_intersect_pair_noalloc: the fused GPU-layout
// intersection for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: a plug-in that only works on
// the buffers its host framework hands it; a server that reserves all device
// memory in its own pool at start-up, so that a further allocation would
// fail; or latency-bound code that must not call cudaMalloc because the call
// can synchronise the device and stall every other stream.
// bp_intersect_pair needs a small scratch buffer for the ordered output (a
// tile ticket and one state word per tile of 1024 values of the shorter
// list); this variant keeps that scratch in a fixed-size array of device
// memory that belongs to the library itself.
// The caller passes only the two compressed lists and the output buffers.
//
// The array below is reserved on every GPU that loads this library and
// stays there until the process exits.  All calls share it: a call clears
// the part it uses before its kernel runs, and two calls whose work overlaps
// on the GPU (different streams, or different host threads without ordering)
// overwrite each other's state -- order them on one stream.
#include <mutex>

#include "decode.h"
#include "intersect.cuh"
#include "tuning.h"

// 256 KiB: the ticket (16 bytes) plus 8 bytes per tile of 1024 values of the
// shorter list, i.e. at most 32766 tiles (BP_NOALLOC_MAX_SHORT_LIST values).
static __device__ __align__(256) uint8_t g_noalloc_scratch[256u << 10];

namespace bp {

namespace {

constexpr size_t kNoAllocScratchBytes = sizeof(g_noalloc_scratch);
constexpr uint64_t kNoAllocMaxTiles = (kNoAllocScratchBytes - 16) / 8;
static_assert(kNoAllocMaxTiles * kIxWarps * 128 == BP_NOALLOC_MAX_SHORT_LIST,
              "header limit out of step with the scratch array");

// Device address of g_noalloc_scratch, looked up once per device and kept
// for the life of the CUDA context (a cudaDeviceReset invalidates it).
std::mutex g_mu;
void *g_addr[64] = {nullptr};

int scratch_address(void **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return BP_ERR_CUDA;
  std::lock_guard<std::mutex> g(g_mu);
  if (!g_addr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return BP_ERR_CUDA;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return BP_OK;
}

struct NoAllocArgs {
  const uint8_t *r_enc;
  uint64_t r_bytes;
  uint32_t nr;
  const uint8_t *f_enc;
  uint64_t f_bytes;
  uint32_t nf;
};

// The intersection of the fused pair kernel of bp_intersect_pair on a fixed
// schedule: one block of the shorter list r per warp (no run-length choice,
// no window of f kept from run to run), the longer list f through its skip
// headers, ordered output by ticketed tiles and look-back.
__global__ void __launch_bounds__(kIxThreads)
    noalloc_pair_kernel(NoAllocArgs a, Compaction cp, TileOut to, uint32_t ntiles,
                        uint32_t dense_max) {
  __shared__ uint32_t s_r[kIxWarps][128];
  __shared__ uint32_t s_f[kIxWarps][kIxDenseMax * 128];
  __shared__ uint32_t s_wcnt[kIxWarps], s_base[1], s_tile;
  if (threadIdx.x == 0) s_tile = atomicAdd(cp.ticket, 1u);
  __syncthreads();
  const uint32_t t = s_tile;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  GlView R, F;
  bool okR = gl_view(a.r_enc, a.r_bytes, R) && R.n == a.nr;
  bool okF = gl_view(a.f_enc, a.f_bytes, F) && F.n == a.nf;
  if ((!okR || !okF) && threadIdx.x == 0 && t == 0) set_status(to.status, BP_ERR_CORRUPT);
  if (okR && okF && (R.kind != 0u || F.kind != 0u)) {  // the probes need D4 columns
    if (threadIdx.x == 0 && t == 0) set_status(to.status, BP_ERR_ARG);
    okR = okF = false;
  }
  uint32_t v[4] = {0, 0, 0, 0};
  bool valid[4] = {false, false, false, false}, hit[4] = {false, false, false, false};
  const uint32_t kb = t * kIxWarps + w;
  if (okR && okF && kb < R.nblocks) {
    const uint32_t cnt = gl_block_into(R, kb, s_r[w], lane, to.status);
    __syncwarp();
#pragma unroll
    for (int k = 0; k < 4; k++) {
      valid[k] = (uint32_t)(32 * k + lane) < cnt;
      v[k] = valid[k] ? s_r[w][32 * k + lane] : 0u;
    }
    if (cnt > 0)
      gl_membership(F, v, valid, hit, s_r[w][0], s_r[w][cnt - 1], s_f[w], lane, dense_max,
                    to.status);
  }
  tile_emit(v, hit, t, t == ntiles - 1, cp, to, s_wcnt, s_base);
}

}  // namespace

}  // namespace bp

extern "C" {

int bp_intersect_pair_noalloc(const uint8_t *d_a, size_t a_bytes, size_t n_a, const uint8_t *d_b,
                              size_t b_bytes, size_t n_b, uint32_t *d_out, size_t out_cap,
                              uint32_t *d_count, uint32_t *d_status, void *stream) {
  if (!d_a || !d_b || !d_count || !d_status || (out_cap && !d_out)) return BP_ERR_ARG;
  if ((reinterpret_cast<uintptr_t>(d_a) & 15u) || (reinterpret_cast<uintptr_t>(d_b) & 15u))
    return BP_ERR_ARG;
  if (n_a > bp_fmt::kMaxList || n_b > bp_fmt::kMaxList) return BP_ERR_ARG;
  const bool swap = n_b < n_a;
  bp::NoAllocArgs a;
  a.r_enc = swap ? d_b : d_a;
  a.r_bytes = swap ? b_bytes : a_bytes;
  a.nr = (uint32_t)(swap ? n_b : n_a);
  a.f_enc = swap ? d_a : d_b;
  a.f_bytes = swap ? a_bytes : b_bytes;
  a.nf = (uint32_t)(swap ? n_a : n_b);
  const uint64_t chunks = (a.nr + 127ull) / 128;
  const uint64_t ntiles = std::max<uint64_t>(1, (chunks + bp::kIxWarps - 1) / bp::kIxWarps);
  if (ntiles > bp::kNoAllocMaxTiles) return BP_ERR_SCRATCH;  // shorter list beyond the limit
  void *scratch = nullptr;
  int rc = bp::scratch_address(&scratch);
  if (rc != BP_OK) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t used = bp::compaction_bytes(ntiles);
  if (cudaMemsetAsync(scratch, 0, used, s) != cudaSuccess) return BP_ERR_CUDA;
  const bp::Compaction cp = bp::compaction_at(scratch);
  bp::TileOut to{d_out, out_cap, d_count, d_status};
  const uint32_t dense = std::min<uint32_t>(bp::tuning().dense_blocks, bp::kIxDenseMax);
  bp::noalloc_pair_kernel<<<(unsigned)ntiles, bp::kIxThreads, 0, s>>>(a, cp, to, (uint32_t)ntiles,
                                                                       dense);
  return cudaPeekAtLastError() == cudaSuccess ? BP_OK : BP_ERR_CUDA;
}

}  // extern "C"
