// decode_ablation.cu -- GL decoding with the differential coding integrated
// into the unpacking or applied as a separate pass (bp_decode_ablation).
//
// Section 7.4 (Figure 6a) compares the integrated unpacking of Algorithm 1
// (the prefix of Section 5 applied to each unpacked 4-vector before it is
// stored) with the regular scheme, in which a block is first unpacked to
// memory and the prefix then runs over it as a second pass.  Both variants
// here are one list-major kernel of identical structure; the two-pass one
// stores every block's deltas to a buffer of 128 words of shared memory per
// warp (the nearest memory, as the paper's block buffer sits in L1; the
// j-th delta of lane l at word 32j + l, free of bank conflicts), reads them
// back and then prefixes and stores the values.  Any kind of differential
// coding.
#include "decode.h"
#include "bulk.cuh"
#include "gl_block.cuh"

namespace bp {

namespace {

constexpr int kThreads = 256;
constexpr int kMinBlocks = 5;
constexpr uint32_t kStageBytes = 4096;

// Shared-memory accesses the compiler keeps (a buffer it could otherwise
// see through and drop).
__device__ __forceinline__ void st_shared_volatile(uint32_t *p, uint32_t v) {
  asm volatile("st.shared.u32 [%0], %1;" ::"r"(smem_addr(p)), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_shared_volatile(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(smem_addr(p)) : "memory");
  return v;
}

template <class L>
__device__ __forceinline__ void block_deltas(int b, const L &ld, int lane, uint32_t d[4]) {
  switch (b) {
#define BP_CASE(B)                    \
  case B:                             \
    gl_lane_deltas<B>(ld, lane, d);   \
    break;
    BP_CASE(0) BP_CASE(1) BP_CASE(2) BP_CASE(3) BP_CASE(4) BP_CASE(5) BP_CASE(6)
    BP_CASE(7) BP_CASE(8) BP_CASE(9) BP_CASE(10) BP_CASE(11) BP_CASE(12) BP_CASE(13)
    BP_CASE(14) BP_CASE(15) BP_CASE(16) BP_CASE(17) BP_CASE(18) BP_CASE(19) BP_CASE(20)
    BP_CASE(21) BP_CASE(22) BP_CASE(23) BP_CASE(24) BP_CASE(25) BP_CASE(26) BP_CASE(27)
    BP_CASE(28) BP_CASE(29) BP_CASE(30) BP_CASE(31) BP_CASE(32)
#undef BP_CASE
    default:
      d[0] = d[1] = d[2] = d[3] = 0u;
  }
}

struct StageWords {
  uint32_t sbase, w0;
  __device__ __forceinline__ SharedWords operator()(uint32_t woff) const {
    return SharedWords{sbase + 4u * (woff - w0)};
  }
};
struct PayloadWords {
  const uint32_t *payload;
  __device__ __forceinline__ GlobalWords operator()(uint32_t woff) const {
    return GlobalWords{payload + woff};
  }
};

// The blocks of superblock q.  Positions past the list's end are neither
// stored nor read back; their deltas are the zero padding of the stream.
template <int KIND, int MODE, class W>
__device__ __forceinline__ void ablation_unit(const GlView &v, const SuperInfo &si, uint32_t q,
                                              W words, int lane, uint32_t *__restrict__ out,
                                              uint32_t *s_blk) {
  for (uint32_t j = 0; j < si.nblk; j++) {
    const int b = (int)__shfl_sync(kFull, si.b, j);
    const uint32_t F = __shfl_sync(kFull, si.F, j);
    const uint32_t woff = __shfl_sync(kFull, si.woff, j);
    const uint32_t blk = q * 32u + j;
    const uint32_t cnt = min(128u, v.n - 128u * blk);
    uint32_t *o = out + 128ull * blk;
    uint32_t d[4];
    block_deltas(b, words(woff), lane, d);
    if (MODE == 1) {
#pragma unroll
      for (int t = 0; t < 4; t++) st_shared_volatile(s_blk + 32 * t + lane, d[t]);
      __syncwarp();
#pragma unroll
      for (int t = 0; t < 4; t++) d[t] = ld_shared_volatile(s_blk + 32 * t + lane);
      __syncwarp();
    }
    uint32_t x[4], ctot;
    prefix_block<KIND>(d, F, lane, x, ctot);
#pragma unroll
    for (int t = 0; t < 4; t++)
      if ((uint32_t)gl_pos(lane, t) < cnt) o[gl_pos(lane, t)] = x[t];
  }
}

template <int MODE, class W>
__device__ __forceinline__ void ablation_unit_kind(const GlView &v, const SuperInfo &si,
                                                   uint32_t q, W words, int lane,
                                                   uint32_t *__restrict__ out, uint32_t *s_blk) {
  switch (v.kind) {
    case kD4: ablation_unit<kD4, MODE>(v, si, q, words, lane, out, s_blk); break;
    case kDM: ablation_unit<kDM, MODE>(v, si, q, words, lane, out, s_blk); break;
    case kD2: ablation_unit<kD2, MODE>(v, si, q, words, lane, out, s_blk); break;
    default: ablation_unit<kD1, MODE>(v, si, q, words, lane, out, s_blk); break;
  }
}

// CTAs come in groups of `parts` per list; the warps of a group share the
// list's superblocks, each staged in shared memory by one bulk copy when
// its payload fits.
template <int MODE>
__global__ void __launch_bounds__(kThreads, kMinBlocks)
    gl_ablation_kernel(const uint8_t *__restrict__ data, const bp_list *__restrict__ lists,
                       uint32_t count, uint32_t parts, uint32_t *__restrict__ out,
                       uint64_t out_cap, uint32_t *status) {
  const uint32_t li = blockIdx.x / parts, part = blockIdx.x % parts;
  if (li >= count) return;
  const bp_list L = lists[li];
  GlView v;
  if (!gl_view(data + L.enc_offset, L.enc_bytes, v) || v.n != L.n) {
    if (part == 0 && threadIdx.x == 0) set_status(status, BP_ERR_CORRUPT);
    return;
  }
  if (L.out_offset + L.n > out_cap) {
    if (part == 0 && threadIdx.x == 0) set_status(status, BP_ERR_CAPACITY);
    return;
  }
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  __shared__ __align__(128) uint8_t s_stage[kThreads / 32][kStageBytes];
  __shared__ __align__(8) uint64_t s_bar[kThreads / 32];
  __shared__ uint32_t s_blk[kThreads / 32][128];
  const uint32_t bar = smem_addr(&s_bar[wl]);
  const uint32_t sbase = smem_addr(&s_stage[wl][0]);
  uint32_t phase = 0;
  if (lane == 0) bulk_bar_init(bar);
  __syncwarp();
  uint32_t *o = out + L.out_offset;
  const uint32_t step = parts * (kThreads / 32);
  for (uint32_t q = part * (kThreads / 32) + wl; q < v.nsuper; q += step) {
    SuperInfo si;
    if (!gl_super(v, q, lane, si, status)) continue;
    const uint32_t w0 = __shfl_sync(kFull, si.woff, 0);
    const uint32_t w1 = __shfl_sync(kFull, si.woff + 4u * si.b, si.nblk - 1);
    const uint32_t bytes = 4u * (w1 - w0);
    if (bytes > 0 && bytes <= kStageBytes) {
      if (lane == 0) bulk_load(bar, sbase, v.payload + w0, bytes);
      const bool done = bulk_wait(bar, phase);
      phase ^= 1u;
      if (!__all_sync(kFull, done)) {  // give up: record it, let the copy land, stop
        if (lane == 0) set_status(status, BP_ERR_TIMEOUT);
        bulk_wait(bar, phase ^ 1u);
        return;
      }
      ablation_unit_kind<MODE>(v, si, q, StageWords{sbase, w0}, lane, o, s_blk[wl]);
      __syncwarp();
    } else {
      ablation_unit_kind<MODE>(v, si, q, PayloadWords{v.payload}, lane, o, s_blk[wl]);
    }
  }
}

}  // namespace

int launch_gl_ablation(const uint8_t *data, const bp_list *lists, uint32_t count, uint32_t *out,
                       uint64_t out_cap, uint32_t *status, int mode, cudaStream_t s) {
  if (count == 0) return BP_OK;
  const uint64_t resident = (uint64_t)device_sm_count() * kMinBlocks;
  const uint32_t parts = (uint32_t)std::max<uint64_t>(1, resident / count);
  const uint64_t grid64 = (uint64_t)parts * count;
  if (grid64 > 0x7FFFFFFFull) return BP_ERR_ARG;
  if (mode == 1)
    gl_ablation_kernel<1><<<(int)grid64, kThreads, 0, s>>>(data, lists, count, parts, out,
                                                           out_cap, status);
  else
    gl_ablation_kernel<0><<<(int)grid64, kThreads, 0, s>>>(data, lists, count, parts, out,
                                                           out_cap, status);
  return cudaPeekAtLastError() == cudaSuccess ? BP_OK : BP_ERR_CUDA;
}

}  // namespace bp
