// decode_gl.cu -- decoding of GPU-layout (GL) streams (bp_decode,
// bp_decode_sum and bp_decode_batch with BP_LAYOUT_GPU).
//
// Work unit: a superblock of 32 blocks (4096 integers) per warp; a persistent
// grid strides over the units of all lists.  Every block decodes on its own
// from its skip header, so no carry crosses blocks (Section 4.3 container,
// Algorithm 1 with the D4 prefix of Section 5 restarted per block).  The
// warp stages the superblock's payload in shared memory with one bulk copy
// and decodes its 32 blocks from there.
#include "decode.h"
#include "bulk.cuh"
#include "gl_block.cuh"

namespace bp {

namespace {

constexpr int kThreads = 256;
constexpr int kMinBlocks = 5;  // 40 resident warps per SM
// Shared-memory stage per warp: a superblock whose payload fits (b <= 8 on
// average) is brought in with one bulk copy; larger ones read global memory.
constexpr uint32_t kStageBytes = 4096;


// Store (or sum) one decoded block: lane l holds positions 16(l%8)+4t+l/8.
template <bool SUM>
__device__ __forceinline__ void store_block(const uint32_t x[4], uint32_t cnt, int lane,
                                            uint32_t *__restrict__ o, uint64_t &acc) {
  if (SUM) {
#pragma unroll
    for (int t = 0; t < 4; t++)
      if ((uint32_t)gl_pos(lane, t) < cnt) acc += x[t];
  } else if (cnt == 128u) {
#pragma unroll
    for (int t = 0; t < 4; t++) o[gl_pos(lane, t)] = x[t];
  } else {
#pragma unroll
    for (int t = 0; t < 4; t++)
      if ((uint32_t)gl_pos(lane, t) < cnt) o[gl_pos(lane, t)] = x[t];
  }
}

template <bool SUM>
__device__ __forceinline__ void gl_decode_unit(const GlView &v, const SuperInfo &si, uint32_t q,
                                               int lane, uint32_t *__restrict__ out,
                                               uint64_t &acc) {
  for (uint32_t j = 0; j < si.nblk; j++) {
    const int b = (int)__shfl_sync(kFull, si.b, j);
    const uint32_t F = __shfl_sync(kFull, si.F, j);
    const uint32_t woff = __shfl_sync(kFull, si.woff, j);
    const uint32_t blk = q * 32u + j;
    uint32_t x[4];
    gl_block_values(b, v.payload + woff, F, lane, x);
    store_block<SUM>(x, min(128u, v.n - 128u * blk), lane, out + 128ull * blk, acc);
  }
}

// Blocks j .. j+run-1 of a staged superblock, all of width B.
template <int B, bool SUM>
__device__ __forceinline__ void gl_run_smem(const GlView &v, const SuperInfo &si, uint32_t q,
                                            uint32_t w0, uint32_t sbase, uint32_t j, uint32_t run,
                                            int lane, uint32_t *__restrict__ out, uint64_t &acc) {
#pragma unroll 1
  for (uint32_t r = 0; r < run; r++) {
    const uint32_t jj = j + r;
    const uint32_t F = __shfl_sync(kFull, si.F, jj);
    const uint32_t woff = __shfl_sync(kFull, si.woff, jj);
    const uint32_t blk = q * 32u + jj;
    uint32_t x[4];
    gl_lane_values<B>(SharedWords{sbase + 4u * (woff - w0)}, F, lane, x);
    store_block<SUM>(x, min(128u, v.n - 128u * blk), lane, out + 128ull * blk, acc);
  }
}

template <bool SUM>
__device__ __forceinline__ void gl_decode_unit_smem(const GlView &v, const SuperInfo &si,
                                                    uint32_t q, uint32_t w0, uint32_t sbase,
                                                    int lane, uint32_t *__restrict__ out,
                                                    uint64_t &acc) {
  if constexpr (SUM) {
    // decode+sum: one width dispatch per run of consecutive blocks of equal
    // width (measured faster for the sum, slower for the store)
    for (uint32_t j = 0; j < si.nblk;) {
      const uint32_t b = __shfl_sync(kFull, si.b, j);
      const uint32_t same = __ballot_sync(kFull, si.b == b) >> j;
      uint32_t run = ~same ? (uint32_t)__ffs(~same) - 1 : 32u - j;
      if (run > si.nblk - j) run = si.nblk - j;
      switch (b) {
#define BP_CASE(B)                                                        \
  case B:                                                                 \
    gl_run_smem<B, SUM>(v, si, q, w0, sbase, j, run, lane, out, acc);     \
    break;
        BP_CASE(0) BP_CASE(1) BP_CASE(2) BP_CASE(3) BP_CASE(4) BP_CASE(5) BP_CASE(6)
        BP_CASE(7) BP_CASE(8) BP_CASE(9) BP_CASE(10) BP_CASE(11) BP_CASE(12) BP_CASE(13)
        BP_CASE(14) BP_CASE(15) BP_CASE(16) BP_CASE(17) BP_CASE(18) BP_CASE(19) BP_CASE(20)
        BP_CASE(21) BP_CASE(22) BP_CASE(23) BP_CASE(24) BP_CASE(25) BP_CASE(26) BP_CASE(27)
        BP_CASE(28) BP_CASE(29) BP_CASE(30) BP_CASE(31) BP_CASE(32)
#undef BP_CASE
        default:
          break;
      }
      j += run;
    }
  } else {
    for (uint32_t j = 0; j < si.nblk; j++) {
      const int b = (int)__shfl_sync(kFull, si.b, j);
      const uint32_t F = __shfl_sync(kFull, si.F, j);
      const uint32_t woff = __shfl_sync(kFull, si.woff, j);
      const uint32_t blk = q * 32u + j;
      uint32_t x[4];
      gl_block_values_from(b, SharedWords{sbase + 4u * (woff - w0)}, F, lane, x);
      store_block<SUM>(x, min(128u, v.n - 128u * blk), lane, out + 128ull * blk, acc);
    }
  }
}

// Kinds DM, D2, D1 (Section 5): the same walk over the superblock, each block
// decoded by the kind's prefix (from shared memory when staged, else from
// global memory).
template <int KIND, bool SUM, class W>
__device__ __forceinline__ void gl_decode_unit_kind(const GlView &v, const SuperInfo &si,
                                                    uint32_t q, W words, int lane,
                                                    uint32_t *__restrict__ out, uint64_t &acc) {
  for (uint32_t j = 0; j < si.nblk; j++) {
    const int b = (int)__shfl_sync(kFull, si.b, j);
    const uint32_t F = __shfl_sync(kFull, si.F, j);
    const uint32_t woff = __shfl_sync(kFull, si.woff, j);
    const uint32_t blk = q * 32u + j;
    uint32_t x[4];
    gl_block_values_kind<KIND>(b, words(woff), F, lane, x);
    store_block<SUM>(x, min(128u, v.n - 128u * blk), lane, out + 128ull * blk, acc);
  }
}

// Word sources of a block at payload word offset woff.
struct StageAt {
  uint32_t sbase, w0;
  __device__ __forceinline__ SharedWords operator()(uint32_t woff) const {
    return SharedWords{sbase + 4u * (woff - w0)};
  }
};
struct PayloadAt {
  const uint32_t *payload;
  __device__ __forceinline__ GlobalWords operator()(uint32_t woff) const {
    return GlobalWords{payload + woff};
  }
};

template <bool SUM, class W>
__device__ __forceinline__ void gl_decode_unit_other(const GlView &v, const SuperInfo &si,
                                                     uint32_t q, W words, int lane,
                                                     uint32_t *__restrict__ out, uint64_t &acc) {
  if (v.kind == kDM) gl_decode_unit_kind<kDM, SUM>(v, si, q, words, lane, out, acc);
  else if (v.kind == kD2) gl_decode_unit_kind<kD2, SUM>(v, si, q, words, lane, out, acc);
  else gl_decode_unit_kind<kD1, SUM>(v, si, q, words, lane, out, acc);
}

__device__ __forceinline__ void flush_sum(uint64_t &acc, uint64_t *dst, int lane) {
#pragma unroll
  for (int dd = 16; dd > 0; dd >>= 1) acc += __shfl_down_sync(kFull, acc, dd);
  if (lane == 0 && acc)
    atomicAdd(reinterpret_cast<unsigned long long *>(dst), (unsigned long long)acc);
  acc = 0;
}

// Unit u belongs to the list with the largest unit_base <= u; the warp keeps
// the current list's parsed header while consecutive units stay in it.  This
// kernel decodes the D4 lists of the call and jumps over the others, which
// gl_decode_other_kernel decodes (each keeps its own register allocation).
template <bool SUM>
__global__ void __launch_bounds__(kThreads, kMinBlocks)
    gl_decode_kernel(const uint8_t *__restrict__ data, ListSrc src, uint64_t total_units,
                     uint32_t *__restrict__ out, uint64_t out_cap, uint64_t *sums,
                     uint32_t *status) {
  const int lane = threadIdx.x & 31;
  const uint64_t warp = (blockIdx.x * (uint64_t)kThreads + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * kThreads) >> 5;
  __shared__ __align__(128) uint8_t s_stage[kThreads / 32][kStageBytes];
  __shared__ __align__(8) uint64_t s_bar[kThreads / 32];
  const int wl = threadIdx.x >> 5;
  const uint32_t bar = smem_addr(&s_bar[wl]);
  const uint32_t sbase = smem_addr(&s_stage[wl][0]);
  uint32_t phase = 0;
  if (lane == 0) bulk_bar_init(bar);
  __syncwarp();
  uint32_t cur = 0xFFFFFFFFu;
  bool ok = false;
  GlView v;
  uint64_t base = 0, out_off = 0, acc = 0;
  for (uint64_t u = warp; u < total_units; u += nwarps) {
    const uint32_t li = src.find(u);
    if (li != cur) {
      if (SUM && cur != 0xFFFFFFFFu) flush_sum(acc, sums + cur, lane);
      cur = li;
      const bp_list L = src.get(li);
      base = L.unit_base;
      out_off = L.out_offset;
      ok = gl_view(data + L.enc_offset, L.enc_bytes, v) && v.n == L.n;
      if (!ok) {
        if (lane == 0) set_status(status, BP_ERR_CORRUPT);
      } else if (v.kind != kD4) {  // gl_decode_other_kernel's list: jump over it
        ok = false;
        const uint64_t end = base + v.nsuper;
        if (u < end) u += ((end - u + nwarps - 1) / nwarps - 1) * nwarps;
        continue;
      } else if (!SUM && L.out_offset + L.n > out_cap) {
        ok = false;
        if (lane == 0) set_status(status, BP_ERR_CAPACITY);
      }
    }
    if (!ok) continue;
    const uint64_t q = u - base;
    if (q >= v.nsuper) continue;
    SuperInfo si;
    if (gl_super(v, (uint32_t)q, lane, si, status)) {
      const uint32_t w0 = __shfl_sync(kFull, si.woff, 0);
      const uint32_t w1 = __shfl_sync(kFull, si.woff + 4u * si.b, si.nblk - 1);
      // The superblock's payload is contiguous, 16-byte aligned and a multiple
      // of 16 bytes: one bulk copy stages it (or, if too large for the stage,
      // one bulk prefetch pulls it into L2), so its 32 blocks cost one memory
      // round trip instead of one each.
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
        gl_decode_unit_smem<SUM>(v, si, (uint32_t)q, w0, sbase, lane, out + out_off, acc);
        __syncwarp();
        continue;
      }
      if (lane == 0 && bytes > 0) bulk_prefetch_l2(v.payload + w0, bytes);
      gl_decode_unit<SUM>(v, si, (uint32_t)q, lane, out + out_off, acc);
    }
  }
  if (SUM && cur != 0xFFFFFFFFu) flush_sum(acc, sums + cur, lane);
}

// The DM, D2 and D1 lists of the call (Section 5).  CTAs come in groups of
// `parts` per list; a CTA whose list is D4 (or has a bad header, which the
// D4 kernel reports) leaves at once, so a call without such lists costs one
// header read per CTA.  The warps of a list's group share its superblocks.
template <bool SUM>
__global__ void __launch_bounds__(kThreads, kMinBlocks)
    gl_decode_other_kernel(const uint8_t *__restrict__ data, ListSrc src, uint32_t parts,
                           uint32_t *__restrict__ out, uint64_t out_cap, uint64_t *sums,
                           uint32_t *status) {
  const uint32_t li = blockIdx.x / parts, part = blockIdx.x % parts;
  if (li >= src.count) return;
  const bp_list L = src.get(li);
  GlView v;
  if (!gl_view(data + L.enc_offset, L.enc_bytes, v) || v.n != L.n || v.kind == kD4) return;
  if (!SUM && L.out_offset + L.n > out_cap) {
    if (part == 0 && threadIdx.x == 0) set_status(status, BP_ERR_CAPACITY);
    return;
  }
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  __shared__ __align__(128) uint8_t s_stage[kThreads / 32][kStageBytes];
  __shared__ __align__(8) uint64_t s_bar[kThreads / 32];
  const uint32_t bar = smem_addr(&s_bar[wl]);
  const uint32_t sbase = smem_addr(&s_stage[wl][0]);
  uint32_t phase = 0;
  if (lane == 0) bulk_bar_init(bar);
  __syncwarp();
  uint64_t acc = 0;
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
      gl_decode_unit_other<SUM>(v, si, q, StageAt{sbase, w0}, lane, o, acc);
      __syncwarp();
    } else {
      gl_decode_unit_other<SUM>(v, si, q, PayloadAt{v.payload}, lane, o, acc);
    }
  }
  if (SUM) flush_sum(acc, sums + li, lane);
}

template <class K>
int persistent_grid(K kernel, uint64_t units, int &per_sm_cache) {
  if (per_sm_cache < 0) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, kThreads, 0) != cudaSuccess ||
        nb < 1)
      nb = 1;
    per_sm_cache = nb;
  }
  const uint64_t want = (units + (kThreads / 32) - 1) / (kThreads / 32);
  const uint64_t cap = (uint64_t)per_sm_cache * device_sm_count();
  return (int)std::max<uint64_t>(1, std::min(want, cap));
}

}  // namespace

int launch_gl_decode(const uint8_t *data, const ListSrc &src, uint64_t total_units,
                     uint32_t *out, uint64_t out_cap, uint64_t *sums, uint32_t *status,
                     cudaStream_t s) {
  if (total_units == 0) return BP_OK;
  static int occ[4] = {-1, -1, -1, -1};
  // CTAs per list of the other kinds' kernel: enough to fill the GPU once
  const uint64_t resident = (uint64_t)device_sm_count() * kMinBlocks;
  const uint32_t parts = (uint32_t)std::max<uint64_t>(1, resident / std::max<uint32_t>(src.count, 1u));
  const uint64_t ogrid64 = (uint64_t)parts * src.count;
  if (ogrid64 > 0x7FFFFFFFull) return BP_ERR_ARG;
  const int ogrid = (int)ogrid64;
  if (sums) {
    const int grid = persistent_grid(gl_decode_kernel<true>, total_units, occ[0]);
    gl_decode_kernel<true><<<grid, kThreads, 0, s>>>(data, src, total_units, out, out_cap, sums,
                                                     status);
    gl_decode_other_kernel<true><<<ogrid, kThreads, 0, s>>>(data, src, parts, out, out_cap,
                                                            sums, status);
  } else {
    const int grid = persistent_grid(gl_decode_kernel<false>, total_units, occ[2]);
    gl_decode_kernel<false><<<grid, kThreads, 0, s>>>(data, src, total_units, out, out_cap,
                                                      sums, status);
    gl_decode_other_kernel<false><<<ogrid, kThreads, 0, s>>>(data, src, parts, out, out_cap,
                                                             sums, status);
  }
  return cudaPeekAtLastError() == cudaSuccess ? BP_OK : BP_ERR_CUDA;
}

}  // namespace bp
