// pl_block.cuh -- warp-level unpacking of one 128-integer block in the
// paper's 4-lane interleave (Section 4.2, Fig. 2): integer n of the block is
// the (n div 4)-th b-bit value of lane stream n mod 4, and lane stream s
// occupies the block words 4k+s, k = 0..b-1 (least significant bit first).
//
// Warp lane l = 8s + c reads its four values (slots 4c..4c+3 of stream s) as
// the bits [4bc, 4bc + 4b) of stream s; as in Algorithm 1 the value that
// straddles two words is joined from both (here with a funnel shift).
// Blocks after the last meta-block start at arbitrary byte offsets, so the
// loader also handles a misaligned block.
#pragma once
#include "common.cuh"

namespace bp {

template <bool ALIGNED>
__device__ __forceinline__ uint32_t pl_word(const uint8_t *blk, uint32_t i) {
  if (ALIGNED) return __ldg(reinterpret_cast<const uint32_t *>(blk) + i);
  const uintptr_t a = reinterpret_cast<uintptr_t>(blk) + 4u * i;
  const uint32_t m = (uint32_t)(a & 3u);
  const uint32_t *p = reinterpret_cast<const uint32_t *>(a - m);
  return __funnelshift_r(__ldg(p), __ldg(p + 1), 8u * m);
}

// Word i of a block in global memory (any byte alignment) or staged in
// shared memory (16-byte aligned).
template <bool ALIGNED>
struct PlGlobalWords {
  const uint8_t *blk;
  __device__ __forceinline__ uint32_t operator()(uint32_t i) const { return pl_word<ALIGNED>(blk, i); }
};
struct PlSharedWords {
  uint32_t base;  // shared-window address of the block
  __device__ __forceinline__ uint32_t operator()(uint32_t i) const {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(base + 4u * i));
    return v;
  }
};

template <int B, class L>
__device__ __forceinline__ void pl_lane_deltas(const L &ld, int lane, uint32_t d[4]) {
  if constexpr (B == 0) {
    d[0] = d[1] = d[2] = d[3] = 0u;
  } else {
    constexpr int G = gcd_c(4 * B, 32);
    constexpr int OMAX = 32 - G;
    constexpr int NW = (OMAX + 4 * B + 31) / 32;
    constexpr int UW = (4 * B + 31) / 32;
    const int s = lane >> 3, c = lane & 7;
    const uint32_t p = 4u * B * (uint32_t)c;
    const uint32_t w0 = p >> 5, o = p & 31u;
    uint32_t a[NW + 1];
#pragma unroll
    for (int k = 0; k < NW; k++)
      a[k] = (w0 + k < (uint32_t)B) ? ld(4u * (w0 + k) + s) : 0u;
    a[NW] = 0u;
    uint32_t u[UW + 1];
#pragma unroll
    for (int k = 0; k < UW; k++) u[k] = (OMAX == 0) ? a[k] : __funnelshift_r(a[k], a[k + 1], o);
    u[UW] = 0u;
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const int q = B * j, k = q >> 5, r = q & 31;
      uint32_t v = (r + B <= 32) ? (u[k] >> r) : __funnelshift_r(u[k], u[k + 1], r);
      d[j] = (B == 32) ? v : (v & ((1u << (B & 31)) - 1u));
    }
  }
}

// Runtime-width dispatch; b is warp-uniform.  Returns the 4 deltas of lane l
// for block positions 16c + 4j + s.
template <class L>
__device__ __forceinline__ void pl_block_deltas_from(int b, const L &ld, int lane, uint32_t d[4]) {
  switch (b) {
#define BP_CASE(B)                       \
  case B:                                \
    pl_lane_deltas<B>(ld, lane, d);      \
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

__device__ __forceinline__ void pl_block_deltas(int b, const uint8_t *__restrict__ blk,
                                                int lane, uint32_t d[4]) {
  if ((reinterpret_cast<uintptr_t>(blk) & 3u) == 0)
    pl_block_deltas_from(b, PlGlobalWords<true>{blk}, lane, d);
  else
    pl_block_deltas_from(b, PlGlobalWords<false>{blk}, lane, d);
}

}  // namespace bp
