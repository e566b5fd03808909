// gl_block.cuh -- warp-level decoder of one 128-integer block of the GPU
// layout (GL).
//
// Mapping: warp lane l = 8s + c owns column s (positions = s mod 4) and rows
// 4c..4c+3 of the block, i.e. block positions 16c + 4j + s, j = 0..3.  In GL
// those four deltas are the contiguous bits [4bl, 4bl + 4b) of the block's
// LSB-first bit string, so each lane reads at most five consecutive words.
//
// D4 (Section 5): x_i = delta_i + x_{i-4}, i.e. a running sum down each
// column.  A lane sums its own four rows sequentially (Algorithm 1 applies
// P(t,v) = t+v one 4-vector at a time; here one column at a time), then the
// eight lanes of a column combine their totals with a 3-step shuffle scan,
// and the block's first value F (the GL skip header) is the seed of every
// column.  The bit extraction is specialised per width b at compile time,
// as the paper generates one routine per b (Section 4.2).
#pragma once
#include "common.cuh"

namespace bp {

// Word sources for the unpacker: the block's 4b words in global memory
// (read-only path) or already staged in shared memory.
struct GlobalWords {
  const uint32_t *w;
  __device__ __forceinline__ uint32_t operator()(uint32_t i) const { return __ldg(w + i); }
};
struct SharedWords {
  uint32_t base;  // shared-window address of word 0
  __device__ __forceinline__ uint32_t operator()(uint32_t i) const {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(base + 4u * i));
    return v;
  }
};

// The four deltas of `lane` from a block of width B (4B words from `ld`).
template <int B, class L>
__device__ __forceinline__ void gl_lane_deltas(const L &ld, int lane, uint32_t d[4]) {
  if constexpr (B == 0) {
    d[0] = d[1] = d[2] = d[3] = 0u;
  } else {
    constexpr int G = gcd_c(4 * B, 32);
    constexpr int OMAX = 32 - G;                // largest in-word start offset
    constexpr int NW = (OMAX + 4 * B + 31) / 32;  // words a lane may touch
    constexpr int UW = (4 * B + 31) / 32;         // words after alignment
    const uint32_t p = 4u * B * (uint32_t)lane;
    const uint32_t w0 = p >> 5, o = p & 31u;
    uint32_t a[NW + 1];
#pragma unroll
    for (int k = 0; k < NW; k++) a[k] = (w0 + k < 4u * B) ? ld(w0 + k) : 0u;
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

// Decoded values of `lane`: x[j] is block position 16c + 4j + s.
template <int B, class L>
__device__ __forceinline__ void gl_lane_values(const L &ld, uint32_t F, int lane, uint32_t x[4]) {
  uint32_t d[4];
  gl_lane_deltas<B>(ld, lane, d);
  x[0] = d[0];
  x[1] = x[0] + d[1];
  x[2] = x[1] + d[2];
  x[3] = x[2] + d[3];
  const int c = lane & 7;
  uint32_t incl = x[3];
#pragma unroll
  for (int dd = 1; dd < 8; dd <<= 1) {
    const uint32_t t = __shfl_up_sync(kFull, incl, dd, 8);
    if (c >= dd) incl += t;
  }
  const uint32_t base = F + (incl - x[3]);
#pragma unroll
  for (int j = 0; j < 4; j++) x[j] += base;
}

// ---- the other kinds of differential coding of Section 5 -----------------
//
// prefix_block<KIND> turns the four deltas d[j] of lane l = 8s + c (block
// positions 16c + 4j + s) into values, given the values before the block:
// s0 is x[-4+s] for D4 (the lane's column), x[-1] for DM and D1, and
// x[-2] (even s) or x[-1] (odd s) for D2; a GL block passes its first value
// F for all of them.  ctot receives the sum of the lane's column of deltas
// over the whole block (what a carried seed needs).
//   D4: a running sum down the column (per lane, then a 3-step scan over
//       the 8 lanes of the column).
//   DM: row t adds x[4t-1], the last value of row t-1, which is the D4-style
//       running value of column 3: 4 shuffles from the column-3 lanes.
//   D2: columns 0/2 and 1/3 form two chains; pair sums (one shuffle per row)
//       run down the rows, column 0 (1) takes the chain before its row plus
//       its own delta, column 2 (3) the chain through its row.
//   D1: an inclusive sum across the row (2 shuffles per row), the row totals
//       run down the rows.
enum { kD4 = 0, kDM = 1, kD2 = 2, kD1 = 3 };

// Exclusive sum of v over the lanes 8s .. 8s+c-1 of the lane's column.
__device__ __forceinline__ uint32_t col_excl(uint32_t v, int lane) {
  const int c = lane & 7;
  uint32_t inc = v;
#pragma unroll
  for (int dd = 1; dd < 8; dd <<= 1) {
    const uint32_t t = __shfl_up_sync(kFull, inc, dd, 8);
    if (c >= dd) inc += t;
  }
  return inc - v;
}

template <int KIND>
__device__ __forceinline__ void prefix_block(const uint32_t d[4], uint32_t s0, int lane,
                                             uint32_t x[4], uint32_t &ctot) {
  const int s = lane >> 3, c = lane & 7;
  if constexpr (KIND == kD4 || KIND == kDM) {
    uint32_t run[4];
    run[0] = d[0];
    run[1] = run[0] + d[1];
    run[2] = run[1] + d[2];
    run[3] = run[2] + d[3];
    const uint32_t e = col_excl(run[3], lane);
    ctot = __shfl_sync(kFull, e + run[3], (lane & ~7) | 7);
    uint32_t y[4];
#pragma unroll
    for (int j = 0; j < 4; j++) y[j] = s0 + e + run[j];
    if constexpr (KIND == kD4) {
#pragma unroll
      for (int j = 0; j < 4; j++) x[j] = y[j];
    } else {
      // y of the column-3 lanes: x[4t+3]; row t's base is x[4t-1]
      const uint32_t p3 = __shfl_sync(kFull, y[3], 24 + ((c + 7) & 7));  // lane (3, c-1)
      const uint32_t b0 = c ? p3 : s0;
      const uint32_t b1 = __shfl_sync(kFull, y[0], 24 + c);
      const uint32_t b2 = __shfl_sync(kFull, y[1], 24 + c);
      const uint32_t b3 = __shfl_sync(kFull, y[2], 24 + c);
      x[0] = d[0] + b0;
      x[1] = d[1] + b1;
      x[2] = d[2] + b2;
      x[3] = d[3] + b3;
    }
  } else if constexpr (KIND == kD2) {
    uint32_t rp[4], rp_prev[4], acc = 0;
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const uint32_t pj = d[j] + __shfl_xor_sync(kFull, d[j], 16);  // columns s and s^2
      rp_prev[j] = acc;
      acc += pj;
      rp[j] = acc;
    }
    const uint32_t e = col_excl(rp[3], lane);
#pragma unroll
    for (int j = 0; j < 4; j++) x[j] = s >= 2 ? s0 + e + rp[j] : s0 + e + rp_prev[j] + d[j];
    uint32_t t = d[0] + d[1] + d[2] + d[3];
    t += __shfl_xor_sync(kFull, t, 1);
    t += __shfl_xor_sync(kFull, t, 2);
    t += __shfl_xor_sync(kFull, t, 4);
    ctot = t;
  } else {  // kD1
    uint32_t q[4];
#pragma unroll
    for (int j = 0; j < 4; j++) {  // inclusive sum over s of row 4c+j
      uint32_t v = d[j];
      uint32_t t = __shfl_up_sync(kFull, v, 8);
      if (s >= 1) v += t;
      t = __shfl_up_sync(kFull, v, 16);
      if (s >= 2) v += t;
      q[j] = v;
    }
    uint32_t rr_prev[4], acc = 0;
#pragma unroll
    for (int j = 0; j < 4; j++) {
      rr_prev[j] = acc;
      acc += __shfl_sync(kFull, q[j], 24 + c);  // the row's total
    }
    const uint32_t e = col_excl(acc, lane);
#pragma unroll
    for (int j = 0; j < 4; j++) x[j] = s0 + e + rr_prev[j] + q[j];
    uint32_t t = d[0] + d[1] + d[2] + d[3];
    t += __shfl_xor_sync(kFull, t, 1);
    t += __shfl_xor_sync(kFull, t, 2);
    t += __shfl_xor_sync(kFull, t, 4);
    ctot = t;
  }
}

// Values of a GL block of width B and kind KIND (all seeds F).
template <int B, int KIND, class L>
__device__ __forceinline__ void gl_lane_values_kind(const L &ld, uint32_t F, int lane,
                                                    uint32_t x[4]) {
  uint32_t d[4], ctot;
  gl_lane_deltas<B>(ld, lane, d);
  prefix_block<KIND>(d, F, lane, x, ctot);
}

template <int KIND, class L>
__device__ __forceinline__ void gl_block_values_kind(int b, const L &ld, uint32_t F, int lane,
                                                     uint32_t x[4]) {
  switch (b) {
#define BP_CASE(B) \
  case B:          \
    gl_lane_values_kind<B, KIND>(ld, F, lane, x); \
    break;
    BP_CASE(0) BP_CASE(1) BP_CASE(2) BP_CASE(3) BP_CASE(4) BP_CASE(5) BP_CASE(6)
    BP_CASE(7) BP_CASE(8) BP_CASE(9) BP_CASE(10) BP_CASE(11) BP_CASE(12) BP_CASE(13)
    BP_CASE(14) BP_CASE(15) BP_CASE(16) BP_CASE(17) BP_CASE(18) BP_CASE(19) BP_CASE(20)
    BP_CASE(21) BP_CASE(22) BP_CASE(23) BP_CASE(24) BP_CASE(25) BP_CASE(26) BP_CASE(27)
    BP_CASE(28) BP_CASE(29) BP_CASE(30) BP_CASE(31) BP_CASE(32)
#undef BP_CASE
    default:
      x[0] = x[1] = x[2] = x[3] = 0u;
  }
}

// Runtime-width dispatch (b is warp-uniform, so the switch never diverges).
template <class L>
__device__ __forceinline__ void gl_block_values_from(int b, const L &ld, uint32_t F, int lane,
                                                     uint32_t x[4]) {
  switch (b) {
#define BP_CASE(B) \
  case B:          \
    gl_lane_values<B>(ld, F, lane, x); \
    break;
    BP_CASE(0) BP_CASE(1) BP_CASE(2) BP_CASE(3) BP_CASE(4) BP_CASE(5) BP_CASE(6)
    BP_CASE(7) BP_CASE(8) BP_CASE(9) BP_CASE(10) BP_CASE(11) BP_CASE(12) BP_CASE(13)
    BP_CASE(14) BP_CASE(15) BP_CASE(16) BP_CASE(17) BP_CASE(18) BP_CASE(19) BP_CASE(20)
    BP_CASE(21) BP_CASE(22) BP_CASE(23) BP_CASE(24) BP_CASE(25) BP_CASE(26) BP_CASE(27)
    BP_CASE(28) BP_CASE(29) BP_CASE(30) BP_CASE(31) BP_CASE(32)
#undef BP_CASE
    default:
      x[0] = x[1] = x[2] = x[3] = 0u;
  }
}

__device__ __forceinline__ void gl_block_values(int b, const uint32_t *__restrict__ w,
                                                uint32_t F, int lane, uint32_t x[4]) {
  gl_block_values_from(b, GlobalWords{w}, F, lane, x);
}

// The same with the width known only at run time: no per-width code, so a
// few dozen instructions instead of 33 specialised routines -- for kernels
// whose instruction footprint matters more than the last shift (the
// intersections decode blocks at several call sites).  Lane l's value j
// sits at bit 4bl + jb of the block's words w[0..4b).  Up to b = 8 the
// lane's 4b bits are read as one 32-bit window (one or two loads); wider
// blocks read each field's word pair.
__device__ __forceinline__ void gl_block_values_rt(uint32_t b, const uint32_t *__restrict__ w,
                                                   uint32_t F, int lane, uint32_t x[4]) {
  uint32_t d[4] = {0u, 0u, 0u, 0u};
  if (b != 0u && b <= 8u) {
    // the lane's 4b <= 32 bits lie in one 32-bit window of the stream: one
    // or two loads and one funnel shift, then the four fields
    const uint32_t p = 4u * b * (uint32_t)lane, k = p >> 5, o = p & 31u;
    const uint32_t lo = __ldg(w + k);
    const uint32_t hi = (o + 4u * b > 32u) ? __ldg(w + k + 1) : 0u;  // still in the lane's bits
    const uint32_t u = __funnelshift_r(lo, hi, o);
    const uint32_t mask = (1u << b) - 1u;
#pragma unroll
    for (int j = 0; j < 4; j++) d[j] = (u >> (b * (uint32_t)j)) & mask;
  } else if (b != 0u) {
    const uint32_t mask = b >= 32u ? 0xFFFFFFFFu : (1u << b) - 1u;
    uint32_t bit = 4u * b * (uint32_t)lane;
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const uint32_t k = bit >> 5, r = bit & 31u;
      const uint32_t lo = __ldg(w + k);
      const uint32_t hi = (r + b > 32u) ? __ldg(w + k + 1) : 0u;
      d[j] = __funnelshift_r(lo, hi, r) & mask;
      bit += b;
    }
  }
  x[0] = d[0];
  x[1] = x[0] + d[1];
  x[2] = x[1] + d[2];
  x[3] = x[2] + d[3];
  const int c = lane & 7;
  uint32_t incl = x[3];
#pragma unroll
  for (int dd = 1; dd < 8; dd <<= 1) {
    const uint32_t t = __shfl_up_sync(kFull, incl, dd, 8);
    if (c >= dd) incl += t;
  }
  const uint32_t base = F + (incl - x[3]);
#pragma unroll
  for (int j = 0; j < 4; j++) x[j] += base;
}

// In-block position of x[j] for `lane`.
__device__ __forceinline__ int gl_pos(int lane, int j) { return 16 * (lane & 7) + 4 * j + (lane >> 3); }

// Superblock q of a GL list as seen by one warp: every lane holds the width,
// first value and payload word offset of block 32q + lane.  Returns false
// (and records BP_ERR_CORRUPT) if the widths or offsets are inconsistent.
struct SuperInfo {
  uint32_t nblk;  // blocks in this superblock (1..32)
  uint32_t b, F, woff;  // per lane
};

__device__ __forceinline__ bool gl_super(const GlView &v, uint32_t q, int lane, SuperInfo &si,
                                         uint32_t *status) {
  const uint32_t k0 = q * 32u;
  si.nblk = min(32u, v.nblocks - k0);
  uint32_t b = 0, F = 0;
  if ((uint32_t)lane < si.nblk) {
    b = v.bw[k0 + lane];
    F = __ldg(v.first + k0 + lane);
  }
  uint32_t incl = 4u * b;
#pragma unroll
  for (int dd = 1; dd < 32; dd <<= 1) {
    const uint32_t t = __shfl_up_sync(kFull, incl, dd);
    if (lane >= dd) incl += t;
  }
  const uint32_t total = __shfl_sync(kFull, incl, 31);
  const uint32_t base = __ldg(v.sbo + q), end = __ldg(v.sbo + q + 1);
  const bool bad = __any_sync(kFull, b > 32u) || end < base || end - base != total || end > v.pw;
  if (bad) {
    if (lane == 0) set_status(status, BP_ERR_CORRUPT);
    return false;
  }
  si.b = b;
  si.F = F;
  si.woff = base + incl - 4u * b;
  return true;
}

}  // namespace bp
