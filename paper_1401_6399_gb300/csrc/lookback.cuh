// lookback.cuh -- single-pass ordered compaction across CTAs: every tile
// takes a ticket (so tiles start in order and a tile only ever waits on
// tiles that are already running), publishes its count, then looks back
// over earlier tiles for the number of outputs before it.
//
// Tile state word (u64): flag << 32 | value; flag 1 = the tile's own count,
// 2 = inclusive count of all tiles up to it.  The words and the ticket live
// in caller scratch and are zeroed by the host before each launch.  Every
// wait is bounded: after `spin_limit` polls (kLookbackSpinLimit unless the
// tuning sets another) it records BP_ERR_TIMEOUT and proceeds as if the
// missing tile had no output.  For testing that path the tuning can name a
// tile that publishes nothing (Compaction::withhold), so that the tiles
// after it run out of polls.
#pragma once
#include "common.cuh"
#include "tuning.h"

namespace bp {

__device__ __forceinline__ uint64_t ld_acquire_u64(const uint64_t *p) {
  uint64_t v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_u64(uint64_t *p, uint64_t v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Called by all 32 lanes of one warp of tile t with the tile's own count;
// returns the number of outputs of tiles 0..t-1.  Each step inspects the 32
// nearest tiles not yet accounted for (lane i: tile top - i), adds their
// counts down to the nearest inclusive one and stops there, or moves 32
// tiles back.
// Scratch of one compaction: ticket counter + one state word per tile, and
// the limits of the look-back's waits.
struct Compaction {
  uint32_t *ticket;
  uint64_t *state;
  uint32_t spin_limit;  // polls of one state word before giving up
  uint32_t withhold;    // tile that publishes nothing (testing), or UINT32_MAX
};

__device__ __forceinline__ uint32_t lookback_exclusive_warp(const Compaction &cp, uint32_t t,
                                                           uint32_t agg, uint32_t *status,
                                                           int lane) {
  uint64_t *state = cp.state;
  const bool publish = t != cp.withhold;
  if (t == 0) {
    if (lane == 0 && publish) st_release_u64(state, (2ull << 32) | agg);
    return 0;
  }
  if (lane == 0 && publish) st_release_u64(state + t, (1ull << 32) | agg);
  uint32_t excl = 0;
  for (int64_t top = (int64_t)t - 1; top >= 0; top -= 32) {
    const int64_t j = top - lane;
    uint64_t s = 2ull << 32;  // before tile 0: an inclusive count of zero
    if (j >= 0) {
      uint32_t spins = 0;
      while (((s = ld_acquire_u64(state + j)) >> 32) == 0) {
        if (++spins > cp.spin_limit) break;
        __nanosleep(64);
      }
    }
    const uint32_t flag = (uint32_t)(s >> 32);
    if (__any_sync(kFull, flag == 0)) {
      if (lane == 0) set_status(status, BP_ERR_TIMEOUT);
      break;
    }
    const uint32_t incl = __ballot_sync(kFull, flag == 2);
    const int stop = incl ? __ffs(incl) - 1 : 31;
    excl += __reduce_add_sync(kFull, lane <= stop ? (uint32_t)s : 0u);
    if (incl) break;
  }
  if (lane == 0 && publish) st_release_u64(state + t, (2ull << 32) | (excl + agg));
  return excl;
}

__host__ __device__ inline size_t compaction_bytes(uint64_t ntiles) { return 16 + 8 * ntiles; }

inline Compaction compaction_at(void *p) {
  Compaction c;
  c.ticket = static_cast<uint32_t *>(p);
  c.state = reinterpret_cast<uint64_t *>(static_cast<uint8_t *>(p) + 16);
  lookback_limits(c.spin_limit, c.withhold);
  return c;
}

}  // namespace bp
