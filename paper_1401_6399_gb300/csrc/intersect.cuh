// intersect.cuh -- warp-level pieces of the intersection kernels, shared by
// the pairwise and the batched query paths.
//
// Section 6: the short list r drives the search; for each r_i we need the
// first f_j >= r_i.  On the GPU a warp takes 128 consecutive values of r
// (one GL block, or 128 decoded values) and:
//  - finds the range of f that can hold them with a 32-way search over f's
//    per-block first values (the GL skip headers) or over decoded f;
//  - "dense" regime (similar lengths, cf. V1/V3): the few blocks of f in that
//    range are decoded into shared memory and every r value is searched
//    there;
//  - "sparse" regime (skewed lengths, cf. galloping / SIMD Galloping): each
//    r value locates its candidate block by binary search over the skip
//    headers, and only the distinct candidate blocks are decoded.
// The span threshold between the regimes is a tuning parameter.
#pragma once
#include "gl_block.cuh"
#include "lookback.cuh"

namespace bp {

constexpr int kIxWarps = 8;
constexpr int kIxThreads = 32 * kIxWarps;
constexpr int kIxDenseMax = 8;  // largest dense span in blocks (smem per warp)

__device__ __forceinline__ int64_t imax64(int64_t a, int64_t b) { return a > b ? a : b; }

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Largest k in [0, n) with a[k] <= v, or -1.  Warp-cooperative 32-way search
// (each round probes 32 evenly spaced entries); v is warp-uniform.
__device__ __forceinline__ int64_t warp_ubound(const uint32_t *__restrict__ a, uint64_t n,
                                               uint32_t v, int lane) {
  uint64_t lo = 0, hi = n;  // answer in [lo-1, hi-1]
  while (hi - lo > 32) {
    const uint64_t step = (hi - lo + 31) / 32;
    const uint64_t p = lo + (uint64_t)lane * step;
    const bool le = p < hi && __ldg(a + p) <= v;
    const uint32_t cnt = __popc(__ballot_sync(kFull, le));
    if (cnt == 0) return (int64_t)lo - 1;
    const uint64_t nlo = lo + (uint64_t)(cnt - 1) * step + 1;
    hi = min(hi, lo + (uint64_t)cnt * step);
    lo = nlo;
  }
  const bool le = lo + lane < hi && __ldg(a + lo + lane) <= v;
  return (int64_t)lo - 1 + __popc(__ballot_sync(kFull, le));
}

// Largest k in [lo, hi] with a[k] <= v, or lo-1 (per lane).
__device__ __forceinline__ int64_t lane_ubound(const uint32_t *__restrict__ a, int64_t lo,
                                               int64_t hi, uint32_t v) {
  int64_t L = lo, H = hi + 1;  // first index with a > v in [L, H]
  while (L < H) {
    const int64_t mid = (L + H) >> 1;
    if (__ldg(a + mid) <= v) L = mid + 1;
    else H = mid;
  }
  return L - 1;
}

// Is v among s[0..len)?  (s ascending, in shared memory)
__device__ __forceinline__ bool smem_contains(const uint32_t *s, uint32_t len, uint32_t v) {
  uint32_t L = 0, H = len;
  while (L < H) {
    const uint32_t mid = (L + H) >> 1;
    if (s[mid] < v) L = mid + 1;
    else H = mid;
  }
  return L < len && s[L] == v;
}

__device__ __forceinline__ bool gmem_contains(const uint32_t *__restrict__ a, int64_t lo,
                                              int64_t hi, uint32_t v) {
  int64_t L = lo, H = hi + 1;  // first a >= v in [lo, hi+1]
  while (L < H) {
    const int64_t mid = (L + H) >> 1;
    if (__ldg(a + mid) < v) L = mid + 1;
    else H = mid;
  }
  return L <= hi && __ldg(a + L) == v;
}

// Decode block k of GL list v into dst[0..128) (natural order) with the
// whole warp; returns the number of real values in it (0 if the block's
// header is inconsistent, which is also recorded as BP_ERR_CORRUPT).
__device__ __forceinline__ uint32_t gl_block_into(const GlView &v, uint32_t k, uint32_t *dst,
                                                  int lane, uint32_t *status) {
  const uint32_t q = k >> 5, j = k & 31u, k0 = q << 5;
  const uint32_t bl = (k0 + lane < v.nblocks) ? (uint32_t)v.bw[k0 + lane] : 0u;
  const uint32_t part = ((uint32_t)lane < j) ? 4u * bl : 0u;
  const uint32_t woff = __ldg(v.sbo + q) + __reduce_add_sync(kFull, part);
  const uint32_t b = __shfl_sync(kFull, bl, j);
  if (b > 32u || woff + 4u * b > v.pw) {
    if (lane == 0) set_status(status, BP_ERR_CORRUPT);
    return 0;
  }
  uint32_t x[4];
  gl_block_values((int)b, v.payload + woff, __ldg(v.first + k), lane, x);
#pragma unroll
  for (int t = 0; t < 4; t++) dst[gl_pos(lane, t)] = x[t];
  return min(128u, v.n - 128u * k);
}

// Membership of the warp's values (lane holds positions 32k + lane, k < 4,
// valid where valid[k]) in GL list f.  smem: kIxDenseMax*128 words of this
// warp.  dense_max: span threshold of the dense regime.
__device__ __forceinline__ void gl_membership(const GlView &f, const uint32_t v[4],
                                              const bool valid[4], bool hit[4], uint32_t rmin,
                                              uint32_t rmax, uint32_t *smem, int lane,
                                              uint32_t dense_max, uint32_t *status) {
#pragma unroll
  for (int k = 0; k < 4; k++) hit[k] = false;
  if (f.nblocks == 0) return;
  const int64_t khi = warp_ubound(f.first, f.nblocks, rmax, lane);
  if (khi < 0) return;
  const int64_t klo = imax64(0, warp_ubound(f.first, f.nblocks, rmin, lane));
  const uint64_t span = (uint64_t)(khi - klo + 1);
  if (span <= dense_max) {
    uint32_t len = 0;
    for (uint32_t i = 0; i < (uint32_t)span; i++) {
      const uint32_t c = gl_block_into(f, (uint32_t)klo + i, smem + 128u * i, lane, status);
      len = 128u * i + c;
      if (c < 128u) break;  // only the last block of f is short
    }
    __syncwarp();
#pragma unroll
    for (int k = 0; k < 4; k++) hit[k] = valid[k] && smem_contains(smem, len, v[k]);
    __syncwarp();
    return;
  }
  int64_t cb[4];
  bool pend[4];
#pragma unroll
  for (int k = 0; k < 4; k++) {
    cb[k] = valid[k] ? lane_ubound(f.first, klo, khi, v[k]) : klo - 1;
    pend[k] = valid[k] && cb[k] >= klo;
  }
  for (;;) {
    int64_t blk = -1;
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const uint32_t m = __ballot_sync(kFull, pend[k]);
      if (blk < 0 && m) blk = __shfl_sync(kFull, cb[k], __ffs(m) - 1);
    }
    if (blk < 0) break;
    const uint32_t c = gl_block_into(f, (uint32_t)blk, smem, lane, status);
    __syncwarp();
#pragma unroll
    for (int k = 0; k < 4; k++)
      if (pend[k] && cb[k] == blk) {
        hit[k] = smem_contains(smem, c, v[k]);
        pend[k] = false;
      }
    __syncwarp();
  }
}

// Same for a decoded, sorted f in global memory.
__device__ __forceinline__ void raw_membership(const uint32_t *__restrict__ f, uint64_t nf,
                                               const uint32_t v[4], const bool valid[4],
                                               bool hit[4], uint32_t rmin, uint32_t rmax,
                                               uint32_t *smem, int lane, uint32_t dense_max) {
#pragma unroll
  for (int k = 0; k < 4; k++) hit[k] = false;
  if (nf == 0) return;
  const int64_t hi = warp_ubound(f, nf, rmax, lane);
  if (hi < 0) return;
  const int64_t lo = imax64(0, warp_ubound(f, nf, rmin, lane));
  const uint64_t span = (uint64_t)(hi - lo + 1);
  if (span <= 128ull * dense_max) {
    for (uint32_t i = lane; i < span; i += 32) smem[i] = __ldg(f + lo + i);
    __syncwarp();
#pragma unroll
    for (int k = 0; k < 4; k++) hit[k] = valid[k] && smem_contains(smem, (uint32_t)span, v[k]);
    __syncwarp();
    return;
  }
#pragma unroll
  for (int k = 0; k < 4; k++) hit[k] = valid[k] && gmem_contains(f, lo, hi, v[k]);
}

// Ordered output of one tile (all threads of the CTA call it).  Lane holds
// positions 32k + lane of its warp's chunk; chunks are in warp order.
struct TileOut {
  uint32_t *out;
  uint64_t out_cap;
  uint32_t *count;  // written by the last tile
  uint32_t *status;
};

__device__ __forceinline__ void tile_emit(const uint32_t v[4], const bool hit[4], uint32_t t,
                                          bool last_tile, const Compaction &cp, const TileOut &to,
                                          uint32_t *s_wcnt, uint32_t *s_base) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t m[4], tot = 0;
#pragma unroll
  for (int k = 0; k < 4; k++) {
    m[k] = __ballot_sync(kFull, hit[k]);
    tot += __popc(m[k]);
  }
  if (lane == 0) s_wcnt[w] = tot;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    for (int i = 0; i < kIxWarps; i++) {
      const uint32_t c = s_wcnt[i];
      s_wcnt[i] = run;
      run += c;
    }
    const uint32_t P = lookback_exclusive(cp.state, t, run, to.status);
    s_base[0] = P;
    if (last_tile) {
      *to.count = P + run;
      if ((uint64_t)P + run > to.out_cap) set_status(to.status, BP_ERR_CAPACITY);
    }
  }
  __syncthreads();
  uint64_t pos = (uint64_t)s_base[0] + s_wcnt[w];
#pragma unroll
  for (int k = 0; k < 4; k++) {
    if (hit[k]) {
      const uint64_t idx = pos + __popc(m[k] & lanemask_lt());
      if (idx < to.out_cap) to.out[idx] = v[k];
    }
    pos += __popc(m[k]);
  }
}

}  // namespace bp
