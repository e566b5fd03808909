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

// For each of a lane's four values, the largest k in [lo, hi] with
// a[k] <= v[k] (lo - 1 if none, or if !valid[k]): four searches by halving
// over the same range, interleaved so that their global loads overlap; the
// range is the same in every lane.
__device__ __forceinline__ void lane_ubound4(const uint32_t *__restrict__ a, int64_t lo,
                                             int64_t hi, const uint32_t v[4],
                                             const bool valid[4], int64_t cb[4]) {
  int64_t base[4] = {lo, lo, lo, lo};
  int64_t n = hi - lo + 1;  // the upper bound of v[k] lies in [base[k], base[k] + n]
  while (n > 1) {
    const int64_t half = n >> 1;
#pragma unroll
    for (int k = 0; k < 4; k++)
      base[k] = (__ldg(a + base[k] + half - 1) <= v[k]) ? base[k] + half : base[k];
    n -= half;
  }
#pragma unroll
  for (int k = 0; k < 4; k++) {
    const int64_t ub = base[k] + ((n == 1 && __ldg(a + base[k]) <= v[k]) ? 1 : 0);
    cb[k] = valid[k] ? ub - 1 : lo - 1;
  }
}

// Which of a lane's four values are among s[0..len) (s ascending, in shared
// memory): four lower-bound searches by halving, interleaved so that their
// shared-memory loads overlap; the number of steps depends only on len (the
// same in every lane).
__device__ __forceinline__ void smem_contains4(const uint32_t *s, uint32_t len,
                                               const uint32_t v[4], const bool valid[4],
                                               bool hit[4]) {
  if (len == 0) {
#pragma unroll
    for (int k = 0; k < 4; k++) hit[k] = false;
    return;
  }
  uint32_t base[4] = {0u, 0u, 0u, 0u};
  uint32_t n = len;
  while (n > 1) {  // invariant: the lower bound of v[k] lies in [base[k], base[k] + n]
    const uint32_t half = n >> 1;
#pragma unroll
    for (int k = 0; k < 4; k++) base[k] = (s[base[k] + half - 1] < v[k]) ? base[k] + half : base[k];
    n -= half;
  }
#pragma unroll
  for (int k = 0; k < 4; k++) {
    const uint32_t lb = base[k] + (s[base[k]] < v[k] ? 1u : 0u);
    hit[k] = valid[k] && lb < len && s[lb] == v[k];
  }
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
// header is inconsistent, which is also recorded as BP_ERR_CORRUPT).  The
// width is handled at run time (gl_block_values_rt): the intersection
// kernels decode blocks at several call sites, and 33 specialised unpackers
// per site made the batched-query kernel stall on instruction fetch
// (measured: +9 % queries/s with the run-time width).
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
  gl_block_values_rt(b, v.payload + woff, __ldg(v.first + k), lane, x);
#pragma unroll
  for (int t = 0; t < 4; t++) dst[gl_pos(lane, t)] = x[t];
  return min(128u, v.n - 128u * k);
}

// Payload word offset of block k of GL list v (the superblock's offset plus
// 4x the widths of the blocks before k in it), computed by one lane.
__device__ __forceinline__ uint32_t gl_block_woff(const GlView &v, uint32_t k) {
  const uint32_t q = k >> 5, j = k & 31u;
  const uint4 *w4 = reinterpret_cast<const uint4 *>(v.bw + 32u * q);
  const uint4 a = __ldg(w4), b = (j > 16u) ? __ldg(w4 + 1) : make_uint4(0, 0, 0, 0);
  const uint32_t wd[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
  uint32_t sum = 0;
#pragma unroll
  for (int i = 0; i < 8; i++) {
    const uint32_t lo = 4u * i;  // bytes lo..lo+3 of the 32 widths
    const uint32_t keep = j >= lo + 4u ? 0xFFFFFFFFu : (j <= lo ? 0u : (0xFFFFFFFFu >> (8u * (4u - (j - lo)))));
    sum = __dp4a(wd[i] & keep, 0x01010101u, sum);
  }
  return __ldg(v.sbo + q) + 4u * sum;
}

// Is p in block k of GL list v?  Four lanes (column s = lane & 3 each) decode
// their column of the block -- the contiguous bit string [32bs, 32b(s+1)),
// a running sum from the block's first value -- and stop as soon as the
// increasing column reaches p.  Returns the lookup's answer in all 4 lanes.
__device__ __forceinline__ bool column_lookup(const GlView &v, uint32_t k, uint32_t p,
                                              bool active, int lane, uint32_t *status) {
  const uint32_t s = lane & 3u;
  bool found = false;
  if (active) {
    const uint32_t b = v.bw[k];
    const uint32_t woff = gl_block_woff(v, k);
    if (b > 32u || woff + 4u * b > v.pw) {
      set_status(status, BP_ERR_CORRUPT);
    } else {
      const uint32_t F = __ldg(v.first + k);
      const uint32_t cnt = min(128u, v.n - 128u * k);
      const uint32_t *w = v.payload + woff + b * s;
      const uint32_t nw = b;  // words of this column
      uint32_t wi = 0;
      uint32_t lo = nw > 0 ? __ldg(w) : 0u, hi = nw > 1 ? __ldg(w + 1) : 0u;
      uint32_t nx = nw > 2 ? __ldg(w + 2) : 0u;
      const uint32_t mask = b >= 32u ? 0xFFFFFFFFu : ((1u << b) - 1u);
      uint32_t off = 0, x = F;
      for (uint32_t t = 0; t < 32u; t++) {
        x += __funnelshift_r(lo, hi, off) & mask;
        if (4u * t + s >= cnt) break;  // past the block's last value
        if (x >= p) {
          found = (x == p);
          break;
        }
        off += b;
        if (off >= 32u) {
          off -= 32u;
          lo = hi;
          hi = nx;
          wi++;
          nx = (wi + 2u < nw) ? __ldg(w + wi + 2u) : 0u;
        }
      }
    }
  }
  const uint32_t grp = 0xFu << (lane & ~3);
  return (__ballot_sync(kFull, found) & grp) != 0;
}

// Resolve the probes of a warp (lane holds positions 32k + lane; cb[k] its
// candidate block, < klo when there is none) eight at a time: probe i of a
// round goes to lanes 4i..4i+3.  The loop over the lane's four registers is
// kept rolled (the values are picked by selects): one copy of the probe
// code instead of four keeps the calling kernels' code small.
__device__ __forceinline__ void lookup_probes(const GlView &f, const uint32_t v[4],
                                              const bool valid[4], const int64_t cb[4],
                                              int64_t klo, bool hit[4], int lane,
                                              uint32_t *status) {
  uint32_t hits = 0;
#pragma unroll 1
  for (int k = 0; k < 4; k++) {
    const uint32_t vk = k == 0 ? v[0] : k == 1 ? v[1] : k == 2 ? v[2] : v[3];
    const int64_t ck = k == 0 ? cb[0] : k == 1 ? cb[1] : k == 2 ? cb[2] : cb[3];
    const bool ok = k == 0 ? valid[0] : k == 1 ? valid[1] : k == 2 ? valid[2] : valid[3];
    uint32_t pend = __ballot_sync(kFull, ok && ck >= klo);  // probes of this register
    while (pend) {                                           // up to 8 per round
      // the i-th set bit of pend goes to lane group i
      const int g = lane >> 2;
      uint32_t m = pend;
      for (int i = 0; i < g && m; i++) m &= m - 1;
      const bool act = m != 0;
      const int src = act ? __ffs(m) - 1 : 0;
      const uint32_t pv = __shfl_sync(kFull, vk, src);
      const uint32_t pb = (uint32_t)__shfl_sync(kFull, (uint32_t)ck, src);
      const bool found = column_lookup(f, pb, pv, act, lane, status);
      // hand each answer back to the lane that owns the probe
      const uint32_t ans = __ballot_sync(kFull, act && (lane & 3) == 0 && found);
      // lane L owns probe number r = popc(pend & lanemask_lt(L)) of this round
      if (pend & (1u << lane)) {
        const uint32_t r = __popc(pend & ((1u << lane) - 1u));
        if (r < 8u && ((ans >> (4u * r)) & 1u)) hits |= 1u << k;
      }
      // drop the (up to 8) probes handled this round
      for (int i = 0; i < 8 && pend; i++) pend &= pend - 1;
    }
  }
#pragma unroll
  for (int k = 0; k < 4; k++) hit[k] = (hits >> k) & 1u;
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
    smem_contains4(smem, len, v, valid, hit);
    __syncwarp();
    return;
  }
  // sparse regime: every value looks up its own candidate block
  int64_t cb[4];
  lane_ubound4(f.first, klo, khi, v, valid, cb);
  lookup_probes(f, v, valid, cb, klo, hit, lane, status);
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
    smem_contains4(smem, (uint32_t)span, v, valid, hit);
    __syncwarp();
    return;
  }
#pragma unroll
  for (int k = 0; k < 4; k++) hit[k] = valid[k] && gmem_contains(f, lo, hi, v[k]);
}

// Decoded blocks [lo, hi] of f held in a warp's shared-memory window (none
// if hi < lo).  A warp that filters increasing runs of values through the
// same f keeps the window from one run to the next: runs of similar density
// move it forward a block or two at a time.
struct FWin {
  int64_t lo, hi;
  uint32_t len;       // decoded values in the window
  uint32_t first_lo;  // f.first[lo]
};

__device__ __forceinline__ FWin fwin_empty() {
  FWin w;
  w.lo = 0;
  w.hi = -1;
  w.len = 0;
  w.first_lo = 0;
  return w;
}

// Largest k in [h, n) with a[k] <= v, given a[h] <= v: one probe of the 32
// entries from h, then the 32-way search beyond them.
__device__ __forceinline__ int64_t fwd_ubound(const uint32_t *__restrict__ a, uint64_t n,
                                              uint32_t v, int64_t h, int lane) {
  const uint64_t p = (uint64_t)h + lane;
  const bool le = p < n && __ldg(a + p) <= v;
  const uint32_t c = __popc(__ballot_sync(kFull, le));
  if (c < 32u) return h + (int64_t)c - 1;
  const uint64_t base = (uint64_t)h + 32;
  return (int64_t)base + warp_ubound(a + base, n - base, v, lane);
}

// As gl_membership (dense or sparse by the span of f's blocks that can hold
// [rmin, rmax]), with the dense blocks kept in `win` over `smem`
// (kIxDenseMax * 128 words of this warp) for the next call: blocks already
// decoded are not decoded again, and the block range is found by probing
// forward from the window.  Runs must come in increasing order of values.
__device__ __forceinline__ void gl_membership_win(const GlView &f, const uint32_t v[4],
                                                  const bool valid[4], bool hit[4], uint32_t rmin,
                                                  uint32_t rmax, uint32_t *smem, FWin &win,
                                                  int lane, uint32_t dense_max, uint32_t *status) {
#pragma unroll
  for (int k = 0; k < 4; k++) hit[k] = false;
  if (f.nblocks == 0) return;
  const bool have = win.hi >= win.lo;
  int64_t klo = (have && win.first_lo <= rmin) ? fwd_ubound(f.first, f.nblocks, rmin, win.lo, lane)
                                              : warp_ubound(f.first, f.nblocks, rmin, lane);
  int64_t khi;
  if (klo >= 0) {
    khi = fwd_ubound(f.first, f.nblocks, rmax, klo, lane);
  } else {
    khi = warp_ubound(f.first, f.nblocks, rmax, lane);
    if (khi < 0) return;  // every value is below f's first value
    klo = 0;
  }
  if (!(have && klo >= win.lo && khi <= win.hi)) {
    const uint64_t span = (uint64_t)(khi - klo + 1);
    if (span > dense_max) {  // sparse: every value looks up its own candidate block
      int64_t cb[4];
      lane_ubound4(f.first, klo, khi, v, valid, cb);
      lookup_probes(f, v, valid, cb, klo, hit, lane, status);
      return;
    }
    // refill the window with blocks [klo, khi]; blocks it already holds move
    // to the front instead of being decoded again
    uint32_t keep = 0;
    if (have && klo >= win.lo && klo <= win.hi) {
      keep = (uint32_t)((win.hi < khi ? win.hi : khi) - klo + 1);
      const uint32_t from = 128u * (uint32_t)(klo - win.lo), words = 128u * keep;
      if (from) {
        for (uint32_t i0 = 0; i0 < words; i0 += 32) {
          const uint32_t i = i0 + lane;
          const uint32_t x = i < words ? smem[from + i] : 0u;
          __syncwarp();
          if (i < words) smem[i] = x;
          __syncwarp();
        }
      }
    }
    uint32_t len = 128u * keep;
    if (keep && (uint64_t)klo + keep == f.nblocks) len = 128u * (keep - 1) + (f.n - 128u * (f.nblocks - 1));
    for (uint32_t i = keep; i < (uint32_t)span; i++) {
      const uint32_t c = gl_block_into(f, (uint32_t)klo + i, smem + 128u * i, lane, status);
      len = 128u * i + c;
      if (c < 128u) break;  // only the last block of f is short
    }
    __syncwarp();
    win.lo = klo;
    win.hi = khi;
    win.len = len;
    win.first_lo = __ldg(f.first + klo);
  }
  smem_contains4(smem, win.len, v, valid, hit);
  __syncwarp();
}

// ---- merge regime (similar lengths; Section 6's scalar merge, split over
// the lanes of a warp by merge path) ----

// Smallest i in [lo, hi) with s[i] >= v (hi if none): warp-cooperative
// 32-way search over a sorted shared-memory array; v is warp-uniform.
__device__ __forceinline__ uint32_t smem_lbound_warp(const uint32_t *s, uint32_t lo, uint32_t hi,
                                                     uint32_t v, int lane) {
  while (hi - lo > 32) {
    const uint32_t step = (hi - lo + 31) / 32;
    const uint32_t p = lo + (uint32_t)lane * step;
    const bool lt = p < hi && s[p] < v;
    const uint32_t cnt = __popc(__ballot_sync(kFull, lt));
    if (cnt == 0) return lo;
    const uint32_t nlo = lo + (cnt - 1) * step + 1;
    hi = min(hi, lo + cnt * step);
    lo = nlo;
  }
  const bool lt = lo + lane < hi && s[lo + lane] < v;
  return lo + __popc(__ballot_sync(kFull, lt));
}

// Intersection of two sorted runs in shared memory, A[0..na) and B[0..nb)
// (distinct values within each), by merging: the merged sequence (A before B
// on ties) is cut into 32 equal parts, each lane finds where its part starts
// by binary search on the cross diagonal and merges it.  When A[i] is taken,
// every B before the next one not yet taken is below A[i], so A[i] is in B
// exactly when that next B equals it.  Sets bit abase + i of `hits` for each
// such A[i].
__device__ __forceinline__ void merge_path_hits(const uint32_t *A, uint32_t na, const uint32_t *B,
                                                uint32_t nb, uint32_t *hits, uint32_t abase,
                                                int lane) {
  const uint32_t T = na + nb;
  const uint32_t per = (T + 31) >> 5;
  const uint32_t d0 = min((uint32_t)lane * per, T), d1 = min(d0 + per, T);
  uint32_t lo = d0 > nb ? d0 - nb : 0u, hi = min(d0, na);  // A's share of the first d0
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (A[mid] <= B[d0 - mid - 1]) lo = mid + 1;
    else hi = mid;
  }
  uint32_t i = lo, j = d0 - lo;
  uint32_t a = i < na ? A[i] : 0u, b = j < nb ? B[j] : 0u;
  // one step per merged value, without branches: the lanes take A or B
  // independently, so a branch per side would run both sides every step
  for (uint32_t s = d0; s < d1; s++) {
    const bool take_a = i < na && (j >= nb || a <= b);
    if (take_a && j < nb && a == b)
      atomicOr(hits + ((abase + i) >> 5), 1u << ((abase + i) & 31u));
    const uint32_t ni = i + (take_a ? 1u : 0u), nj = j + (take_a ? 0u : 1u);
    const bool in = take_a ? ni < na : nj < nb;
    const uint32_t x = in ? (take_a ? A[ni] : B[nj]) : 0u;
    a = take_a ? x : a;
    b = take_a ? b : x;
    i = ni;
    j = nj;
  }
}

// Which values of a warp's sorted run A[0..na) (shared memory) are in GL
// list f.  kfirst: the block of f holding A[0] (-1 if A[0] is below f's
// first value); klast >= 0: the block holding A[na-1].  f's blocks between
// them are decoded window by window (up to kIxDenseMax blocks into smem) and
// each window is merged with the part of A inside its value range.  A window
// ends before the block that holds the first value of A beyond it, so no
// block is decoded twice.  Sets bit i of `hits` (zeroed by the caller) for
// each A[i] in f.  Kept out of line: one copy of its code per kernel, away
// from the hot loops of the other regimes.
static __device__ __noinline__ void merge_run_hits(const GlView &f, const uint32_t *A, uint32_t na,
                                                      int64_t kfirst, int64_t klast, uint32_t *smem,
                                                      uint32_t *hits, int lane, uint32_t *status) {
  uint32_t a0 = 0;
  int64_t klo = kfirst;
  if (kfirst < 0) {  // values below f's first one cannot match
    a0 = smem_lbound_warp(A, 0, na, __ldg(f.first), lane);
    if (a0 >= na) return;
    klo = warp_ubound(f.first, f.nblocks, A[a0], lane);
  }
  while (true) {
    const int64_t khi = klo + kIxDenseMax - 1 < klast ? klo + kIxDenseMax - 1 : klast;
    uint32_t len = 0;
    for (int64_t k = klo; k <= khi; k++) {
      const uint32_t i = (uint32_t)(k - klo);
      const uint32_t c = gl_block_into(f, (uint32_t)k, smem + 128u * i, lane, status);
      len = 128u * i + c;
      if (c < 128u) break;  // only f's last block is short (or a corrupt one)
    }
    __syncwarp();
    const bool more = khi + 1 < (int64_t)f.nblocks;
    const uint32_t a1 = more ? smem_lbound_warp(A, a0, na, __ldg(f.first + khi + 1), lane) : na;
    const uint32_t b0 = smem_lbound_warp(smem, 0, len, A[a0], lane);
    merge_path_hits(A + a0, a1 - a0, smem + b0, len - b0, hits, a0, lane);
    __syncwarp();
    if (a1 >= na || !more) return;
    klo = fwd_ubound(f.first, f.nblocks, A[a1], khi + 1, lane);  // f.first[khi+1] <= A[a1]
    a0 = a1;
  }
}

// Candidate bookkeeping of a warp's run in shared memory: bit 4g + j of
// `alive` (lane-held) stands for position 128g + 32j + lane.

// The alive mask of a run whose first na positions are all candidates.
__device__ __forceinline__ uint32_t alive_prefix(uint32_t na, int lane) {
  uint32_t alive = 0;
  for (uint32_t g = 0; 128u * g < na; g++) {
#pragma unroll
    for (int j = 0; j < 4; j++)
      if (128u * g + 32u * j + (uint32_t)lane < na) alive |= 1u << (4 * g + j);
  }
  return alive;
}

// The alive mask restricted to the positions whose bit is set in `hits`
// (one bit per position, shared memory).
__device__ __forceinline__ uint32_t alive_and_hits(uint32_t alive, uint32_t ng,
                                                   const uint32_t *hits, int lane) {
  for (uint32_t g = 0; g < ng; g++) {
#pragma unroll
    for (int j = 0; j < 4; j++)
      if (!((hits[4 * g + j] >> lane) & 1u)) alive &= ~(1u << (4 * g + j));
  }
  return alive;
}

// Move the alive values of the ng groups of s_r, in order, to its front;
// returns how many there are.
__device__ __forceinline__ uint32_t compact_alive(uint32_t *s_r, uint32_t ng, uint32_t alive,
                                                  int lane) {
  uint32_t count = 0;
  for (uint32_t g = 0; g < ng; g++) {
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const bool a = (alive >> (4 * g + j)) & 1u;
      const uint32_t x = s_r[128u * g + 32 * j + lane];
      const uint32_t m = __ballot_sync(kFull, a);
      __syncwarp();
      if (a) s_r[count + __popc(m & lanemask_lt())] = x;
      count += __popc(m);
      __syncwarp();
    }
  }
  return count;
}

// Ordered output of one tile (all threads of the CTA call it).  Lane holds
// positions 32k + lane of its warp's chunk; chunks are in warp order.
struct TileOut {
  uint32_t *out;
  uint64_t out_cap;
  uint32_t *count;  // written by the last tile
  uint32_t *status;
};

// Output position of warp w's first value in tile t, given each warp's count
// (all threads of the CTA call it; warp 0 does the scan and the look-back).
__device__ __forceinline__ uint64_t tile_base(uint32_t count, uint32_t t, bool last_tile,
                                              const Compaction &cp, const TileOut &to,
                                              uint32_t *s_wcnt, uint32_t *s_base) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) s_wcnt[w] = count;
  __syncthreads();
  if (w == 0) {
    const uint32_t c = lane < kIxWarps ? s_wcnt[lane] : 0u;
    uint32_t inc = c;
#pragma unroll
    for (int d = 1; d < kIxWarps; d <<= 1) {
      const uint32_t y = __shfl_up_sync(kFull, inc, d);
      if (lane >= d) inc += y;
    }
    const uint32_t run = __shfl_sync(kFull, inc, kIxWarps - 1);
    if (lane < kIxWarps) s_wcnt[lane] = inc - c;
    const uint32_t P = lookback_exclusive_warp(cp, t, run, to.status, lane);
    if (lane == 0) {
      s_base[0] = P;
      if (last_tile) {
        *to.count = P + run;
        if ((uint64_t)P + run > to.out_cap) set_status(to.status, BP_ERR_CAPACITY);
      }
    }
  }
  __syncthreads();
  return (uint64_t)s_base[0] + s_wcnt[w];
}

__device__ __forceinline__ void tile_emit(const uint32_t v[4], const bool hit[4], uint32_t t,
                                          bool last_tile, const Compaction &cp, const TileOut &to,
                                          uint32_t *s_wcnt, uint32_t *s_base) {
  uint32_t m[4], tot = 0;
#pragma unroll
  for (int k = 0; k < 4; k++) {
    m[k] = __ballot_sync(kFull, hit[k]);
    tot += __popc(m[k]);
  }
  uint64_t pos = tile_base(tot, t, last_tile, cp, to, s_wcnt, s_base);
#pragma unroll
  for (int k = 0; k < 4; k++) {
    if (hit[k]) {
      const uint64_t idx = pos + __popc(m[k] & lanemask_lt());
      if (idx < to.out_cap) to.out[idx] = v[k];
    }
    pos += __popc(m[k]);
  }
}

// Same for a warp whose `count` outputs are already compacted, in order, in
// its shared buffer `buf`.
__device__ __forceinline__ void tile_emit_buf(const uint32_t *buf, uint32_t count, uint32_t t,
                                              bool last_tile, const Compaction &cp,
                                              const TileOut &to, uint32_t *s_wcnt,
                                              uint32_t *s_base) {
  const uint64_t pos = tile_base(count, t, last_tile, cp, to, s_wcnt, s_base);
  for (uint32_t i = threadIdx.x & 31; i < count; i += 32)
    if (pos + i < to.out_cap) to.out[pos + i] = buf[i];
}

}  // namespace bp
