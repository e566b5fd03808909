// query.cu -- conjunctive queries over an index of GL lists.
//
// bp_query_batch (many queries, fused, one persistent kernel):
//  1. q_plan: per query, order the terms by list length (Set-vs-Set: the
//     shortest list drives, Section 6), and cut the shortest list into work
//     items of `chunk` blocks.
//  2. scan of the item counts.
//  3. q_main: a persistent grid; every warp takes the next item from a device
//     counter, decodes the item's blocks of the shortest list into shared
//     memory, and filters their values through the other lists in order,
//     one list at a time and one block-sized run at a time
//     (gl_membership_win: skip-header search, candidate blocks decoded into
//     a shared-memory window that moves forward with the runs, never to
//     HBM), then appends the survivors to an arena slot.
//  4. q_count / scan / q_gather: per-query counts and the survivors copied in
//     query and item order into the caller's output.
// No kernel waits on another CTA, and every size is fixed by the number of
// queries, so the whole sequence can be captured once in a CUDA graph.
//
// bp_query_one (one query, plain): decode every list of the query to
// scratch, then intersect the decoded arrays two at a time from the
// shortest (the paper's decompress-then-intersect SvS of Section 7.6).
#include <mutex>
#include <vector>

#include "decode.h"
#include "intersect.cuh"
#include "tuning.h"

namespace bp {

namespace {

constexpr int kMaxTerms = 64;
constexpr int kMaxChunk = 8;
// per warp: the item's decoded blocks (survivors are compacted in place),
// the dense window of the list being searched, and in the merge instance one
// hit bit per candidate (kept out of the other instance: 1 KiB more per CTA
// crossed a shared-memory carveout step and cost L1 space, 4 % of queries/s)
constexpr int kWarpSmemBase = kMaxChunk * 128 + kIxDenseMax * 128;
constexpr int warp_smem_words(bool merge) { return kWarpSmemBase + (merge ? kMaxChunk * 4 : 0); }

inline size_t up256(size_t v) { return (v + 255) & ~(size_t)255; }

struct QScratch {
  uint32_t *sorted;    // [total_terms] term ids in SvS order
  uint32_t *base;      // [nq + 1] items per query, scanned in place
  unsigned long long *counters;  // [0] next item, [1] arena top, [2] any bitmap term
  uint32_t *item_q;    // [max_items]
  uint64_t *item_off;  // [max_items] arena offset
  uint32_t *item_cnt;  // [max_items]
  uint32_t *item_pre;  // [max_items] outputs of earlier items of the query
  uint32_t *arena;     // [arena_cap]
};

struct QLayout {
  size_t sorted, base, counters, arena, item_q, item_off, item_cnt, item_pre, total;
  uint64_t max_items;
};

// Fixed regions first; the four per-item arrays share what is left.
QLayout q_layout(uint64_t total_terms, uint32_t nq, uint64_t arena_cap, uint64_t max_items) {
  QLayout L;
  L.sorted = 0;
  L.base = up256(4 * total_terms);
  L.counters = up256(L.base + 4 * ((size_t)nq + 1));
  L.arena = L.counters + 256;
  L.item_q = up256(L.arena + 4 * arena_cap);
  L.max_items = max_items;
  L.item_off = up256(L.item_q + 4 * max_items);
  L.item_cnt = up256(L.item_off + 8 * max_items);
  L.item_pre = up256(L.item_cnt + 4 * max_items);
  L.total = up256(L.item_pre + 4 * max_items);
  return L;
}

// Largest item capacity that fits in scratch_bytes.
QLayout q_layout_fit(uint64_t total_terms, uint32_t nq, uint64_t arena_cap, size_t scratch_bytes) {
  QLayout L = q_layout(total_terms, nq, arena_cap, 0);
  const size_t fixed = L.total + 4 * 256;
  L = q_layout(total_terms, nq, arena_cap, scratch_bytes > fixed ? (scratch_bytes - fixed) / 20 : 0);
  return L;
}

QScratch q_carve(void *p, const QLayout &L) {
  uint8_t *b = static_cast<uint8_t *>(p);
  QScratch s;
  s.sorted = reinterpret_cast<uint32_t *>(b + L.sorted);
  s.base = reinterpret_cast<uint32_t *>(b + L.base);
  s.counters = reinterpret_cast<unsigned long long *>(b + L.counters);
  s.item_q = reinterpret_cast<uint32_t *>(b + L.item_q);
  s.item_off = reinterpret_cast<uint64_t *>(b + L.item_off);
  s.item_cnt = reinterpret_cast<uint32_t *>(b + L.item_cnt);
  s.item_pre = reinterpret_cast<uint32_t *>(b + L.item_pre);
  s.arena = reinterpret_cast<uint32_t *>(b + L.arena);
  return s;
}

// ---- 1. planning ---------------------------------------------------------------------

// Set-vs-Set order of a query's terms: compressed lists by length, then the
// bitmaps of a hybrid index (hyb+m2: the compressed lists are intersected
// first and the survivors tested against the bitmaps).
__host__ __device__ inline uint64_t svs_key(const bp_list &L) {
  return ((uint64_t)(L.layout == BP_LAYOUT_BITMAP) << 32) | L.n;
}

// Words of the bitmaps that one work item ANDs (32 per lane).
constexpr uint32_t kBitmapItemWords = 1024;

// Work items of a query driven by list L: `chunk` blocks of a GL list each,
// or kBitmapItemWords words (32,768 docIDs) of a bitmap.
__host__ __device__ inline uint64_t driver_items(const bp_list &L, uint32_t chunk) {
  if (L.layout == BP_LAYOUT_BITMAP) {
    const uint64_t words = L.enc_bytes >= 16 ? (L.enc_bytes - 16) / 4 : 0;
    return (words + kBitmapItemWords - 1) / kBitmapItemWords;
  }
  return ((L.n + 127ull) / 128 + chunk - 1) / chunk;
}

__global__ void q_plan_kernel(const bp_list *__restrict__ lists, uint32_t n_terms,
                              const uint32_t *__restrict__ terms, const uint64_t *__restrict__ toff,
                              uint32_t nq, QScratch sc, uint32_t chunk, uint32_t *status) {
  const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nq) return;
  const uint64_t b = toff[q], e = toff[q + 1];
  const uint32_t k = (uint32_t)(e - b);
  uint32_t items = 0;
  bool any_bitmap = false;
  if (e < b || k > (uint32_t)kMaxTerms) {
    set_status(status, BP_ERR_ARG);
  } else if (k > 0) {
    bool ok = true;
    for (uint32_t i = 0; i < k; i++) {  // insertion sort by (n, id)
      const uint32_t t = terms[b + i];
      if (t >= n_terms) {
        ok = false;
        break;
      }
      const uint64_t nt = svs_key(lists[t]);
      if (nt >> 32) any_bitmap = true;
      uint32_t p = i;
      while (p > 0) {
        const uint32_t u = sc.sorted[b + p - 1];
        const uint64_t nu = svs_key(lists[u]);
        if (nu < nt || (nu == nt && u <= t)) break;
        sc.sorted[b + p] = u;
        p--;
      }
      sc.sorted[b + p] = t;
    }
    if (!ok) {
      set_status(status, BP_ERR_ARG);
    } else {
      items = (uint32_t)driver_items(lists[sc.sorted[b]], chunk);
    }
  }
  sc.base[q] = items;
  if (any_bitmap && sc.counters[2] == 0ull) sc.counters[2] = 1ull;
}

// Exclusive scan of a[0..n) in place by one CTA of 1024 threads; a[n] =
// total, saturated at 2^32 - 1 (more work items than any scratch holds: the
// kernels that read a[n] then stop with BP_ERR_SCRATCH).
__global__ void __launch_bounds__(1024) scan_u32_kernel(uint32_t *a, uint32_t n) {
  __shared__ uint64_t s_w[32];
  __shared__ uint64_t s_carry;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  for (uint32_t base = 0; base < n; base += 1024) {
    const uint32_t i = base + threadIdx.x;
    const uint32_t x = i < n ? a[i] : 0u;
    uint64_t incl = x;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint64_t t = __shfl_up_sync(kFull, incl, d);
      if (lane >= d) incl += t;
    }
    if (lane == 31) s_w[w] = incl;
    __syncthreads();
    if (w == 0) {
      uint64_t v = s_w[lane], vi = v;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint64_t t = __shfl_up_sync(kFull, vi, d);
        if (lane >= d) vi += t;
      }
      s_w[lane] = vi - v;
    }
    __syncthreads();
    const uint64_t carry = s_carry;
    if (i < n) a[i] = (uint32_t)(carry + s_w[w] + incl - x);
    __syncthreads();
    if (threadIdx.x == 1023) s_carry = carry + s_w[w] + incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) a[n] = s_carry > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)s_carry;
}

// ---- 3. the persistent fused kernel --------------------------------------------------------

// A term's list as the kernel sees it: a GL stream, or a bitmap (then
// gl.payload holds its words and gl.pw their count; no other field is set).
struct TermView {
  bool bitmap;
  GlView gl;
};

// 0, or the status of a term whose list cannot be used: BP_ERR_CORRUPT, or
// BP_ERR_ARG for a GL list that is not D4 (the probes need D4 columns).
template <bool HYB>
__device__ __forceinline__ uint32_t term_view(const uint8_t *data, const bp_list *lists,
                                              uint32_t t, TermView &v) {
  const bp_list L = lists[t];
  v.bitmap = HYB && L.layout == BP_LAYOUT_BITMAP;
  if (v.bitmap) {
    const uint8_t *enc = data + L.enc_offset;
    if (L.enc_bytes < 16 || (L.enc_offset & 15u)) return BP_ERR_CORRUPT;
    const uint4 h = __ldg(reinterpret_cast<const uint4 *>(enc));
    if (h.x != bp_fmt::kBitmapMagic || h.y != (uint32_t)BP_LAYOUT_BITMAP || h.z != L.n ||
        16ull + 4ull * h.w > L.enc_bytes)
      return BP_ERR_CORRUPT;
    v.gl.payload = reinterpret_cast<const uint32_t *>(enc + 16);
    v.gl.pw = h.w;
    return 0u;
  }
  if (!gl_view(data + L.enc_offset, L.enc_bytes, v.gl) || v.gl.n != L.n) return BP_ERR_CORRUPT;
  return v.gl.kind == 0u ? 0u : (uint32_t)BP_ERR_ARG;
}

// Clears the bits of `alive` whose candidates (value 128g + 32j + lane of
// s_r for bit 4g+j) are not set in the bitmap: one load per candidate.
__device__ __forceinline__ uint32_t bitmap_filter(const uint32_t *__restrict__ bm,
                                                  uint32_t words, const uint32_t *s_r, uint32_t ng,
                                                  uint32_t alive, int lane) {
  for (uint32_t g = 0; g < ng; g++)
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const uint32_t bit = 1u << (4 * g + j);
      const uint32_t x = s_r[128u * g + 32 * j + lane];
      if ((alive & bit) && !((x >> 5) < words && ((__ldg(bm + (x >> 5)) >> (x & 31u)) & 1u)))
        alive &= ~bit;
    }
  return alive;
}

// One work item of a query whose terms are all bitmaps (only the hybrid
// instance of q_main_kernel contains it).
__device__ __forceinline__ void bitmap_and_item(const uint8_t *__restrict__ data,
                                                const bp_list *__restrict__ lists,
                                                const TermView &V1, const uint32_t *sorted,
                                                uint32_t k, uint32_t c, uint32_t q, uint32_t item,
                                                QScratch sc, uint64_t arena_cap, uint32_t *s_r,
                                                int lane, uint32_t *status) {
  // Bitmaps sort last, so every term is a bitmap: AND kBitmapItemWords
  // words of all of them (lane l keeps words 32i + l in s_r), then write
  // the set bits of the result straight to the arena
  const uint32_t w0 = kBitmapItemWords * c;
  uint32_t any = 0;
#pragma unroll 8
  for (uint32_t i = 0; i < 32; i++) {
    const uint32_t wi = w0 + 32u * i + lane;
    const uint32_t x = wi < V1.gl.pw ? __ldg(V1.gl.payload + wi) : 0u;
    s_r[32u * i + lane] = x;
    any |= x;
  }
  for (uint32_t t = 1; t < k && __any_sync(kFull, any != 0u); t++) {
    TermView F;
    uint32_t tf = term_view<true>(data, lists, sorted[t], F);
    if (tf == 0u && !F.bitmap) tf = BP_ERR_CORRUPT;  // cannot follow a bitmap
    if (tf != 0u) {
      if (lane == 0) set_status(status, tf);
      any = 0;
      break;
    }
    any = 0;
#pragma unroll 8
    for (uint32_t i = 0; i < 32; i++) {
      const uint32_t wi = w0 + 32u * i + lane;
      const uint32_t x = s_r[32u * i + lane] & (wi < F.gl.pw ? __ldg(F.gl.payload + wi) : 0u);
      s_r[32u * i + lane] = x;
      any |= x;
    }
  }
  uint32_t n = 0;
  if (any)
    for (uint32_t i = 0; i < 32; i++) n += __popc(s_r[32u * i + lane]);
  const uint32_t tot = __reduce_add_sync(kFull, n);
  uint64_t off = 0;
  if (lane == 0 && tot) off = atomicAdd(sc.counters + 1, (unsigned long long)tot);
  off = __shfl_sync(kFull, off, 0);
  const bool fits = off + tot <= arena_cap;
  if (!fits && lane == 0) set_status(status, BP_ERR_CAPACITY);
  if (fits && tot) {
    uint32_t run = 0;
    for (uint32_t i = 0; i < 32; i++) {
      uint32_t x = s_r[32u * i + lane];
      const uint32_t p = __popc(x);
      uint32_t inc = p;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, inc, d);
        if (lane >= d) inc += y;
      }
      uint64_t pos = off + run + inc - p;
      const uint32_t base = 32u * (w0 + 32u * i + lane);
      while (x) {
        sc.arena[pos++] = base + (uint32_t)(__ffs(x) - 1);
        x &= x - 1;
      }
      run += __shfl_sync(kFull, inc, 31);
    }
  }
  if (lane == 0) {
    sc.item_q[item] = q;
    sc.item_off[item] = fits ? off : ~0ull;
    sc.item_cnt[item] = tot;
  }
  __syncwarp();
}

// At most 80 registers: 3 CTAs of 8 warps (or 6 of 4) per SM; more warps
// in flight matter more here than the few values it would keep in registers.
// Two instances: HYB = false for batches of compressed lists only, HYB =
// true for batches with bitmap terms (hybrid index); the plan kernel records
// which, and the other instance leaves at once.  The bitmap code would cost
// the all-compressed kernel registers (measured: about 4 % of its speed).
// MERGE: the instance with the merge regime for a query's first list, run
// when the tuning's merge_span is not 0; its call costs the kernel about
// 7 % where it is not taken (measured), so it is not compiled in otherwise.
template <bool HYB, bool MERGE>
__global__ void __launch_bounds__(256, 3)
    q_main_kernel(const uint8_t *__restrict__ data, const bp_list *__restrict__ lists,
                              const uint64_t *__restrict__ toff, uint32_t nq, QScratch sc,
                              uint32_t max_items, uint64_t arena_cap, uint32_t chunk,
                              uint32_t dense_max, uint32_t merge_span, uint32_t *status) {
  if ((sc.counters[2] != 0ull) != HYB) return;
  extern __shared__ uint32_t smem[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t *s_r = smem + w * warp_smem_words(MERGE);
  uint32_t *s_f = s_r + kMaxChunk * 128;
  uint32_t *s_hit = s_f + kIxDenseMax * 128;  // MERGE only
  const uint32_t total = sc.base[nq];
  if (total > max_items) {  // the caller's scratch holds fewer work items
    if (threadIdx.x == 0 && blockIdx.x == 0) set_status(status, BP_ERR_SCRATCH);
    return;
  }
  for (;;) {
    uint32_t item = 0;
    if (lane == 0) item = (uint32_t)atomicAdd(sc.counters, 1ull);
    item = __shfl_sync(kFull, item, 0);
    if (item >= total) break;
    const int64_t qq = warp_ubound(sc.base, (uint64_t)nq + 1, item, lane);
    const uint32_t q = (uint32_t)qq;
    const uint32_t c = item - sc.base[q];
    const uint64_t tb = toff[q];
    const uint32_t k = (uint32_t)(toff[q + 1] - tb);
    TermView V1;
    uint32_t scount = 0;
    const uint32_t tv = term_view<HYB>(data, lists, sc.sorted[tb], V1);
    if (HYB && tv == 0u && V1.bitmap) {
      bitmap_and_item(data, lists, V1, sc.sorted + tb, k, c, q, item, sc, arena_cap, s_r, lane,
                      status);
      continue;
    }
    if (tv == 0u) {
      // the item's candidates, ascending, in s_r: `chunk` blocks of the
      // shortest compressed list; bit 4g+j of `alive`: value 128g + 32j +
      // lane is still a candidate
      uint32_t alive = 0, na = 0;
      const uint32_t b0 = c * chunk, b1 = min(V1.gl.nblocks, b0 + chunk);
      const uint32_t ng = b1 > b0 ? b1 - b0 : 0u;
      for (uint32_t g = 0; g < ng; g++) {
        const uint32_t cnt = gl_block_into(V1.gl, b0 + g, s_r + 128u * g, lane, status);
        na = 128u * g + cnt;
#pragma unroll
        for (int j = 0; j < 4; j++)
          if ((uint32_t)(32 * j + lane) < cnt) alive |= 1u << (4 * g + j);
      }
      __syncwarp();
      // Set-vs-Set: the candidates go through the other lists in order, each
      // list searched run by run with its dense window moving forward
      for (uint32_t t = 1; t < k && __any_sync(kFull, alive != 0u); t++) {
        TermView F;
        const uint32_t tf = term_view<HYB>(data, lists, sc.sorted[tb + t], F);
        if (tf != 0u) {
          if (lane == 0) set_status(status, tf);
          alive = 0;
          break;
        }
        if (HYB && F.bitmap) {
          alive = bitmap_filter(F.gl.payload, F.gl.pw, s_r, ng, alive, lane);
          continue;
        }
        if (MERGE && t == 1 && F.gl.nblocks > 0u && na > 0u) {
          // merge regime for the first list, while the candidates are the
          // whole decoded run s_r[0..na)
          const int64_t kl = warp_ubound(F.gl.first, F.gl.nblocks, s_r[na - 1], lane);
          if (kl < 0) {  // every candidate is below the list's first value
            alive = 0;
            continue;
          }
          const int64_t kf = warp_ubound(F.gl.first, F.gl.nblocks, s_r[0], lane);
          if ((uint64_t)(kl - imax64(kf, 0) + 1) <= (uint64_t)merge_span * ng) {
            s_hit[lane] = 0u;
            __syncwarp();
            merge_run_hits(F.gl, s_r, na, kf, kl, s_f, s_hit, lane, status);
            alive = alive_and_hits(alive, ng, s_hit, lane);
            __syncwarp();
            continue;
          }
        }
        FWin win = fwin_empty();
        for (uint32_t g = 0; g < ng; g++) {
          uint32_t v[4];
          bool valid[4], hit[4];
          uint32_t lo = 0xFFFFFFFFu, hi = 0u;
#pragma unroll
          for (int j = 0; j < 4; j++) {
            valid[j] = (alive >> (4 * g + j)) & 1u;
            v[j] = s_r[128u * g + 32 * j + lane];
            if (valid[j]) {
              lo = min(lo, v[j]);
              hi = max(hi, v[j]);
            }
          }
          if (!__any_sync(kFull, (alive >> (4 * g)) & 0xFu)) continue;
          lo = __reduce_min_sync(kFull, lo);
          hi = __reduce_max_sync(kFull, hi);
          gl_membership_win(F.gl, v, valid, hit, lo, hi, s_f, win, lane, dense_max, status);
#pragma unroll
          for (int j = 0; j < 4; j++)
            if (valid[j] && !hit[j]) alive &= ~(1u << (4 * g + j));
        }
      }
      // compact the survivors, in order, to the front of s_r
      for (uint32_t g = 0; g < ng; g++) {
#pragma unroll
        for (int j = 0; j < 4; j++) {
          const bool a = (alive >> (4 * g + j)) & 1u;
          const uint32_t x = s_r[128u * g + 32 * j + lane];
          const uint32_t m = __ballot_sync(kFull, a);
          __syncwarp();
          if (a) s_r[scount + __popc(m & lanemask_lt())] = x;
          scount += __popc(m);
          __syncwarp();
        }
      }
    } else if (lane == 0) {
      set_status(status, tv);
    }
    __syncwarp();
    uint64_t off = 0;
    if (lane == 0 && scount) off = atomicAdd(sc.counters + 1, (unsigned long long)scount);
    off = __shfl_sync(kFull, off, 0);
    const bool fits = off + scount <= arena_cap;
    if (!fits && lane == 0) set_status(status, BP_ERR_CAPACITY);
    if (fits)
      for (uint32_t i = lane; i < scount; i += 32) sc.arena[off + i] = s_r[i];
    if (lane == 0) {
      sc.item_q[item] = q;
      sc.item_off[item] = fits ? off : ~0ull;
      sc.item_cnt[item] = scount;
    }
    __syncwarp();
  }
}

// ---- 4. counts, output offsets and gather ------------------------------------------------------

__global__ void q_count_kernel(uint32_t nq, QScratch sc, uint32_t max_items, uint32_t *counts) {
  const int lane = threadIdx.x & 31;
  const bool fits = sc.base[nq] <= max_items;
  const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t q = warp; q < nq; q += nwarps) {
    const uint32_t b = sc.base[q], e = sc.base[q + 1];
    uint32_t run = 0;
    for (uint32_t i0 = b; i0 < e; i0 += 32) {
      const uint32_t i = i0 + lane;
      const uint32_t x = (fits && i < e) ? sc.item_cnt[i] : 0u;
      uint32_t incl = x;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t t = __shfl_up_sync(kFull, incl, d);
        if (lane >= d) incl += t;
      }
      if (fits && i < e) sc.item_pre[i] = run + incl - x;
      run += __shfl_sync(kFull, incl, 31);
    }
    if (lane == 0) counts[q] = run;
  }
}

__global__ void __launch_bounds__(1024) scan_counts_kernel(const uint32_t *counts, uint32_t n,
                                                           uint64_t *out_off, uint64_t out_cap,
                                                           uint32_t *status) {
  __shared__ uint64_t s_w[32];
  __shared__ uint64_t s_carry;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  for (uint32_t base = 0; base < n; base += 1024) {
    const uint32_t i = base + threadIdx.x;
    const uint64_t x = i < n ? counts[i] : 0u;
    uint64_t incl = x;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint64_t t = __shfl_up_sync(kFull, incl, d);
      if (lane >= d) incl += t;
    }
    if (lane == 31) s_w[w] = incl;
    __syncthreads();
    if (w == 0) {
      uint64_t v = s_w[lane], vi = v;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint64_t t = __shfl_up_sync(kFull, vi, d);
        if (lane >= d) vi += t;
      }
      s_w[lane] = vi - v;
    }
    __syncthreads();
    const uint64_t carry = s_carry;
    if (i < n) out_off[i] = carry + s_w[w] + incl - x;
    __syncthreads();
    if (threadIdx.x == 1023) s_carry = carry + s_w[w] + incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out_off[n] = s_carry;
    if (s_carry > out_cap) set_status(status, BP_ERR_CAPACITY);
  }
}

__global__ void q_gather_kernel(QScratch sc, uint32_t nq, uint32_t max_items,
                                const uint64_t *__restrict__ out_off, uint32_t *__restrict__ out,
                                uint64_t out_cap) {
  const int lane = threadIdx.x & 31;
  const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  const uint32_t total = sc.base[nq];
  if (total > max_items) return;
  for (uint64_t item = warp; item < total; item += nwarps) {
    const uint32_t cnt = sc.item_cnt[item];
    const uint64_t off = sc.item_off[item];
    if (cnt == 0 || off == ~0ull) continue;
    const uint64_t dst = out_off[sc.item_q[item]] + sc.item_pre[item];
    for (uint32_t i = lane; i < cnt; i += 32)
      if (dst + i < out_cap) out[dst + i] = sc.arena[off + i];
  }
}

__global__ void set_u32_kernel(uint32_t *p, uint32_t v) { *p = v; }

// Devices (bit d: device d) on which q_main_kernel's shared-memory limit
// was raised.
std::mutex g_main_mu;
uint64_t g_main_smem_set = 0;

}  // namespace

// ---- host side -----------------------------------------------------------------------------------

uint64_t query_items_of(const bp_list &driver) {
  const uint32_t chunk = std::max<uint32_t>(1, std::min<uint32_t>(tuning().query_chunk_blocks,
                                                                 kMaxChunk));
  return driver_items(driver, chunk);
}

size_t query_batch_scratch_for(uint64_t total_terms, uint32_t nq, uint64_t out_cap,
                               uint64_t items) {
  return q_layout(total_terms, nq, out_cap, items).total + 4 * 256;
}

size_t query_batch_scratch_bytes(const bp_list *h_lists, uint32_t n_terms, const uint32_t *h_terms,
                                 const uint64_t *h_term_off, uint32_t nq, uint64_t out_cap) {
  const uint32_t chunk = std::max<uint32_t>(1, std::min<uint32_t>(tuning().query_chunk_blocks,
                                                                 kMaxChunk));
  uint64_t items = 0;
  for (uint32_t q = 0; q < nq; q++) {
    uint64_t kmin = UINT64_MAX;
    const bp_list *drv = nullptr;
    for (uint64_t i = h_term_off[q]; i < h_term_off[q + 1]; i++)
      if (h_terms[i] < n_terms && svs_key(h_lists[h_terms[i]]) < kmin) {
        kmin = svs_key(h_lists[h_terms[i]]);
        drv = &h_lists[h_terms[i]];
      }
    if (!drv) continue;
    items += driver_items(*drv, chunk);
  }
  return q_layout(h_term_off[nq], nq, out_cap, items).total + 4 * 256;
}

int launch_query_batch(const uint8_t *data, const bp_list *lists, uint32_t n_terms,
                       const uint32_t *terms, const uint64_t *term_off, uint64_t total_terms,
                       uint32_t nq, uint32_t *out, uint64_t out_cap,
                       uint64_t *out_off, uint32_t *counts, void *scratch, size_t scratch_bytes,
                       uint32_t *status, cudaStream_t s) {
  const Tuning tu = tuning();
  const uint32_t chunk = std::max<uint32_t>(1, std::min<uint32_t>(tu.query_chunk_blocks, kMaxChunk));
  const uint32_t warps = tu.query_warps == 4 ? 4 : 8;
  const uint64_t arena_cap = out_cap;
  const QLayout L = q_layout_fit(total_terms, nq, arena_cap, scratch_bytes);
  if (scratch_bytes < L.total) return BP_ERR_SCRATCH;
  const uint32_t max_items = (uint32_t)std::min<uint64_t>(L.max_items, 0xFFFFFFF0ull);
  const QScratch sc = q_carve(scratch, L);
  if (cudaMemsetAsync(sc.counters, 0, 256, s) != cudaSuccess) return BP_ERR_CUDA;
  if (nq == 0) return BP_OK;
  const int threads = 32 * (int)warps;
  const bool mrg = tu.merge_span != 0u;
  const size_t smem = sizeof(uint32_t) * warp_smem_words(mrg) * warps;
  {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return BP_ERR_CUDA;
    std::lock_guard<std::mutex> g(g_main_mu);
    if (!((g_main_smem_set >> dev) & 1u)) {
      const int plain = (int)(sizeof(uint32_t) * warp_smem_words(false) * 8);
      const int merge = (int)(sizeof(uint32_t) * warp_smem_words(true) * 8);
      if (cudaFuncSetAttribute(q_main_kernel<false, false>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, plain) != cudaSuccess ||
          cudaFuncSetAttribute(q_main_kernel<true, false>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, plain) != cudaSuccess ||
          cudaFuncSetAttribute(q_main_kernel<false, true>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, merge) != cudaSuccess ||
          cudaFuncSetAttribute(q_main_kernel<true, true>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, merge) != cudaSuccess)
        return BP_ERR_CUDA;
      g_main_smem_set |= 1ull << dev;
    }
  }
  // the instances for this tuning: compressed-only and hybrid, with or
  // without the merge regime
  auto *const kc = mrg ? q_main_kernel<false, true> : q_main_kernel<false, false>;
  auto *const kh = mrg ? q_main_kernel<true, true> : q_main_kernel<true, false>;
  int per_sm = 0, per_sm_h = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kc, threads, smem) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_h, kh, threads, smem) != cudaSuccess ||
      per_sm_h < 1)
    per_sm_h = 1;
  const int grid = per_sm * device_sm_count(), grid_h = per_sm_h * device_sm_count();
  q_plan_kernel<<<(nq + 255) / 256, 256, 0, s>>>(lists, n_terms, terms, term_off, nq, sc, chunk,
                                                  status);
  scan_u32_kernel<<<1, 1024, 0, s>>>(sc.base, nq);
  const uint32_t dense = std::min<uint32_t>(tu.dense_blocks, kIxDenseMax);
  kc<<<grid, threads, smem, s>>>(data, lists, term_off, nq, sc, max_items, arena_cap, chunk, dense,
                                 tu.merge_span, status);
  kh<<<grid_h, threads, smem, s>>>(data, lists, term_off, nq, sc, max_items, arena_cap, chunk,
                                   dense, tu.merge_span, status);
  const int cgrid = (int)std::min<uint64_t>((nq + 7) / 8, 65535);
  q_count_kernel<<<cgrid, 256, 0, s>>>(nq, sc, max_items, counts);
  scan_counts_kernel<<<1, 1024, 0, s>>>(counts, nq, out_off, out_cap, status);
  q_gather_kernel<<<device_sm_count() * 8, 256, 0, s>>>(sc, nq, max_items, out_off, out, out_cap);
  return cudaPeekAtLastError() == cudaSuccess ? BP_OK : BP_ERR_CUDA;
}

// ---- the plain per-query path ------------------------------------------------------------------

namespace {

__global__ void __launch_bounds__(kIxThreads)
    sorted_pair_dev_kernel(const uint32_t *__restrict__ r, const uint32_t *nr_dev, uint32_t nr_host,
                           const uint32_t *__restrict__ f, const uint32_t *nf_dev, uint32_t nf_host,
                           Compaction cp, TileOut to, uint32_t ntiles, uint32_t dense_max) {
  __shared__ uint32_t s_f[kIxWarps][kIxDenseMax * 128];
  __shared__ uint32_t s_wcnt[kIxWarps], s_base[1], s_tile;
  if (threadIdx.x == 0) s_tile = atomicAdd(cp.ticket, 1u);
  __syncthreads();
  const uint32_t t = s_tile;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint32_t nr = nr_dev ? min(*nr_dev, nr_host) : nr_host;
  const uint32_t nf = nf_dev ? min(*nf_dev, nf_host) : nf_host;
  uint32_t v[4] = {0, 0, 0, 0};
  bool valid[4] = {false, false, false, false}, hit[4] = {false, false, false, false};
  const uint64_t base = (uint64_t)(t * kIxWarps + w) * 128u;
  if (base < nr) {
    const uint32_t cnt = (nr - base) < 128u ? (uint32_t)(nr - base) : 128u;
#pragma unroll
    for (int k = 0; k < 4; k++) {
      valid[k] = (uint32_t)(32 * k + lane) < cnt;
      v[k] = valid[k] ? __ldg(r + base + 32 * k + lane) : 0u;
    }
    raw_membership(f, nf, v, valid, hit, __ldg(r + base), __ldg(r + base + cnt - 1), s_f[w],
                   lane, dense_max);
  }
  tile_emit(v, hit, t, t == ntiles - 1, cp, to, s_wcnt, s_base);
}

}  // namespace

size_t query_one_scratch_bytes(const bp_list *h_lists, const uint32_t *h_terms, uint32_t k) {
  uint64_t sum = 0, nmin = UINT64_MAX;
  for (uint32_t i = 0; i < k; i++) {
    sum += up256(4ull * h_lists[h_terms[i]].n + 16);
    nmin = std::min<uint64_t>(nmin, h_lists[h_terms[i]].n);
  }
  if (k == 0) nmin = 0;
  const uint64_t tiles = std::max<uint64_t>(1, ((nmin + 127) / 128 + kIxWarps - 1) / kIxWarps);
  return up256(compaction_bytes(tiles)) + sum + 2 * up256(4 * nmin + 16) + 256;
}

int launch_query_one(const uint8_t *data, const bp_list *h_lists, const uint32_t *h_terms,
                     uint32_t k, uint32_t *out, uint64_t out_cap, uint32_t *count, void *scratch,
                     size_t scratch_bytes, uint32_t *status, cudaStream_t s) {
  if (scratch_bytes < query_one_scratch_bytes(h_lists, h_terms, k)) return BP_ERR_SCRATCH;
  for (uint32_t i = 0; i < k; i++)  // the plain path decodes GL lists only
    if (h_lists[h_terms[i]].layout != BP_LAYOUT_GPU) return BP_ERR_ARG;
  if (k == 0) {
    set_u32_kernel<<<1, 1, 0, s>>>(count, 0u);
    return cudaPeekAtLastError() == cudaSuccess ? BP_OK : BP_ERR_CUDA;
  }
  std::vector<uint32_t> ord(h_terms, h_terms + k);
  std::stable_sort(ord.begin(), ord.end(),
                   [&](uint32_t a, uint32_t b) { return h_lists[a].n < h_lists[b].n; });
  const uint32_t n1 = h_lists[ord[0]].n;
  const uint64_t tiles = std::max<uint64_t>(1, ((n1 + 127ull) / 128 + kIxWarps - 1) / kIxWarps);
  uint8_t *p = static_cast<uint8_t *>(scratch);
  const Compaction cp = compaction_at(p);
  p += up256(compaction_bytes(tiles));
  uint32_t *cnt_dev = reinterpret_cast<uint32_t *>(p);  // two running counts
  p += 256;
  std::vector<uint32_t *> dec(k);
  int rc;
  for (uint32_t i = 0; i < k; i++) {  // decompress every list of the query
    const bp_list L = h_lists[ord[i]];
    dec[i] = reinterpret_cast<uint32_t *>(p);
    p += up256(4ull * L.n + 16);
    rc = launch_gl_decode(data + L.enc_offset, single_list(L.enc_bytes, L.n, BP_LAYOUT_GPU),
                          bp_fmt::units_of(L.n, BP_LAYOUT_GPU), dec[i], L.n, nullptr, status, s);
    if (rc != BP_OK) return rc;
  }
  if (k == 1) {
    if (out_cap < n1) return BP_ERR_CAPACITY;
    if (cudaMemcpyAsync(out, dec[0], 4ull * n1, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return BP_ERR_CUDA;
    set_u32_kernel<<<1, 1, 0, s>>>(count, n1);
    return cudaPeekAtLastError() == cudaSuccess ? BP_OK : BP_ERR_CUDA;
  }
  uint32_t *buf[2] = {reinterpret_cast<uint32_t *>(p), nullptr};
  p += up256(4ull * n1 + 16);
  buf[1] = reinterpret_cast<uint32_t *>(p);
  const uint32_t dense = std::min<uint32_t>(tuning().dense_blocks, kIxDenseMax);
  const uint32_t *cur = dec[0];
  const uint32_t *cur_n = nullptr;  // device length of cur (null: n1)
  for (uint32_t i = 1; i < k; i++) {
    const bool last = i == k - 1;
    uint32_t *dst = last ? out : buf[i & 1];
    uint32_t *dst_n = last ? count : cnt_dev + (i & 1);
    if (cudaMemsetAsync(cp.ticket, 0, compaction_bytes(tiles), s) != cudaSuccess)
      return BP_ERR_CUDA;
    TileOut to{dst, last ? out_cap : n1, dst_n, status};
    sorted_pair_dev_kernel<<<(unsigned)tiles, kIxThreads, 0, s>>>(
        cur, cur_n, n1, dec[i], nullptr, h_lists[ord[i]].n, cp, to, (uint32_t)tiles, dense);
    cur = dst;
    cur_n = dst_n;
  }
  return cudaPeekAtLastError() == cudaSuccess ? BP_OK : BP_ERR_CUDA;
}

}  // namespace bp
