// decode_pl.cu -- decoding of the paper's S4-BP128-D4 layout (PL).
//
// In this layout only the blocks before a block say where it is: meta-block
// m+1 starts where meta-block m ends (16 width bytes, then 16 blocks of 16b
// bytes, Section 4.3), and the D4 seed of a block is the sum of the column
// deltas of every earlier block of its list (Section 5).  Both sequential
// dependencies are resolved by parallel passes over all lists of a call:
//
//  parse   A stream is read as 16-byte lines, and meta-blocks start on line
//          boundaries.  Every line is a candidate start: its successor is
//          line + 1 + (sum of its 16 bytes), or none (a dead line) if a byte
//          exceeds 32 or the meta-block would run past the stream.  pl_parse
//          takes segments of kSeg lines; pointer jumping over the live lines
//          of a segment gives, for each of the kEnt lines where the true
//          chain can enter it (a meta-block spans at most 513 lines), where
//          the chain leaves and how many meta-blocks it passed, and a group
//          of kGrp segments composes these maps.  pl_resolve follows the
//          group maps of each list from line 1; pl_emit walks every segment
//          from its entry and records the byte offset and width of each block.
//  rest    pl_leftover reads the fewer than 16 blocks after the meta-blocks
//          (one width byte each) and checks the stream's size.
//  decode  pl_tiles takes tiles of kTileChunks chunks of kChunk work units
//          in ticket order, one chunk per warp.  A warp stages its chunk's
//          blocks in shared memory with one bulk copy (a chunk too wide for
//          the stage is pulled into L2 instead and read from global memory)
//          and sums their columns (one lane per block); the CTA publishes
//          the tile's column sums, restarting at every list head.  The
//          seed of a tile -- the column
//          sums of its first list's earlier blocks (Section 5) -- comes from
//          a decoupled look-back over the tiles before it, and the warps
//          then unpack the staged blocks again (Algorithm 1, 4-lane
//          interleave) and store them with the seed added.  So the
//          compressed stream is read from memory once here (and once by
//          parse).  pl_tail decodes the varint tail (Section 4.1) from the
//          last packed value.
//
// Work unit u of a list: its block u - unit_base, then one unit for the tail.
#include <type_traits>

#include "decode.h"
#include "bulk.cuh"
#include "gl_block.cuh"
#include "pl_block.cuh"
#include "tuning.h"

namespace bp {

namespace {

constexpr int kThreads = 256;
constexpr uint32_t kSeg = 4096;     // lines per parse segment
constexpr uint32_t kEnt = 513;      // lines where a chain can enter a segment
constexpr uint32_t kGrp = 8;        // segments per group
constexpr uint32_t kLiveCap = 256;  // live lines kept per segment for pl_emit
constexpr uint32_t kMapChunk = 16;  // group maps staged at a time by pl_resolve
constexpr uint32_t kChunk = 32;          // work units per warp and tile step
constexpr int kTileChunks = 7;           // chunk warps per CTA of pl_tiles (+ a control warp)
constexpr int kTileThreads = 32 * (kTileChunks + 1);
constexpr int kTileMinBlocks = 4;        // resident CTAs per SM for pl_tiles
constexpr uint32_t kStageBytes = 3776;   // per warp and buffer: 32 blocks of average width <= 7.3
constexpr uint32_t kStageWide = 5120;    // the same for wide lists (average width <= 9.9), 3 CTAs per SM
constexpr uint64_t kOffMask = (1ull << 56) - 1;
constexpr uint64_t kBadEntry = ~0ull;  // width byte 0xFF: no block to decode
constexpr uint32_t kNone = 0xFFFFFFFFu;
constexpr uint32_t kDead = 0xFFFFu;  // chain state: the chain stopped earlier

// A chain state is packed as (entry line offset | meta-blocks passed << 16);
// a line's jump as (target line - segment start | meta-blocks passed << 16).
__device__ __forceinline__ uint32_t lo16(uint32_t v) { return v & 0xFFFFu; }

size_t a256(size_t v) { return (v + 255) & ~(size_t)255; }

// Lists with at least one meta-block have at least 17 work units.
uint64_t max_long_lists(uint64_t units, uint32_t count) {
  const uint64_t m = units / 17;
  return m < count ? m : count;
}
// A list of nb blocks has at most 32.07 nb + 42 lines, so fewer than
// nb / 127 + 1.02 segments.
uint64_t max_segs(uint64_t units, uint32_t count) {
  return units / 127 + 2 * max_long_lists(units, count) + 1;
}
uint64_t max_groups(uint64_t units, uint32_t count) {
  return max_segs(units, count) / kGrp + max_long_lists(units, count) + 1;
}

struct PlScratch {
  uint64_t *boffw;      // [units] byte offset | width << 56; tail unit: tail offset
  uint32_t *seg_base;   // [count + 1] first segment of each list; [count]: total
  uint32_t *grp_base;   // [count + 1] first group of each list; [count]: total
  uint32_t *ctl;        // [0] nonzero: the lists do not tile the units, do nothing;
                        // [1] nonzero: some list is not D4; [2] nonzero: some list is D4;
                        // [3] nonzero: the average chunk is wider than kStageBytes
  uint32_t *seg_in;     // [segs][kEnt] chain state entering the segment, by group entry
  uint32_t *live;       // [segs][kLiveCap] live line | successor distance << 16
  uint32_t *live_cnt;   // [segs]
  uint32_t *grp_map;    // [groups][kEnt] chain state after the group, by group entry
  uint32_t *grp_entry;  // [groups] entry line offset of the true chain (kNone: off it)
  uint32_t *grp_mbase;  // [groups] meta-blocks before the group
  uint32_t *list_qm;    // [count] line after the last meta-block; 0: the list is bad
  // look-back state of pl_tiles, one set per instance (D4 lists, other kinds):
  unsigned long long *op_ticket;  // [2] next tile
  uint32_t *op_flag;    // [2][tiles] 0 nothing yet, 1 aggregate, 2 inclusive
  uint4 *op_agg;        // [2][tiles] column sums of the tile since its last list head
  uint4 *op_inc;        // [2][tiles] the same from the first block of the tile's last list
  uint32_t *lastval;    // [count] last packed value of each list
};

struct PlLayout {
  size_t boffw, seg_base, grp_base, ctl, seg_in, live, live_cnt, grp_map, grp_entry, grp_mbase,
      list_qm, op_ticket, op_flag, op_agg, op_inc, lastval, total;
};

PlLayout pl_layout(uint64_t units, uint32_t count) {
  const uint64_t S = max_segs(units, count), G = max_groups(units, count);
  const uint64_t nch = (units + kChunk - 1) / kChunk;
  const uint64_t ntl = (nch + kTileChunks - 1) / kTileChunks;  // tiles
  size_t o = 0;
  auto take = [&o](size_t bytes) {
    const size_t r = o;
    o = a256(o + bytes);
    return r;
  };
  PlLayout L;
  L.boffw = take(8 * units);
  L.seg_base = take(4 * ((size_t)count + 1));
  L.grp_base = take(4 * ((size_t)count + 1));
  L.ctl = take(16);
  L.seg_in = take(4 * kEnt * S);
  L.live = take(4 * kLiveCap * S);
  L.live_cnt = take(4 * S);
  L.grp_map = take(4 * kEnt * G);
  L.grp_entry = take(4 * G);
  L.grp_mbase = take(4 * G);
  L.list_qm = take(4 * (size_t)count);
  L.op_ticket = take(16);  // the flags follow: one memset clears tickets and flags
  L.op_flag = take(8 * ntl);
  L.op_agg = take(32 * ntl);
  L.op_inc = take(32 * ntl);
  L.lastval = take(4 * (size_t)count);
  L.total = o;
  return L;
}

PlScratch carve(void *scratch, const PlLayout &L) {
  uint8_t *b = static_cast<uint8_t *>(scratch);
  PlScratch sc;
  sc.boffw = reinterpret_cast<uint64_t *>(b + L.boffw);
  sc.seg_base = reinterpret_cast<uint32_t *>(b + L.seg_base);
  sc.grp_base = reinterpret_cast<uint32_t *>(b + L.grp_base);
  sc.ctl = reinterpret_cast<uint32_t *>(b + L.ctl);
  sc.seg_in = reinterpret_cast<uint32_t *>(b + L.seg_in);
  sc.live = reinterpret_cast<uint32_t *>(b + L.live);
  sc.live_cnt = reinterpret_cast<uint32_t *>(b + L.live_cnt);
  sc.grp_map = reinterpret_cast<uint32_t *>(b + L.grp_map);
  sc.grp_entry = reinterpret_cast<uint32_t *>(b + L.grp_entry);
  sc.grp_mbase = reinterpret_cast<uint32_t *>(b + L.grp_mbase);
  sc.list_qm = reinterpret_cast<uint32_t *>(b + L.list_qm);
  sc.op_ticket = reinterpret_cast<unsigned long long *>(b + L.op_ticket);
  sc.op_flag = reinterpret_cast<uint32_t *>(b + L.op_flag);
  sc.op_agg = reinterpret_cast<uint4 *>(b + L.op_agg);
  sc.op_inc = reinterpret_cast<uint4 *>(b + L.op_inc);
  sc.lastval = reinterpret_cast<uint32_t *>(b + L.lastval);
  return sc;
}

// The look-back state of the second pl_tiles instance (lists of the other
// kinds): the upper halves of the state arrays.
__host__ __device__ inline PlScratch sc_other(const PlScratch &sc, uint64_t ntiles) {
  PlScratch o = sc;
  o.op_ticket = sc.op_ticket + 1;
  o.op_flag = sc.op_flag + ntiles;
  o.op_agg = sc.op_agg + ntiles;
  o.op_inc = sc.op_inc + ntiles;
  return o;
}

__device__ __forceinline__ uint32_t rd_u32(const uint8_t *p) {
  return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}

__device__ __forceinline__ uint32_t meta_blocks(const bp_list &L) { return (L.n / 128u) / 16u; }

__device__ __forceinline__ bool header_ok(const uint8_t *enc, const bp_list &L) {
  return L.enc_bytes >= 16 && (L.enc_offset & 15u) == 0 && rd_u32(enc) == L.n &&
         rd_u32(enc + 4) == 0u && rd_u32(enc + 12) <= 3u;  // word 3: kind of deltas
}

// Largest i < count with base[i] <= g (the list owning segment or group g).
__device__ __forceinline__ uint32_t owner(const uint32_t *base, uint32_t count, uint32_t g) {
  uint32_t lo = 0, hi = count - 1;
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) >> 1;
    if (base[mid] <= g) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ uint32_t lanemask_lt(int lane) { return (1u << lane) - 1u; }

// ---- plan: segments and groups of every list; the lists must tile the units ---------------

__device__ __forceinline__ uint64_t warp_incl_u64(uint64_t v, int lane) {
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint64_t t = __shfl_up_sync(kFull, v, d);
    if (lane >= d) v += t;
  }
  return v;
}

__global__ void __launch_bounds__(1024)
    pl_plan(const uint8_t *__restrict__ data, ListSrc src, uint64_t total_units, uint64_t max_s,
            uint64_t max_g, PlScratch sc, uint32_t *status) {
  __shared__ uint64_t s_w[32][3];
  __shared__ uint64_t s_carry[3];
  __shared__ uint32_t s_bad, s_other, s_d4;
  __shared__ unsigned long long s_enc;  // compressed bytes of all lists
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  if (tid == 0) {
    s_enc = 0;
    s_carry[0] = s_carry[1] = s_carry[2] = 0;
    s_bad = 0;
    s_other = 0;
    s_d4 = 0;
  }
  __syncthreads();
  for (uint64_t base = 0; base < src.count; base += 1024) {
    const uint64_t i = base + tid;
    uint64_t v[3] = {0, 0, 0};  // units, segments, groups
    bp_list L{};
    if (i < src.count) {
      L = src.get((uint32_t)i);
      v[0] = bp_fmt::units_of(L.n, BP_LAYOUT_PAPER);
      if (meta_blocks(L) > 0 && L.enc_bytes <= bp_fmt::pl_bound(L.n)) {
        v[1] = (L.enc_bytes / 16 + kSeg - 1) / kSeg;
        v[2] = (v[1] + kGrp - 1) / kGrp;
      }
    }
    uint64_t inc[3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
      inc[k] = warp_incl_u64(v[k], lane);
      if (lane == 31) s_w[w][k] = inc[k];
    }
    __syncthreads();
    uint64_t ex[3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
      uint64_t p = s_carry[k];
      for (int j = 0; j < w; j++) p += s_w[j][k];
      ex[k] = p + inc[k] - v[k];
    }
    if (i < src.count) {
      if (L.unit_base != ex[0]) s_bad = 1;
      // a list of another kind than D4 (header word 3): the decode passes for
      // those kinds have work
      if (L.enc_bytes >= 16 && (L.enc_offset & 15u) == 0 && rd_u32(data + L.enc_offset + 12) != 0u)
        s_other = 1;
      else
        s_d4 = 1;  // D4, or a bad header that the D4 passes report
      sc.seg_base[i] = (uint32_t)ex[1];
      sc.grp_base[i] = (uint32_t)ex[2];
      atomicAdd(&s_enc, (unsigned long long)L.enc_bytes);
    }
    __syncthreads();
    if (tid == 0) {
#pragma unroll
      for (int k = 0; k < 3; k++)
        for (int j = 0; j < 32; j++) s_carry[k] += s_w[j][k];
    }
    __syncthreads();
  }
  if (tid == 0) {
    const bool bad = s_bad || s_carry[0] != total_units || s_carry[1] > max_s ||
                     s_carry[2] > max_g;
    sc.seg_base[src.count] = bad ? 0u : (uint32_t)s_carry[1];
    sc.grp_base[src.count] = bad ? 0u : (uint32_t)s_carry[2];
    sc.ctl[0] = bad ? 1u : 0u;
    sc.ctl[1] = s_other;
    sc.ctl[2] = s_d4;
    // pl_tiles with the wider stage runs when a chunk of kChunk units
    // averages more bytes than the narrow stage holds
    sc.ctl[3] = (uint64_t)kChunk * s_enc > (uint64_t)kStageBytes * total_units ? 1u : 0u;
    if (bad) set_status(status, BP_ERR_ARG);
  }
}

// ---- parse: segment maps, composed per group -------------------------------------------------

__global__ void __launch_bounds__(kThreads)
    pl_parse(const uint8_t *__restrict__ data, ListSrc src, PlScratch sc) {
  constexpr int kRounds = kSeg / kThreads;  // lines per thread
  constexpr int kWarps = kThreads / 32;
  __shared__ uint32_t s_p[kSeg];
  __shared__ uint16_t s_live[kSeg];
  __shared__ uint32_t s_state[kEnt];
  __shared__ uint32_t s_ball[kRounds * kWarps];
  __shared__ uint32_t s_pre[kRounds * kWarps];
  __shared__ uint32_t s_nlive;
  if (sc.ctl[0]) return;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  volatile uint32_t *vp = s_p;
  const uint32_t ngroups = sc.grp_base[src.count];
  for (uint32_t h = blockIdx.x; h < ngroups; h += gridDim.x) {
    const uint32_t li = owner(sc.grp_base, src.count, h);
    const bp_list L = src.get(li);
    const uint4 *lines = reinterpret_cast<const uint4 *>(data + L.enc_offset);
    // whole lines of the stream (none if it is misaligned: pl_resolve rejects it)
    const uint64_t nu = (L.enc_offset & 15u) ? 0 : L.enc_bytes / 16;
    const uint32_t sb = sc.seg_base[li];
    const uint32_t nseg = sc.seg_base[li + 1] - sb;
    const uint32_t ls0 = (h - sc.grp_base[li]) * kGrp;
    const uint32_t ls1 = min(ls0 + kGrp, nseg);
    for (uint32_t x = tid; x < kEnt; x += kThreads) s_state[x] = x;
    __syncthreads();
    for (uint32_t ls = ls0; ls < ls1; ls++) {
      const uint32_t g = sb + ls;
      const uint64_t u0 = (uint64_t)ls * kSeg;
      for (uint32_t x = tid; x < kEnt; x += kThreads) sc.seg_in[(size_t)g * kEnt + x] = s_state[x];
      // one step from every line
      uint32_t livemask = 0;
#pragma unroll 4
      for (int r = 0; r < kRounds; r++) {
        const uint32_t i = r * kThreads + tid;
        const uint64_t u = u0 + i;
        uint32_t p = i;  // dead: stays put, no meta-block
        if (u >= 1 && u < nu) {
          const uint4 v = __ldg(lines + u);
          const uint32_t big = __vcmpgtu4(v.x, 0x20202020u) | __vcmpgtu4(v.y, 0x20202020u) |
                               __vcmpgtu4(v.z, 0x20202020u) | __vcmpgtu4(v.w, 0x20202020u);
          const uint32_t sum =
              __dp4a(v.x, 0x01010101u,
                     __dp4a(v.y, 0x01010101u, __dp4a(v.z, 0x01010101u, __dp4a(v.w, 0x01010101u, 0u))));
          if (big == 0u && u + 1 + sum <= nu) {
            p = (i + 1 + sum) | (1u << 16);
            livemask |= 1u << r;
          }
        }
        s_p[i] = p;
        const uint32_t bal = __ballot_sync(kFull, (livemask >> r) & 1u);
        if (lane == 0) s_ball[r * kWarps + w] = bal;
      }
      __syncthreads();
      if (w == 0) {  // exclusive prefix of the live counts in (round, warp) order
        uint32_t c[4], t = 0;
#pragma unroll
        for (int k = 0; k < 4; k++) {
          c[k] = __popc(s_ball[4 * lane + k]);
          t += c[k];
        }
        uint32_t inc = t;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          const uint32_t y = __shfl_up_sync(kFull, inc, d);
          if (lane >= d) inc += y;
        }
        uint32_t ex = inc - t;
#pragma unroll
        for (int k = 0; k < 4; k++) {
          s_pre[4 * lane + k] = ex;
          ex += c[k];
        }
        if (lane == 31) s_nlive = inc;
      }
      __syncthreads();
      const uint32_t nlive = s_nlive;
      uint32_t *gl_live = sc.live + (size_t)g * kLiveCap;
#pragma unroll 4
      for (int r = 0; r < kRounds; r++) {
        if ((livemask >> r) & 1u) {
          const uint32_t i = r * kThreads + tid;
          const uint32_t rank =
              s_pre[r * kWarps + w] + __popc(s_ball[r * kWarps + w] & lanemask_lt(lane));
          s_live[rank] = (uint16_t)i;
          if (nlive <= kLiveCap) gl_live[rank] = i | ((lo16(s_p[i]) - i) << 16);
        }
      }
      if (tid == 0) sc.live_cnt[g] = nlive;
      __syncthreads();
      // pointer jumping over the live lines (in place: every value read is a
      // consistent (target, count) pair, so rounds only converge faster)
      for (int round = 0; round < 16; round++) {
        int changed = 0;
        for (uint32_t k = tid; k < nlive; k += kThreads) {
          const uint32_t i = s_live[k];
          const uint32_t p = vp[i];
          const uint32_t a = lo16(p);
          if (a < kSeg) {
            const uint32_t q = vp[a];
            const uint32_t np = lo16(q) | ((p & 0xFFFF0000u) + (q & 0xFFFF0000u));
            if (np != p) {
              vp[i] = np;
              changed = 1;
            }
          }
        }
        if (!__syncthreads_or(changed)) break;
      }
      // compose the group's map with this segment's
      for (uint32_t x = tid; x < kEnt; x += kThreads) {
        const uint32_t st = s_state[x];
        const uint32_t off = lo16(st);
        if (off != kDead) {
          const uint32_t p = s_p[off];
          const uint32_t nr = lo16(p);
          const uint32_t cnt = (st >> 16) + (p >> 16);
          s_state[x] = (nr >= kSeg ? nr - kSeg : kDead) | (cnt << 16);
        }
      }
      __syncthreads();
    }
    for (uint32_t x = tid; x < kEnt; x += kThreads) sc.grp_map[(size_t)h * kEnt + x] = s_state[x];
    __syncthreads();
  }
}

// ---- resolve: the true chain through the groups of each list ----------------------------------

__global__ void __launch_bounds__(kThreads)
    pl_resolve(const uint8_t *__restrict__ data, ListSrc src, PlScratch sc, uint32_t *status) {
  __shared__ uint32_t s_map[kMapChunk * kEnt];
  __shared__ uint32_t s_e, s_m, s_st;  // s_st: 0 walking, 1 done, 2 bad
  if (sc.ctl[0]) return;
  const int tid = threadIdx.x;
  for (uint32_t li = blockIdx.x; li < src.count; li += gridDim.x) {
    const bp_list L = src.get(li);
    const uint32_t M = meta_blocks(L);
    const uint32_t h0 = sc.grp_base[li], h1 = sc.grp_base[li + 1];
    if (tid == 0) {
      s_e = 1;  // the first meta-block follows the 16-byte header
      s_m = 0;
      s_st = !header_ok(data + L.enc_offset, L) ? 2u : (M == 0 ? 1u : 0u);
    }
    __syncthreads();
    for (uint32_t hc = h0; hc < h1; hc += kMapChunk) {
      const uint32_t nh = min(kMapChunk, h1 - hc);
      if (s_st == 0)
        for (uint32_t k = tid; k < nh * kEnt; k += kThreads)
          s_map[k] = sc.grp_map[(size_t)hc * kEnt + k];
      __syncthreads();
      if (tid == 0) {
        uint32_t e = s_e, m = s_m, st = s_st;
        for (uint32_t j = 0; j < nh; j++) {
          const uint32_t h = hc + j;
          if (st != 0) {
            sc.grp_entry[h] = kNone;
            continue;
          }
          const uint32_t p = s_map[j * kEnt + e];
          sc.grp_entry[h] = e;
          sc.grp_mbase[h] = m;
          m += p >> 16;
          if (m >= M) st = 1;
          else if (lo16(p) == kDead) st = 2;
          else e = lo16(p);
        }
        s_e = e;
        s_m = m;
        s_st = st;
      }
      __syncthreads();
    }
    if (tid == 0) {
      const bool ok = s_st == 1;
      if (!ok) set_status(status, BP_ERR_CORRUPT);
      sc.list_qm[li] = ok ? (M == 0 ? 1u : kNone) : 0u;
    }
    __syncthreads();
  }
}

// ---- emit: block offsets and widths of every meta-block -----------------------------------

// One lane: the 16 blocks of the meta-block at `line`.
__device__ __forceinline__ void emit_meta(const uint4 *lines, uint64_t line, uint64_t *dst) {
  const uint4 v = __ldg(lines + line);
  const uint32_t wds[4] = {v.x, v.y, v.z, v.w};
  uint64_t off = 16ull * (line + 1);
#pragma unroll
  for (int j = 0; j < 16; j++) {
    const uint32_t b = (wds[j >> 2] >> (8 * (j & 3))) & 0xFFu;
    dst[j] = off | ((uint64_t)b << 56);
    off += 16ull * b;
  }
}

__global__ void __launch_bounds__(kThreads)
    pl_emit(const uint8_t *__restrict__ data, ListSrc src, PlScratch sc, uint32_t *status) {
  if (sc.ctl[0]) return;
  const int lane = threadIdx.x & 31;
  const uint32_t warp = (blockIdx.x * kThreads + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * kThreads) >> 5;
  const uint32_t nsegs = sc.seg_base[src.count];
  for (uint32_t g = warp; g < nsegs; g += nwarps) {
    const uint32_t li = owner(sc.seg_base, src.count, g);
    if (sc.list_qm[li] == 0u) continue;
    const uint32_t ls = g - sc.seg_base[li];
    const uint32_t h = sc.grp_base[li] + ls / kGrp;
    const uint32_t x = sc.grp_entry[h];
    if (x == kNone) continue;
    const uint32_t st = sc.seg_in[(size_t)g * kEnt + x];
    if (lo16(st) == kDead) continue;
    const bp_list L = src.get(li);
    const uint32_t M = meta_blocks(L);
    const uint32_t mb = sc.grp_mbase[h] + (st >> 16);
    if (mb >= M) continue;
    const uint32_t need = M - mb;
    const uint4 *lines = reinterpret_cast<const uint4 *>(data + L.enc_offset);
    const uint64_t nu = L.enc_bytes / 16;
    const uint64_t u0 = (uint64_t)ls * kSeg;
    uint64_t *dst = sc.boffw + L.unit_base + 16ull * mb;
    uint32_t t = lo16(st), done = 0;
    bool fail = false;
    const uint32_t nlive = sc.live_cnt[g];
    if (nlive <= kLiveCap) {
      // the live lines, in order, 32 at a time: find the chain's nodes among them
      const uint32_t *lv = sc.live + (size_t)g * kLiveCap;
      for (uint32_t p0 = 0; p0 < nlive && t < kSeg && done < need; p0 += 32) {
        const uint32_t e = p0 + lane < nlive ? lv[p0 + lane] : kNone;
        const uint32_t line = lo16(e);  // padding 0xFFFF never equals t < kSeg
        bool node = false;
        const uint32_t before = done;
        for (int it = 0; it < 32 && done < need; it++) {
          const uint32_t m = __ballot_sync(kFull, line == t);
          if (!m) break;
          const int sl = __ffs(m) - 1;
          node |= lane == sl;
          t += __shfl_sync(kFull, e >> 16, sl);
          done++;
        }
        const uint32_t nm = __ballot_sync(kFull, node);
        if (node) emit_meta(lines, u0 + line, dst + 16ull * (before + __popc(nm & lanemask_lt(lane))));
      }
    } else {
      // more live lines than kept: read each node's width line from the stream
      for (uint32_t it = 0; t < kSeg && done < need && it < kSeg; it++) {
        const uint64_t line = u0 + t;
        if (line >= nu) {
          fail = true;
          break;
        }
        const uint32_t wb = lane < 16 ? reinterpret_cast<const uint8_t *>(lines)[16 * line + lane] : 0u;
        if (__any_sync(kFull, wb > 32u)) {
          fail = true;
          break;
        }
        uint32_t inc = wb;
#pragma unroll
        for (int d = 1; d < 16; d <<= 1) {
          const uint32_t y = __shfl_up_sync(kFull, inc, d);
          if (lane >= d) inc += y;
        }
        const uint32_t tot = __shfl_sync(kFull, inc, 15);
        if (line + 1 + tot > nu) {
          fail = true;
          break;
        }
        if (lane < 16)
          dst[16ull * done + lane] = (16ull * (line + 1) + 16ull * (inc - wb)) | ((uint64_t)wb << 56);
        t += 1 + tot;
        done++;
      }
    }
    if (done == need) {
      if (lane == 0) sc.list_qm[li] = (uint32_t)(u0 + t);
    } else if (t < kSeg || fail) {
      // the segment maps promised a longer chain: the stream changed under us
      if (lane == 0) {
        set_status(status, BP_ERR_CORRUPT);
        sc.list_qm[li] = 0u;
      }
    }
  }
}

// ---- leftover blocks and the tail position ---------------------------------------------

__global__ void __launch_bounds__(kThreads)
    pl_leftover(const uint8_t *__restrict__ data, ListSrc src, PlScratch sc, uint64_t out_cap,
                bool sum, uint32_t *status) {
  if (sc.ctl[0]) return;
  const int lane = threadIdx.x & 31;
  const uint32_t warp = (blockIdx.x * kThreads + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * kThreads) >> 5;
  for (uint32_t li = warp; li < src.count; li += nwarps) {
    const bp_list L = src.get(li);
    const uint8_t *enc = data + L.enc_offset;
    const uint64_t bytes = L.enc_bytes, U0 = L.unit_base;
    const uint32_t nb = L.n / 128u;
    const uint32_t qm = sc.list_qm[li];
    bool ok = qm != 0u && qm != kNone;
    uint32_t why = BP_ERR_CORRUPT;
    if (ok && !sum && L.out_offset + L.n > out_cap) {
      ok = false;
      why = BP_ERR_CAPACITY;
    }
    uint64_t pos = 16ull * qm;
    for (uint32_t k = 16u * meta_blocks(L); ok && k < nb; k++) {
      if (pos + 1 > bytes) {
        ok = false;
        break;
      }
      const uint32_t wd = enc[pos];
      if (wd > 32u || pos + 1 + 16ull * wd > bytes) {
        ok = false;
        break;
      }
      if (lane == 0) sc.boffw[U0 + k] = (pos + 1) | ((uint64_t)wd << 56);
      pos += 1 + 16ull * wd;
    }
    if (ok && pos + rd_u32(enc + 8) != bytes) ok = false;
    if (ok) {
      if (lane == 0) sc.boffw[U0 + nb] = pos;
    } else {
      if (lane == 0) {
        set_status(status, why);
        sc.list_qm[li] = 0u;
      }
      for (uint32_t j = lane; j <= nb; j += 32) sc.boffw[U0 + j] = kBadEntry;
    }
  }
}

// ---- decode in one pass over tiles of work units ------------------------------------------

enum { kColsum = 0, kStore = 1, kSum = 2 };

__device__ __forceinline__ void flush_sum(uint64_t &acc, uint64_t *dst, int lane) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) acc += __shfl_down_sync(kFull, acc, d);
  if (lane == 0 && acc) atomicAdd(reinterpret_cast<unsigned long long *>(dst), acc);
  acc = 0;
}

// The values before a block, for each kind of Section 5, from the running
// column sums C_s of the deltas of the list's earlier blocks (lane 8s+c
// holds C_s in `carry`): D4 x[-4+s] = C_s; DM and D1 x[-1] = C_3 or
// C_0+C_1+C_2+C_3; D2 x[-2] = C_0+C_2 (even s), x[-1] = C_1+C_3 (odd s).
template <int KIND>
__device__ __forceinline__ uint32_t kind_seed(uint32_t carry) {
  if constexpr (KIND == kDM) return __shfl_sync(kFull, carry, 24);
  if constexpr (KIND == kD2) return carry + __shfl_xor_sync(kFull, carry, 16);
  if constexpr (KIND == kD1) {
    const uint32_t t = carry + __shfl_xor_sync(kFull, carry, 8);
    return t + __shfl_xor_sync(kFull, t, 16);
  }
  return carry;
}

// The list's last packed value x[128 nb - 1] (what the varint tail follows),
// from the column sums of all its blocks.
__device__ __forceinline__ uint32_t kind_last(uint32_t kind, uint32_t carry) {
  const uint32_t c3 = __shfl_sync(kFull, carry, 24), c1 = __shfl_sync(kFull, carry, 8);
  const uint32_t c0 = __shfl_sync(kFull, carry, 0), c2 = __shfl_sync(kFull, carry, 16);
  if (kind == kD2) return c1 + c3;
  if (kind == kD1) return c0 + c1 + c2 + c3;
  return c3;  // D4 and DM: position 128 nb - 1 is in column 3
}

__device__ __forceinline__ uint32_t comp(const uint4 &v, int s) {
  return s == 0 ? v.x : s == 1 ? v.y : s == 2 ? v.z : v.w;
}

__device__ __forceinline__ uint4 add4(const uint4 &a, const uint4 &b) {
  return make_uint4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_u32(uint32_t *p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Publish the state of tile t: its column sums `v` as an aggregate (flag 1:
// its first list continues from earlier tiles) or as the inclusive sums of
// its last list (flag 2).  Aggregates and inclusive sums are kept apart, so
// a reader that saw flag 1 never reads a later inclusive value.  One thread.
__device__ __forceinline__ void tile_publish(const PlScratch &sc, uint64_t t, uint32_t flag,
                                             const uint4 &v) {
  __stcg(flag == 2u ? sc.op_inc + t : sc.op_agg + t, v);
  st_release_u32(sc.op_flag + t, flag);
}

// Column sums of tile t's first list over all tiles before t (decoupled
// look-back by one warp): each step reads the 32 nearest tiles not yet
// accounted for, adds their aggregates down to the nearest inclusive sums
// and stops there, or moves 32 tiles back.  Every poll is bounded; on
// timeout it records BP_ERR_TIMEOUT and goes on with what it has.
__device__ __forceinline__ uint4 tile_lookback(const PlScratch &sc, uint64_t t,
                                               uint32_t spin_limit, uint32_t *status, int lane) {
  uint4 excl = make_uint4(0, 0, 0, 0);
  for (int64_t top = (int64_t)t - 1; top >= 0; top -= 32) {
    const int64_t j = top - lane;
    uint32_t f = 2u;  // before tile 0: inclusive sums of zero
    uint4 v = make_uint4(0, 0, 0, 0);
    if (j >= 0) {
      uint32_t spins = 0;
      while ((f = ld_acquire_u32(sc.op_flag + j)) == 0u) {
        if (++spins > spin_limit) break;
        __nanosleep(64);
      }
      if (f == 1u) v = __ldcg(sc.op_agg + j);
      else if (f == 2u) v = __ldcg(sc.op_inc + j);
    }
    if (__any_sync(kFull, f == 0u)) {
      if (lane == 0) set_status(status, BP_ERR_TIMEOUT);
      break;
    }
    const uint32_t incl = __ballot_sync(kFull, f == 2u);
    const int stop = incl ? __ffs(incl) - 1 : 31;
    const bool take = lane <= stop;
    excl.x += __reduce_add_sync(kFull, take ? v.x : 0u);
    excl.y += __reduce_add_sync(kFull, take ? v.y : 0u);
    excl.z += __reduce_add_sync(kFull, take ? v.z : 0u);
    excl.w += __reduce_add_sync(kFull, take ? v.w : 0u);
    if (incl) break;
  }
  return excl;
}

// Where a full chunk's blocks are read from: the shared-memory stage, or
// global memory for a chunk too wide for the stage (after one L2 prefetch);
// `off` is a block's byte offset from the chunk's first block.
struct StagedBlocks {
  uint32_t sbase;
  __device__ __forceinline__ PlSharedWords at(uint32_t off) const { return PlSharedWords{sbase + off}; }
};
struct GlobalBlocks {
  const uint8_t *p;  // 16-byte aligned
  __device__ __forceinline__ PlGlobalWords<true> at(uint32_t off) const {
    return PlGlobalWords<true>{p + off};
  }
};

// One block of a run: its deltas d become values, stored or summed, with
// the running column sums `carry`.
template <int MODE, int KIND>
__device__ __forceinline__ void staged_block(uint32_t d[4], int lane, uint32_t &carry,
                                             uint32_t *&o, uint64_t &acc) {
  const int c = lane & 7;
  if (MODE == kColsum) {
    carry += d[0] + d[1] + d[2] + d[3];
    return;
  }
  if constexpr (KIND != kD4) {
    uint32_t x[4], ctot;
    prefix_block<KIND>(d, kind_seed<KIND>(carry), lane, x, ctot);
    carry += ctot;
    if (MODE == kSum) {
      acc += (uint64_t)x[0] + x[1] + x[2] + x[3];
    } else {
      o[0] = x[0];
      o[4] = x[1];
      o[8] = x[2];
      o[12] = x[3];
      o += 128;
    }
    return;
  }
  const uint32_t x0 = d[0], x1 = x0 + d[1], x2 = x1 + d[2], x3 = x2 + d[3];
  uint32_t inc = x3;
#pragma unroll
  for (int dd = 1; dd < 8; dd <<= 1) {
    const uint32_t t = __shfl_up_sync(kFull, inc, dd, 8);
    if (c >= dd) inc += t;
  }
  const uint32_t base = carry + inc - x3;
  carry += __shfl_sync(kFull, inc, (lane & ~7) | 7);
  if (MODE == kSum) {
    acc += (uint64_t)(x0 + base) + (x1 + base) + (x2 + base) + (x3 + base);
  } else {
    o[0] = x0 + base;
    o[4] = x1 + base;
    o[8] = x2 + base;
    o[12] = x3 + base;
    o += 128;
  }
}

template <int B, int MODE, int KIND, class BL>
__device__ __forceinline__ void staged_run(uint32_t pk, uint32_t j, uint32_t run, const BL &blocks,
                                           int lane, uint32_t &carry, uint32_t *&o,
                                           uint64_t &acc) {
  if constexpr (std::is_same<BL, GlobalBlocks>::value && KIND == kD4) {
    // D4 blocks in global memory: the loads of two blocks are issued before
    // either is used, so they share one round trip
    uint32_t r = 0;
#pragma unroll 1
    for (; r + 1 < run; r += 2) {
      const uint32_t p0 = __shfl_sync(kFull, pk, j + r), p1 = __shfl_sync(kFull, pk, j + r + 1);
      uint32_t d0[4], d1[4];
      pl_lane_deltas<B>(blocks.at(p0 & 0xFFFFu), lane, d0);
      pl_lane_deltas<B>(blocks.at(p1 & 0xFFFFu), lane, d1);
      staged_block<MODE, KIND>(d0, lane, carry, o, acc);
      staged_block<MODE, KIND>(d1, lane, carry, o, acc);
    }
    if (r < run) {
      const uint32_t p0 = __shfl_sync(kFull, pk, j + r);
      uint32_t d0[4];
      pl_lane_deltas<B>(blocks.at(p0 & 0xFFFFu), lane, d0);
      staged_block<MODE, KIND>(d0, lane, carry, o, acc);
    }
  } else {
#pragma unroll 1
    for (uint32_t r = 0; r < run; r++) {
      const uint32_t p = __shfl_sync(kFull, pk, j + r);
      uint32_t d[4];
      pl_lane_deltas<B>(blocks.at(p & 0xFFFFu), lane, d);
      staged_block<MODE, KIND>(d, lane, carry, o, acc);
    }
  }
}

// The 32 blocks of a full chunk, one width dispatch per run of consecutive
// blocks of equal width.
template <int MODE, int KIND, class BL>
__device__ __forceinline__ void staged_chunk(uint32_t pk, const BL &blocks, int lane,
                                             uint32_t &carry, uint32_t *o, uint64_t &acc) {
  const uint32_t bw = pk >> 16;
  for (uint32_t j = 0; j < kChunk;) {
    const uint32_t b = __shfl_sync(kFull, bw, j);
    const uint32_t same = __ballot_sync(kFull, bw == b) >> j;  // bit r: block j + r
    const uint32_t run = ~same ? (uint32_t)__ffs(~same) - 1 : kChunk - j;
    switch (b) {
#define BP_CASE(B)                                                      \
  case B:                                                               \
    staged_run<B, MODE, KIND>(pk, j, run, blocks, lane, carry, o, acc); \
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
}


// Column sums of a full chunk (staged, or read from global memory), one
// lane per block.  Line k of a block (16 bytes) holds word k of each of the
// 4 lane streams, and field i of stream s is bits [b i, b i + b) of that
// stream (Section 4.2, Fig. 2): lane j reads block j's lines in order
// through a window of three lines and adds the 4 deltas of each field, one
// funnel shift each.  The width is a run-time value: every lane runs the
// same 32 field steps.
struct LbWin {
  uint4 w0, w1, w2;  // lines kc, kc + 1 and kc + 2 (zeros past the block)
  uint32_t kc;
};

__device__ __forceinline__ uint4 lb_line(const uint4 *lines, uint32_t k, uint32_t b) {
  return k < b ? lines[k] : make_uint4(0, 0, 0, 0);
}

// Sum of the 4 b-bit fields (b <= 8) at the bottom of v: fields 0 + 2 and
// 1 + 3 are added in place (each sum fits in b + 1 <= 2b bits), then folded.
__device__ __forceinline__ uint32_t lb_sum4(uint32_t v, uint32_t b, uint32_t m02, uint32_t low) {
  const uint32_t t = (v & m02) + ((v >> b) & m02);
  return (t & low) + (t >> (2u * b));
}

__device__ __forceinline__ uint4 lb_colsum(const uint4 *lines, uint32_t b) {
  const uint32_t mask = b >= 32u ? ~0u : (1u << b) - 1u;
  LbWin win{lb_line(lines, 0, b), lb_line(lines, 1, b), lb_line(lines, 2, b), 0};
  uint4 sum = make_uint4(0, 0, 0, 0);
  if (b <= 8u) {
    // 4 fields (4b <= 32 bits) per step, from one funnel shift per stream
    const uint32_t m02 = mask | (mask << (2u * b)), low = (1u << (2u * b)) - 1u;
    uint32_t p = 0;
#pragma unroll 2
    for (int i = 0; i < 8; i++, p += 4u * b) {
      const uint32_t k = p >> 5, r = p & 31u;
      if (k != win.kc) {
        win.kc = k;
        win.w0 = win.w1;
        win.w1 = win.w2;
        win.w2 = lb_line(lines, k + 2, b);
      }
      sum.x += lb_sum4(__funnelshift_r(win.w0.x, win.w1.x, r), b, m02, low);
      sum.y += lb_sum4(__funnelshift_r(win.w0.y, win.w1.y, r), b, m02, low);
      sum.z += lb_sum4(__funnelshift_r(win.w0.z, win.w1.z, r), b, m02, low);
      sum.w += lb_sum4(__funnelshift_r(win.w0.w, win.w1.w, r), b, m02, low);
    }
    return sum;
  }
  uint32_t p = 0;
#pragma unroll 4
  for (int i = 0; i < 32; i++, p += b) {
    // field i starts at bit p: word k = p / 32 of each stream, joined with
    // word k + 1 when it straddles; the window moves by at most one line
    const uint32_t k = p >> 5, r = p & 31u;
    if (k != win.kc) {
      win.kc = k;
      win.w0 = win.w1;
      win.w1 = win.w2;
      win.w2 = lb_line(lines, k + 2, b);
    }
    sum.x += __funnelshift_r(win.w0.x, win.w1.x, r) & mask;
    sum.y += __funnelshift_r(win.w0.y, win.w1.y, r) & mask;
    sum.z += __funnelshift_r(win.w0.z, win.w1.z, r) & mask;
    sum.w += __funnelshift_r(win.w0.w, win.w1.w, r) & mask;
  }
  return sum;
}

// The list table as pl_tiles reads it: a copy in shared memory (with each
// list's kind of deltas) when it has at most kListCache lists, so that
// finding a chunk's list costs no global memory round trips.
constexpr uint32_t kListCache = 32;

struct TileLists {
  ListSrc src;
  const bp_list *sl;      // shared copy, or nullptr
  const uint32_t *skind;  // shared kinds
  uint32_t count;
  __device__ __forceinline__ bp_list get(uint32_t i) const { return sl ? sl[i] : src.get(i); }
  __device__ __forceinline__ uint64_t unit_base(uint32_t i) const {
    return sl ? sl[i].unit_base : src.unit_base(i);
  }
  // list owning unit u: largest i with unit_base(i) <= u
  __device__ __forceinline__ uint32_t find(uint64_t u) const {
    uint32_t lo = 0, hi = count - 1;
    while (lo < hi) {
      const uint32_t mid = (lo + hi + 1) >> 1;
      if (unit_base(mid) <= u) lo = mid;
      else hi = mid - 1;
    }
    return lo;
  }
  // kind of differential coding (header word 3; kD4 for a short or bad
  // header, whose list is marked bad and never decoded)
  __device__ __forceinline__ uint32_t kind(const uint8_t *data, uint32_t i, const bp_list &L) const {
    if (sl) return skind[i];
    const uint32_t k = L.enc_bytes >= 16 ? rd_u32(data + L.enc_offset + 12) : 0u;
    return k <= 3u ? k : (uint32_t)kD4;
  }
};

// A warp's chunk of kChunk work units and how much of it sits in the stage.
struct Chunk {
  uint64_t u0;
  uint32_t cnt;
  uint64_t eL;      // lane j < cnt: boffw of unit u0 + j
  uint32_t staged;  // leading units whose blocks are in the stage
  uint64_t st0;     // stream offset of the stage's first byte
  bool gl;          // a full chunk too wide for the stage: its blocks are read from global
};

// Stage the chunk's leading blocks of its first list: they lie back to back
// in the meta-block region, 16-byte aligned, only width lines between them,
// so one bulk copy brings them in when they fit.  False if the copy's wait
// ran out (recorded; the copy has landed or given up when this returns).
__device__ __forceinline__ bool stage_chunk(const uint8_t *data, const TileLists &src,
                                            const PlScratch &sc, uint64_t ch,
                                            uint64_t total_units, int lane, uint32_t bar,
                                            uint32_t sbase, uint32_t stage_bytes,
                                            uint32_t &phase, Chunk &cx, uint32_t *status) {
  cx.u0 = ch * kChunk;
  cx.cnt = total_units - cx.u0 < kChunk ? (uint32_t)(total_units - cx.u0) : kChunk;
  cx.eL = (uint32_t)lane < cx.cnt ? sc.boffw[cx.u0 + lane] : kBadEntry;
  cx.staged = 0;
  cx.st0 = 0;
  cx.gl = false;
  const uint32_t li = src.find(cx.u0);
  const bp_list L = src.get(li);
  const uint64_t nxt = li + 1 < src.count ? src.unit_base(li + 1) : ~0ull;
  const uint64_t k0 = cx.u0 - L.unit_base, nb0 = L.n / 128u;
  uint64_t m = nb0 > k0 ? nb0 - k0 : 0;
  if (m > cx.cnt) m = cx.cnt;
  if (m > nxt - cx.u0) m = nxt - cx.u0;
  const uint64_t offl = cx.eL & kOffMask;
  const uint32_t bl = (uint32_t)(cx.eL >> 56);
  const bool fit = __all_sync(kFull, (uint32_t)lane >= m || (bl <= 32u && (offl & 15u) == 0));
  if (m > 0 && fit) {
    const uint64_t st0 = __shfl_sync(kFull, offl, 0);
    const uint64_t bytes = __shfl_sync(kFull, offl + 16ull * bl, (int)m - 1) - st0;
    if (bytes > 0 && bytes <= stage_bytes) {
      if (lane == 0) bulk_load(bar, sbase, data + L.enc_offset + st0, (uint32_t)bytes);
      const bool done = bulk_wait(bar, phase);
      phase ^= 1u;
      if (!__all_sync(kFull, done)) {  // record it and let the copy land (bounded)
        if (lane == 0) set_status(status, BP_ERR_TIMEOUT);
        bulk_wait(bar, phase ^ 1u);
        return false;
      }
      cx.staged = (uint32_t)m;
      cx.st0 = st0;
    } else if (bytes > 0 && m == kChunk) {
      // too wide for this instance's stage: the fast paths read the
      // blocks from global memory, pulled into L2 here
      if (lane == 0) bulk_prefetch_l2(data + L.enc_offset + st0, (uint32_t)bytes);
      cx.staged = kChunk;
      cx.st0 = st0;
      cx.gl = true;
    }
  }
  return true;
}

// Decode or sum a full chunk of this instance's kind.
template <int MODE, bool OTHER, class BL>
__device__ __forceinline__ void full_chunk(uint32_t kind, uint32_t pk, const BL &blocks, int lane,
                                           uint32_t &carry, uint32_t *o, uint64_t &acc) {
  if constexpr (MODE == kColsum || !OTHER) {
    staged_chunk<MODE, kD4>(pk, blocks, lane, carry, o, acc);
  } else {
    if (kind == kDM) staged_chunk<MODE, kDM>(pk, blocks, lane, carry, o, acc);
    else if (kind == kD2) staged_chunk<MODE, kD2>(pk, blocks, lane, carry, o, acc);
    else staged_chunk<MODE, kD1>(pk, blocks, lane, carry, o, acc);
  }
}

// The chunk's units, once the stage is filled.  MODE kColsum: `carry` ends
// as this lane's part of the column sums of the chunk's last list within the
// chunk (from its head if it starts here: `head`); a fully staged chunk sums
// one block per lane and leaves all of column s in lane 8s.  MODE kStore / kSum: the
// blocks of lists of this instance's kind (D4, or the others if OTHER) are
// decoded with the running column sums `carry` (the chunk's seed on entry;
// the same in the 8 lanes of a column), stored or summed; a list's tail unit
// records its last packed value.
template <int MODE, bool OTHER>
__device__ __forceinline__ void chunk_units(const uint8_t *data, const TileLists &src,
                                            const PlScratch &sc, const Chunk &cx,
                                            uint32_t *out, uint64_t *sums, const uint4 *stage,
                                            int lane, uint32_t &carry, bool &head,
                                            uint64_t &acc, uint32_t &acc_list, uint32_t *status) {
  const int s = lane >> 3, c = lane & 7;
  const uint32_t sbase = smem_addr(stage);
  uint32_t li = src.find(cx.u0);
  bp_list L = src.get(li);
  uint64_t nxt = li + 1 < src.count ? src.unit_base(li + 1) : ~0ull;
  uint32_t kind = MODE == kColsum ? (uint32_t)kD4 : src.kind(data, li, L);
  if (MODE != kColsum && cx.u0 + cx.cnt <= nxt && (kind != kD4) != OTHER) return;
  if (cx.staged == kChunk && (MODE == kColsum || (kind != kD4) == OTHER)) {
    // Fast path: all 32 units are staged blocks of list li (no list change,
    // no tail unit).
    const uint64_t k0 = cx.u0 - L.unit_base;
    if (k0 == 0) {
      carry = 0;
      head = true;
    }
    const uint8_t *gblk = data + L.enc_offset + cx.st0;  // the chunk's first block in global
    if (MODE == kColsum) {
      // one lane per block, then a sum over the lanes
      const uint32_t off = (uint32_t)((cx.eL & kOffMask) - cx.st0);
      const uint32_t b = (uint32_t)(cx.eL >> 56);
      uint4 v = cx.gl ? lb_colsum(reinterpret_cast<const uint4 *>(gblk + off), b)
                      : lb_colsum(stage + (off >> 4), b);
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        v.x += __shfl_xor_sync(kFull, v.x, d);
        v.y += __shfl_xor_sync(kFull, v.y, d);
        v.z += __shfl_xor_sync(kFull, v.z, d);
        v.w += __shfl_xor_sync(kFull, v.w, d);
      }
      carry = c ? 0u : comp(v, s);
      return;
    }
    // decode: each lane's block offset in the stage and width packed in one word
    const uint32_t pk = (uint32_t)((cx.eL & kOffMask) - cx.st0) | (uint32_t)((cx.eL >> 56) << 16);
    if (MODE == kSum && acc_list != li) {
      if (acc_list != kNone) flush_sum(acc, sums + acc_list, lane);
      acc_list = li;
    }
    uint32_t *o = MODE == kStore ? out + L.out_offset + 128ull * k0 + 16 * c + s : nullptr;
    if (cx.gl) full_chunk<MODE, OTHER>(kind, pk, GlobalBlocks{gblk}, lane, carry, o, acc);
    else full_chunk<MODE, OTHER>(kind, pk, StagedBlocks{sbase}, lane, carry, o, acc);
    return;
  }
  for (uint32_t j = 0; j < cx.cnt; j++) {
    const uint64_t u = cx.u0 + j;
    if (u == nxt) {
      li++;
      L = src.get(li);
      nxt = li + 1 < src.count ? src.unit_base(li + 1) : ~0ull;
      kind = MODE == kColsum ? (uint32_t)kD4 : src.kind(data, li, L);
    }
    const uint64_t k = u - L.unit_base;
    if (k == 0) {
      carry = 0;
      head = true;
    }
    if (MODE != kColsum && (kind != kD4) != OTHER) continue;  // the other instance's list
    const uint64_t e = __shfl_sync(kFull, cx.eL, j);
    if (k >= L.n / 128u) {  // the tail unit: record the last packed value
      if (MODE != kColsum) {
        const uint32_t lv = kind_last(kind, carry);
        if (lane == 24) sc.lastval[li] = lv;
      }
      continue;
    }
    const uint32_t b = (uint32_t)(e >> 56);
    if (b > 32u) {
      if (MODE == kColsum && !OTHER && lane == 0 && sc.list_qm[li] != 0u)
        set_status(status, BP_ERR_CORRUPT);
      continue;
    }
    uint32_t d[4];
    if (j < cx.staged)
      pl_block_deltas_from((int)b, PlSharedWords{sbase + (uint32_t)((e & kOffMask) - cx.st0)}, lane, d);
    else
      pl_block_deltas((int)b, data + L.enc_offset + (e & kOffMask), lane, d);
    if (MODE == kColsum) {
      carry += d[0] + d[1] + d[2] + d[3];
      continue;
    }
    uint32_t x0, x1, x2, x3;
    if constexpr (!OTHER) {
      x0 = d[0];
      x1 = x0 + d[1];
      x2 = x1 + d[2];
      x3 = x2 + d[3];
      uint32_t inc = x3;
#pragma unroll
      for (int dd = 1; dd < 8; dd <<= 1) {
        const uint32_t t = __shfl_up_sync(kFull, inc, dd, 8);
        if (c >= dd) inc += t;
      }
      const uint32_t bs = carry + inc - x3;
      x0 += bs;
      x1 += bs;
      x2 += bs;
      x3 += bs;
      carry += __shfl_sync(kFull, inc, (lane & ~7) | 7);
    } else {
      uint32_t x[4], ctot;
      if (kind == kDM) prefix_block<kDM>(d, kind_seed<kDM>(carry), lane, x, ctot);
      else if (kind == kD2) prefix_block<kD2>(d, kind_seed<kD2>(carry), lane, x, ctot);
      else prefix_block<kD1>(d, kind_seed<kD1>(carry), lane, x, ctot);
      carry += ctot;
      x0 = x[0];
      x1 = x[1];
      x2 = x[2];
      x3 = x[3];
    }
    if (MODE == kSum) {
      if (acc_list != li) {
        if (acc_list != kNone) flush_sum(acc, sums + acc_list, lane);
        acc_list = li;
      }
      acc += (uint64_t)x0 + x1 + x2 + x3;
    } else {
      uint32_t *o = out + L.out_offset + 128ull * k + 16 * c + s;
      o[0] = x0;
      o[4] = x1;
      o[8] = x2;
      o[12] = x3;
    }
  }
}

// A tile is kTileChunks chunks of kChunk units, one per chunk warp, taken by
// a CTA in ticket order (a tile only waits for tiles that running CTAs
// hold).  The CTA has kTileChunks chunk warps and one control warp, and it
// works on two tiles at once:
//  - the chunk warps stage their chunk of tile i+1 in one of their two
//    buffers and sum its columns (phase 1), while the control warp looks
//    back for tile i's seed (the column sums of its first list over the
//    earlier tiles) and hands each chunk warp its seed;
//  - after a barrier the chunk warps decode their chunk of tile i from the
//    other buffer (phase 2), while the control warp publishes tile i+1's
//    sums and takes the next ticket.
// So the look-back's latency overlaps phase 1, and the compressed stream
// is read from memory once.  OTHER = false decodes the D4 lists, OTHER =
// true the DM, D2 and D1 lists (launched after the first, leaving at once
// if there are none); each runs its own tiles and look-back state.
template <int MODE, bool OTHER, uint32_t STAGE>
__global__ void __launch_bounds__(kTileThreads, STAGE > kStageBytes ? 3 : kTileMinBlocks)
    pl_tiles(const uint8_t *__restrict__ data, ListSrc src_in, uint64_t total_units,
             uint32_t *__restrict__ out, uint64_t *sums, PlScratch sc, uint32_t spin_limit,
             uint32_t *status) {
  if (sc.ctl[0] || (OTHER ? !sc.ctl[1] : !sc.ctl[2])) return;  // no list of this kind
  if ((sc.ctl[3] != 0u) != (STAGE > kStageBytes)) return;      // the other stage size runs
  constexpr int kW = kTileChunks;  // chunk warps; warp kW is the control warp
  __shared__ __align__(128) uint8_t s_stage[2][kW][STAGE];
  __shared__ bp_list s_lists[kListCache];
  __shared__ uint32_t s_kinds[kListCache];
  __shared__ __align__(8) uint64_t s_bar[2][kW];
  __shared__ uint4 s_sum[2][kW], s_seed[kW];
  __shared__ uint32_t s_head[2][kW];
  __shared__ uint64_t s_u0[2][kW], s_st0[2][kW];  // a chunk's first unit, stage offset
  __shared__ uint32_t s_cnt[2][kW], s_staged[2][kW];
  __shared__ bool s_gl[2][kW];
  __shared__ unsigned long long s_tile[2];
  __shared__ uint32_t s_abort;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const bool control = w == kW;
  uint32_t parity = 0;  // bit b: phase parity of buffer b's mbarrier
  if (!control && lane == 0) {
    bulk_bar_init(smem_addr(&s_bar[0][w]));
    bulk_bar_init(smem_addr(&s_bar[1][w]));
  }
  const uint64_t nch = (total_units + kChunk - 1) / kChunk;
  const uint64_t ntiles = (nch + kW - 1) / kW;
  const PlScratch st = OTHER ? sc_other(sc, ntiles) : sc;  // this instance's look-back state
  const bool cached = src_in.count <= kListCache;
  if (cached) {
    for (uint32_t k = threadIdx.x; k < src_in.count; k += kTileThreads) {
      const bp_list L = src_in.get(k);
      s_lists[k] = L;
      const uint32_t kd = L.enc_bytes >= 16 ? rd_u32(data + L.enc_offset + 12) : 0u;
      s_kinds[k] = kd <= 3u ? kd : (uint32_t)kD4;
    }
  }
  const TileLists src{src_in, cached ? s_lists : nullptr, s_kinds, src_in.count};
  if (threadIdx.x == 0) {
    s_abort = 0;
    s_tile[0] = atomicAdd(st.op_ticket, 1ull);
  }
  __syncthreads();
  uint64_t acc = 0;
  uint32_t acc_list = kNone;
  bool pub_any = false;
  for (int i = 0, first = 1;; i ^= 1, first = 0) {
    // phase 1 of a chunk warp: stage chunk w of tile `t` in buffer b and sum
    // its columns; the control warp then publishes the tile's sums
    const int b = first ? 0 : i ^ 1;
    const uint64_t t = first ? s_tile[0] : s_tile[i ^ 1];
    uint64_t tile = 0;
    if (!first) {
      tile = s_tile[i];
      if (tile >= ntiles || s_abort) break;
    }
    if (control) {
      if (!first) {
        // the seed of `tile`: its first list continues from earlier tiles
        // unless the tile starts at a list head
        uint4 agg = make_uint4(0, 0, 0, 0);
        for (int k = 0; k < kW; k++) agg = s_head[i][k] ? s_sum[i][k] : add4(agg, s_sum[i][k]);
        const uint64_t u0 = tile * kW * kChunk;
        const bool starts = src.unit_base(src.find(u0)) == u0;
        uint4 e = starts ? make_uint4(0, 0, 0, 0)
                         : tile_lookback(st, tile, spin_limit, status, lane);
        if (!pub_any && lane == 0) tile_publish(st, tile, 2u, add4(e, agg));
        if (lane == 0) {
          for (int k = 0; k < kW; k++) {
            s_seed[k] = e;
            e = s_head[i][k] ? s_sum[i][k] : add4(e, s_sum[i][k]);
          }
        }
      }
    } else {
      const uint64_t ch = t * kW + w;
      bool ok = true, head = false;
      uint32_t carry = 0;
      // a chunk inside one list of the other instance's kind: nothing to sum
      // or decode here, and no chunk of this kind looks back past it (a
      // look-back stays within one list), so it counts as a list head
      bool mine = true;
      if (t < ntiles && ch < nch) {
        const uint64_t u0 = ch * kChunk;
        const uint32_t li = src.find(u0);
        const uint64_t nxt = li + 1 < src.count ? src.unit_base(li + 1) : ~0ull;
        const uint64_t end = u0 + kChunk < total_units ? u0 + kChunk : total_units;
        const bp_list L = src.get(li);
        mine = !(end <= nxt && (src.kind(data, li, L) != kD4) != OTHER);
      }
      if (t < ntiles && ch < nch && mine) {
        const uint32_t sb = smem_addr(&s_stage[b][w][0]);
        Chunk cx;
        uint32_t ph = (parity >> b) & 1u;
        ok = stage_chunk(data, src, sc, ch, total_units, lane, smem_addr(&s_bar[b][w]), sb, STAGE,
                         ph, cx, status);
        parity = (parity & ~(1u << b)) | (ph << b);
        if (lane == 0) {
          s_u0[b][w] = cx.u0;
          s_cnt[b][w] = cx.cnt;
          s_staged[b][w] = cx.staged;
          s_st0[b][w] = cx.st0;
          s_gl[b][w] = cx.gl;
        }
        if (ok)
          chunk_units<kColsum, OTHER>(data, src, sc, cx, out, sums,
                                      reinterpret_cast<const uint4 *>(&s_stage[b][w][0]), lane,
                                      carry, head, acc, acc_list, status);
        carry += __shfl_xor_sync(kFull, carry, 1);
        carry += __shfl_xor_sync(kFull, carry, 2);
        carry += __shfl_xor_sync(kFull, carry, 4);
      }
      const uint4 cs = make_uint4(__shfl_sync(kFull, carry, 0), __shfl_sync(kFull, carry, 8),
                                  __shfl_sync(kFull, carry, 16), __shfl_sync(kFull, carry, 24));
      if (lane == 0) {
        if (!(t < ntiles && ch < nch && mine)) s_cnt[b][w] = 0u;  // no phase 2
        s_sum[b][w] = cs;
        s_head[b][w] = (ch >= nch || head || !mine) ? 1u : 0u;  // past the end: nothing continues
        if (!ok) s_abort = 1;
      }
    }
    __syncthreads();
    if (s_abort) break;
    if (control) {
      if (t < ntiles) {  // publish t's sums, take the ticket after it
        uint4 agg = make_uint4(0, 0, 0, 0);
        bool any = false;
        for (int k = 0; k < kW; k++) {
          agg = s_head[b][k] ? s_sum[b][k] : add4(agg, s_sum[b][k]);
          any |= s_head[b][k] != 0u;
        }
        if (lane == 0) tile_publish(st, t, any ? 2u : 1u, agg);
        pub_any = any;
      }
      if (lane == 0) s_tile[first ? 1 : i] = t < ntiles ? atomicAdd(st.op_ticket, 1ull) : t;
    } else if (!first && tile * kW + w < nch && s_cnt[i][w] != 0u) {
      // phase 2: decode chunk w of `tile` from buffer i with its seed
      Chunk cx;
      cx.u0 = s_u0[i][w];
      cx.cnt = s_cnt[i][w];
      cx.staged = s_staged[i][w];
      cx.st0 = s_st0[i][w];
      cx.gl = s_gl[i][w];
      cx.eL = (uint32_t)lane < cx.cnt ? sc.boffw[cx.u0 + lane] : kBadEntry;
      uint32_t carry = comp(s_seed[w], lane >> 3);
      bool head = false;
      chunk_units<MODE, OTHER>(data, src, sc, cx, out, sums,
                               reinterpret_cast<const uint4 *>(&s_stage[i][w][0]), lane, carry,
                               head, acc, acc_list, status);
      __syncwarp();  // every lane is done with buffer i before it is refilled
    }
    __syncthreads();
    if (first) i = 1;  // after the first pass tile s_tile[0] sits in buffer 0: i becomes 0
  }
  if (MODE == kSum && acc_list != kNone) flush_sum(acc, sums + acc_list, lane);
}

template <bool SUM>
__global__ void __launch_bounds__(kThreads)
    pl_tail(const uint8_t *__restrict__ data, ListSrc src, uint32_t *__restrict__ out,
            uint64_t *sums, PlScratch sc, uint32_t *status) {
  __shared__ uint8_t s_bytes[kThreads / 32][640];
  if (sc.ctl[0]) return;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint32_t warp = (blockIdx.x * kThreads + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * kThreads) >> 5;
  for (uint32_t li = warp; li < src.count; li += nwarps) {
    const bp_list L = src.get(li);
    const uint32_t nb = L.n / 128u, np = 128u * nb, nt = L.n - np;
    const uint64_t e = sc.boffw[L.unit_base + nb];
    if (nt == 0 || e == kBadEntry) continue;
    const uint8_t *enc = data + L.enc_offset;
    const uint32_t tail_bytes = rd_u32(enc + 8);
    if (tail_bytes > 5u * nt) {
      if (lane == 0) set_status(status, BP_ERR_CORRUPT);
      continue;
    }
    for (uint32_t j = lane; j < tail_bytes; j += 32) s_bytes[w][j] = enc[e + j];
    __syncwarp();
    if (lane == 0) {
      uint32_t prev = np ? sc.lastval[li] : 0u, p = 0;
      uint64_t acc = 0;
      bool ok = true;
      for (uint32_t i = 0; i < nt && ok; i++) {
        uint32_t v = 0, shift = 0;
        for (;;) {
          if (p >= tail_bytes || shift > 28) {
            ok = false;
            break;
          }
          const uint32_t byte = s_bytes[w][p++];
          v |= (byte & 127u) << shift;
          shift += 7;
          if (byte & 128u) break;
        }
        prev += v;
        if (SUM) acc += prev;
        else out[L.out_offset + np + i] = prev;
      }
      if (!ok || p != tail_bytes) set_status(status, BP_ERR_CORRUPT);
      else if (SUM) atomicAdd(reinterpret_cast<unsigned long long *>(sums + li), acc);
    }
    __syncwarp();
  }
}

template <class K>
int resident_grid(K kernel, int threads, int &per_sm_cache) {
  if (per_sm_cache < 0) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, threads, 0) != cudaSuccess ||
        nb < 1)
      nb = 1;
    per_sm_cache = nb;
  }
  return per_sm_cache * device_sm_count();
}

}  // namespace

size_t pl_scratch_bytes(uint64_t total_units, uint32_t count) {
  return pl_layout(total_units, count).total;
}

int launch_pl_decode(const uint8_t *data, const ListSrc &src, uint64_t total_units,
                     uint32_t *out, uint64_t out_cap, uint64_t *sums, void *scratch,
                     size_t scratch_bytes, uint32_t *status, cudaStream_t s) {
  if (total_units == 0 || src.count == 0) return BP_OK;
  const uint64_t S = max_segs(total_units, src.count), G = max_groups(total_units, src.count);
  if (S >= 0xFFFFFFFFull || G >= 0xFFFFFFFFull) return BP_ERR_ARG;
  if (!scratch || scratch_bytes < pl_scratch_bytes(total_units, src.count)) return BP_ERR_SCRATCH;
  const PlLayout L = pl_layout(total_units, src.count);
  const PlScratch sc = carve(scratch, L);
  const uint64_t nch = (total_units + kChunk - 1) / kChunk;
  const uint64_t ntl = (nch + kTileChunks - 1) / kTileChunks;
  const int sms = device_sm_count();
  const int lgrid = (int)std::min<uint64_t>((src.count + 7) / 8, 4096);
  uint32_t spin_limit = 0, withhold = 0;
  lookback_limits(spin_limit, withhold);
  if (cudaMemsetAsync(sc.boffw, 0xFF, 8 * total_units, s) != cudaSuccess) return BP_ERR_CUDA;
  // tickets and look-back flags of both pl_tiles instances
  const size_t op_clear = (size_t)(reinterpret_cast<uint8_t *>(sc.op_flag) -
                                   reinterpret_cast<uint8_t *>(sc.op_ticket)) + 8 * ntl;
  if (cudaMemsetAsync(sc.op_ticket, 0, op_clear, s) != cudaSuccess) return BP_ERR_CUDA;
  pl_plan<<<1, 1024, 0, s>>>(data, src, total_units, S, G, sc, status);
  pl_parse<<<8 * sms, kThreads, 0, s>>>(data, src, sc);
  pl_resolve<<<(int)std::min<uint64_t>(src.count, 4ull * sms), kThreads, 0, s>>>(data, src, sc,
                                                                                   status);
  pl_emit<<<8 * sms, kThreads, 0, s>>>(data, src, sc, status);
  pl_leftover<<<lgrid, kThreads, 0, s>>>(data, src, sc, out_cap, sums != nullptr, status);
  // persistent grids of resident CTAs; tiles are taken in ticket order
  static int occ[8] = {-1, -1, -1, -1, -1, -1, -1, -1};
  auto grid = [&](int resident) {
    return (int)std::max<uint64_t>(1, std::min<uint64_t>(ntl, (uint64_t)resident));
  };
  // D4 lists, then the other kinds; of each pair of stage sizes the one
  // pl_plan did not choose leaves at once
  auto tiles = [&](auto kernel, int &cache) {
    kernel<<<grid(resident_grid(kernel, kTileThreads, cache)), kTileThreads, 0, s>>>(
        data, src, total_units, out, sums, sc, spin_limit, status);
  };
  if (sums) {
    tiles(pl_tiles<kSum, false, kStageBytes>, occ[0]);
    tiles(pl_tiles<kSum, false, kStageWide>, occ[1]);
    tiles(pl_tiles<kSum, true, kStageBytes>, occ[2]);
    tiles(pl_tiles<kSum, true, kStageWide>, occ[3]);
    pl_tail<true><<<lgrid, kThreads, 0, s>>>(data, src, out, sums, sc, status);
  } else {
    tiles(pl_tiles<kStore, false, kStageBytes>, occ[4]);
    tiles(pl_tiles<kStore, false, kStageWide>, occ[5]);
    tiles(pl_tiles<kStore, true, kStageBytes>, occ[6]);
    tiles(pl_tiles<kStore, true, kStageWide>, occ[7]);
    pl_tail<false><<<lgrid, kThreads, 0, s>>>(data, src, out, sums, sc, status);
  }
  return cudaPeekAtLastError() == cudaSuccess ? BP_OK : BP_ERR_CUDA;
}

}  // namespace bp
