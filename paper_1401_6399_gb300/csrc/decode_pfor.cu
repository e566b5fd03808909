// decode_pfor.cu -- decoding of S4-FastPFOR streams in the GPU layout (GP):
// bp_decode, bp_decode_sum and bp_decode_batch with BP_LAYOUT_PFOR.
//
// Section 4.4: a block is unpacked at its width b', the exceptions are
// patched with their high bits, and only then does the prefix of Section 5
// run (patching sits between the two, so unpacking and prefix cannot be
// fused as for S4-BP128; the paper makes the same observation).  Work unit:
// one page of 32 blocks per warp, as for GL; the page (low bits, exception
// positions and high bits, contiguous and 16-byte aligned) is staged in
// shared memory by one bulk copy when it fits.
#include "decode.h"
#include "bulk.cuh"
#include "gl_block.cuh"

namespace bp {

namespace {

constexpr int kThreads = 256;
constexpr int kMinBlocks = 3;
constexpr uint32_t kStageBytes = 4096;

struct GpView {
  uint32_t n, nblocks, npages, pw, kind;
  const uint32_t *first;
  const uint32_t *spo;
  const uint32_t *meta;  // {b', b - b', c, 0} per block
  const uint32_t *payload;
};

__device__ __forceinline__ bool gp_view(const uint8_t *enc, uint64_t enc_bytes, GpView &v) {
  if (enc_bytes < bp_fmt::kGlHeader || (reinterpret_cast<uintptr_t>(enc) & 15u) != 0) return false;
  const uint4 *h4 = reinterpret_cast<const uint4 *>(enc);
  const uint4 a = __ldg(h4 + 0), b = __ldg(h4 + 1), c = __ldg(h4 + 2), d = __ldg(h4 + 3);
  if (a.x != bp_fmt::kGpMagic || a.y != 3u) return false;
  const bp_fmt::GpGeometry g = bp_fmt::gp_geometry(a.z);
  const uint64_t total = (uint64_t)c.z | ((uint64_t)c.w << 32);
  if (a.w != g.nblocks || b.x != g.npages || b.z != g.off_first || b.w != g.off_spo ||
      c.x != g.off_meta || c.y != g.off_payload || total != g.off_payload + 4ull * b.y ||
      total > enc_bytes || d.x > 3u)
    return false;
  v.n = a.z;
  v.nblocks = a.w;
  v.npages = b.x;
  v.pw = b.y;
  v.kind = d.x;
  v.first = reinterpret_cast<const uint32_t *>(enc + g.off_first);
  v.spo = reinterpret_cast<const uint32_t *>(enc + g.off_spo);
  v.meta = reinterpret_cast<const uint32_t *>(enc + g.off_meta);
  v.payload = reinterpret_cast<const uint32_t *>(enc + g.off_payload);
  return true;
}

// A page's words and bytes, staged in shared memory or read from global.
struct StagedPage {
  uint32_t sbase;
  __device__ __forceinline__ SharedWords words(uint32_t w) const {
    return SharedWords{sbase + 4u * w};
  }
  __device__ __forceinline__ uint32_t word(uint32_t w) const { return words(w)(0); }
  __device__ __forceinline__ uint32_t byte(uint32_t i) const {
    uint32_t v;
    asm volatile("ld.shared.u8 %0, [%1];" : "=r"(v) : "r"(sbase + i));
    return v;
  }
};
struct GlobalPage {
  const uint32_t *p;
  __device__ __forceinline__ GlobalWords words(uint32_t w) const { return GlobalWords{p + w}; }
  __device__ __forceinline__ uint32_t word(uint32_t w) const { return __ldg(p + w); }
  __device__ __forceinline__ uint32_t byte(uint32_t i) const {
    return __ldg(reinterpret_cast<const uint8_t *>(p) + i);
  }
};

template <class W>
__device__ __forceinline__ void unpack_block(int b, const W &ld, int lane, uint32_t d[4]) {
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

template <bool SUM>
__device__ __forceinline__ void put_block(const uint32_t x[4], uint32_t cnt, int lane,
                                          uint32_t *__restrict__ o, uint64_t &acc) {
#pragma unroll
  for (int t = 0; t < 4; t++) {
    const uint32_t p = (uint32_t)gl_pos(lane, t);
    if (p < cnt) {
      if (SUM) acc += x[t];
      else o[p] = x[t];
    }
  }
}

// Page layout, per lane j (block 32q + j): its meta entry and the exclusive
// sums over the page's earlier blocks of low words, exceptions and high bits.
struct PageInfo {
  uint32_t bp, w, c, F;
  uint32_t woff, poff, hoff;       // this lane's block
  uint32_t nblk, pos_w, high_w;    // page: blocks, word of positions, of high bits
  uint32_t words;                  // page words
};

// false (and BP_ERR_CORRUPT recorded) if the page's meta data is inconsistent.
__device__ __forceinline__ bool gp_page(const GpView &v, uint32_t q, int lane, PageInfo &pi,
                                        uint32_t *status) {
  const uint32_t k0 = 32u * q;
  pi.nblk = min(32u, v.nblocks - k0);
  const bool mine = (uint32_t)lane < pi.nblk;
  const uint32_t m = mine ? __ldg(v.meta + k0 + lane) : 0u;
  pi.bp = m & 0xFFu;
  pi.w = (m >> 8) & 0xFFu;
  pi.c = (m >> 16) & 0xFFu;
  pi.F = mine ? __ldg(v.first + k0 + lane) : 0u;
  const bool bad = mine && (pi.bp + pi.w > 32u || (pi.w == 0u) != (pi.c == 0u) || pi.c > 128u);
  uint32_t a = 4u * pi.bp, e = pi.c, h = pi.c * pi.w;
#pragma unroll
  for (int dd = 1; dd < 32; dd <<= 1) {
    const uint32_t ta = __shfl_up_sync(kFull, a, dd), te = __shfl_up_sync(kFull, e, dd),
                   th = __shfl_up_sync(kFull, h, dd);
    if (lane >= dd) {
      a += ta;
      e += te;
      h += th;
    }
  }
  pi.woff = a - 4u * pi.bp;
  pi.poff = e - pi.c;
  pi.hoff = h - pi.c * pi.w;
  const uint32_t low = __shfl_sync(kFull, a, 31), ne = __shfl_sync(kFull, e, 31),
                 hb = __shfl_sync(kFull, h, 31);
  pi.pos_w = low;
  pi.high_w = low + (ne + 3u) / 4u;
  pi.words = (pi.high_w + (hb + 31u) / 32u + 3u) & ~3u;
  const uint32_t p0 = __ldg(v.spo + q), p1 = __ldg(v.spo + q + 1);
  if (__any_sync(kFull, bad) || p1 < p0 || p1 - p0 != pi.words || p1 > v.pw) {
    if (lane == 0) set_status(status, BP_ERR_CORRUPT);
    return false;
  }
  return true;
}

// Slot of block position p in a per-warp patch array: lane l's four
// positions 16c + 4t + s (l = 8s + c) sit at 32t + l, so the lanes' reads
// of one t fall in 32 different banks.
__device__ __forceinline__ uint32_t patch_slot(uint32_t p) {
  return 32u * ((p >> 2) & 3u) + 8u * (p & 3u) + (p >> 4);
}

// The blocks of one page.  Exceptions are patched through a per-warp
// array of 128 patch words in shared memory, zero between blocks: the lanes
// that take an exception (one each) write its high bits, shifted to above
// the low b' bits, at its position's slot; every lane ORs in the words of its
// four positions; the exception lanes zero their words again.
template <bool SUM, int KIND, class P>
__device__ __forceinline__ void gp_decode_page(const GpView &v, const PageInfo &pi, uint32_t q,
                                               const P &pg, uint32_t *s_patch, int lane,
                                               uint32_t *__restrict__ out, uint64_t &acc,
                                               uint32_t *status) {
  for (uint32_t j = 0; j < pi.nblk; j++) {
    const int bp = (int)__shfl_sync(kFull, pi.bp, j);
    const uint32_t F = __shfl_sync(kFull, pi.F, j);
    const uint32_t woff = __shfl_sync(kFull, pi.woff, j);
    const uint32_t c = __shfl_sync(kFull, pi.c, j);
    const uint32_t blk = q * 32u + j;
    uint32_t d[4];
    unpack_block(bp, pg.words(woff), lane, d);
    if (c) {
      const uint32_t w = __shfl_sync(kFull, pi.w, j);
      const uint32_t poff = __shfl_sync(kFull, pi.poff, j);
      const uint32_t hoff = __shfl_sync(kFull, pi.hoff, j);
      for (uint32_t e0 = 0; e0 < c; e0 += 32) {
        const uint32_t e = e0 + lane;
        uint32_t p = 128u;
        if (e < c) {
          p = pg.byte(4u * pi.pos_w + poff + e);
          const uint32_t bit = hoff + e * w;
          const uint32_t k = pi.high_w + (bit >> 5), o = bit & 31u;
          uint64_t hv = pg.word(k) >> o;
          if (o + w > 32u) hv |= (uint64_t)pg.word(k + 1) << (32u - o);
          const uint32_t high = (uint32_t)hv & (w >= 32u ? 0xFFFFFFFFu : (1u << w) - 1u);
          if (p < 128u) s_patch[patch_slot(p)] = high << bp;  // bp < 32 here
          else set_status(status, BP_ERR_CORRUPT);
        }
        __syncwarp();
#pragma unroll
        for (int t = 0; t < 4; t++) d[t] |= s_patch[32 * t + lane];
        __syncwarp();
        if (p < 128u) s_patch[patch_slot(p)] = 0u;
        __syncwarp();
      }
    }
    uint32_t x[4], ctot;
    prefix_block<KIND>(d, F, lane, x, ctot);
    const uint32_t cnt = min(128u, v.n - 128u * blk);
    if (!SUM && cnt == 128u) {
#pragma unroll
      for (int t = 0; t < 4; t++) out[128ull * blk + gl_pos(lane, t)] = x[t];
    } else {
      put_block<SUM>(x, cnt, lane, out + 128ull * blk, acc);
    }
  }
}

// The page with the list's kind of differential coding (one dispatch per
// page, not per block).
template <bool SUM, class P>
__device__ __forceinline__ void gp_decode_page_kind(const GpView &v, const PageInfo &pi,
                                                    uint32_t q, const P &pg, uint32_t *s_patch,
                                                    int lane, uint32_t *__restrict__ out,
                                                    uint64_t &acc, uint32_t *status) {
  switch (v.kind) {
    case kD4: gp_decode_page<SUM, kD4>(v, pi, q, pg, s_patch, lane, out, acc, status); break;
    case kDM: gp_decode_page<SUM, kDM>(v, pi, q, pg, s_patch, lane, out, acc, status); break;
    case kD2: gp_decode_page<SUM, kD2>(v, pi, q, pg, s_patch, lane, out, acc, status); break;
    default: gp_decode_page<SUM, kD1>(v, pi, q, pg, s_patch, lane, out, acc, status); break;
  }
}

__device__ __forceinline__ void flush_sum(uint64_t &acc, uint64_t *dst, int lane) {
#pragma unroll
  for (int dd = 16; dd > 0; dd >>= 1) acc += __shfl_down_sync(kFull, acc, dd);
  if (lane == 0 && acc)
    atomicAdd(reinterpret_cast<unsigned long long *>(dst), (unsigned long long)acc);
  acc = 0;
}

// Persistent grid over the pages of all lists (unit u belongs to the list
// with the largest unit_base <= u), as the GL decoder.
template <bool SUM>
__global__ void __launch_bounds__(kThreads, kMinBlocks)
    gp_decode_kernel(const uint8_t *__restrict__ data, ListSrc src, uint64_t total_units,
                     uint32_t *__restrict__ out, uint64_t out_cap, uint64_t *sums,
                     uint32_t *status) {
  const int lane = threadIdx.x & 31;
  const uint64_t warp = (blockIdx.x * (uint64_t)kThreads + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * kThreads) >> 5;
  __shared__ __align__(128) uint8_t s_stage[kThreads / 32][kStageBytes];
  __shared__ uint32_t s_patch[kThreads / 32][128];
  __shared__ __align__(8) uint64_t s_bar[kThreads / 32];
  const int wl = threadIdx.x >> 5;
  const uint32_t bar = smem_addr(&s_bar[wl]);
  const uint32_t sbase = smem_addr(&s_stage[wl][0]);
  uint32_t phase = 0;
  if (lane == 0) bulk_bar_init(bar);
  for (int i = lane; i < 128; i += 32) s_patch[wl][i] = 0u;
  __syncwarp();
  uint32_t cur = 0xFFFFFFFFu;
  bool ok = false;
  GpView v;
  uint64_t base = 0, out_off = 0, acc = 0;
  for (uint64_t u = warp; u < total_units; u += nwarps) {
    const uint32_t li = src.find(u);
    if (li != cur) {
      if (SUM && cur != 0xFFFFFFFFu) flush_sum(acc, sums + cur, lane);
      cur = li;
      const bp_list L = src.get(li);
      base = L.unit_base;
      out_off = L.out_offset;
      ok = gp_view(data + L.enc_offset, L.enc_bytes, v) && v.n == L.n;
      if (!ok) {
        if (lane == 0) set_status(status, BP_ERR_CORRUPT);
      } else if (!SUM && L.out_offset + L.n > out_cap) {
        ok = false;
        if (lane == 0) set_status(status, BP_ERR_CAPACITY);
      }
    }
    if (!ok) continue;
    const uint64_t q = u - base;
    if (q >= v.npages) continue;
    PageInfo pi;
    if (!gp_page(v, (uint32_t)q, lane, pi, status)) continue;
    const uint32_t p0 = __ldg(v.spo + q);
    const uint32_t bytes = 4u * pi.words;
    if (bytes > 0 && bytes <= kStageBytes) {
      if (lane == 0) bulk_load(bar, sbase, v.payload + p0, bytes);
      const bool done = bulk_wait(bar, phase);
      phase ^= 1u;
      if (!__all_sync(kFull, done)) {  // give up: record it, let the copy land, stop
        if (lane == 0) set_status(status, BP_ERR_TIMEOUT);
        bulk_wait(bar, phase ^ 1u);
        return;
      }
      gp_decode_page_kind<SUM>(v, pi, (uint32_t)q, StagedPage{sbase}, s_patch[wl], lane,
                               out + out_off, acc, status);
      __syncwarp();
    } else {
      gp_decode_page_kind<SUM>(v, pi, (uint32_t)q, GlobalPage{v.payload + p0}, s_patch[wl],
                               lane, out + out_off, acc, status);
    }
  }
  if (SUM && cur != 0xFFFFFFFFu) flush_sum(acc, sums + cur, lane);
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

int launch_gp_decode(const uint8_t *data, const ListSrc &src, uint64_t total_units,
                     uint32_t *out, uint64_t out_cap, uint64_t *sums, uint32_t *status,
                     cudaStream_t s) {
  if (total_units == 0) return BP_OK;
  static int occ[2] = {-1, -1};
  if (sums) {
    const int grid = persistent_grid(gp_decode_kernel<true>, total_units, occ[0]);
    gp_decode_kernel<true><<<grid, kThreads, 0, s>>>(data, src, total_units, out, out_cap, sums,
                                                     status);
  } else {
    const int grid = persistent_grid(gp_decode_kernel<false>, total_units, occ[1]);
    gp_decode_kernel<false><<<grid, kThreads, 0, s>>>(data, src, total_units, out, out_cap,
                                                      sums, status);
  }
  return cudaPeekAtLastError() == cudaSuccess ? BP_OK : BP_ERR_CUDA;
}

}  // namespace bp
