// intersect.cu -- bp_intersect_pair: sorted intersection of two compressed
// lists (Section 6; the result is output-to-input safe in the paper's sense
// because each output value comes from the shorter list, in order).
//
//  fused (both GL): each warp decodes a run of up to 8 blocks of the
//      shorter list r into shared memory; candidate blocks of the longer
//      list f are located through f's skip headers and decoded into a
//      shared-memory window that moves forward with r's values (or probed
//      one by one for very skewed pairs); nothing decoded is written back
//      to HBM.
//  unfused (any layout): both lists are decoded into scratch, then the
//      decoded arrays are intersected by the same warp-level regimes.
// Output: ballot/popc inside warps, a CTA scan, and a decoupled look-back
// across CTAs, so the result is written once, sorted, in a single pass.
#include <mutex>

#include "decode.h"
#include "intersect.cuh"
#include "tuning.h"

namespace bp {

namespace {

struct PairArgs {
  const uint8_t *r_enc;
  uint64_t r_bytes;
  uint32_t nr;
  const uint8_t *f_enc;
  uint64_t f_bytes;
  uint32_t nf;
};

// Shared memory per warp: up to 8 decoded blocks of r (survivors compacted
// in place), the window of f, and in the merge instance one hit bit per
// value of r (kept out of the other instance, whose 3 CTAs per SM then stay
// within the smaller shared-memory carveout).
constexpr int kPairGroups = 8;
constexpr int pair_warp_words(bool merge) {
  return kPairGroups * 128 + kIxDenseMax * 128 + (merge ? kPairGroups * 4 : 0);
}

// vpw: values of the shorter list per warp: a power of two 8..128 (a slice
// of one block, for very skewed pairs) or 128 g for g = 1..8 blocks.  A run
// whose value range covers at most merge_span blocks of f per block of r
// (similar densities) is merged with those blocks of f (merge_run_hits);
// otherwise the warp filters it 128 values at a time with its window of f
// moving forward (dense) or by per-value probes (sparse).  MERGE: the
// instance with the merge regime, launched when the tuning's merge_span is
// not 0 (the out-of-line merge call alone costs the kernel instructions
// where it is not taken).
template <bool MERGE>
__global__ void __launch_bounds__(kIxThreads, 3)
    fused_pair_kernel(PairArgs a, Compaction cp, TileOut to, uint32_t ntiles, uint32_t dense_max,
                      uint32_t vpw, uint32_t merge_span) {
  extern __shared__ uint32_t smem[];
  __shared__ uint32_t s_wcnt[kIxWarps], s_base[1], s_tile;
  if (threadIdx.x == 0) s_tile = atomicAdd(cp.ticket, 1u);
  __syncthreads();
  const uint32_t t = s_tile;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t *s_r = smem + w * pair_warp_words(MERGE);
  uint32_t *s_f = s_r + kPairGroups * 128;
  uint32_t *s_hit = s_f + kIxDenseMax * 128;  // MERGE only

  GlView R, F;
  bool okR = gl_view(a.r_enc, a.r_bytes, R) && R.n == a.nr;
  bool okF = gl_view(a.f_enc, a.f_bytes, F) && F.n == a.nf;
  if ((!okR || !okF) && threadIdx.x == 0 && t == 0) set_status(to.status, BP_ERR_CORRUPT);
  if (okR && okF && (R.kind != 0u || F.kind != 0u)) {  // the probes need D4 columns
    if (threadIdx.x == 0 && t == 0) set_status(to.status, BP_ERR_ARG);
    okR = okF = false;
  }

  uint32_t scount = 0;
  const uint64_t p0 = ((uint64_t)t * kIxWarps + w) * vpw;  // first r position of this warp
  if (okR && okF && p0 < a.nr) {
    const uint64_t p1 = min((uint64_t)a.nr, p0 + vpw);       // one past the last
    const uint32_t kb0 = (uint32_t)(p0 >> 7), ng = (uint32_t)(((p1 - 1) >> 7) - kb0 + 1);
    // bit 4g+j of `alive`: value 32j + lane of block kb0+g is in the range
    uint32_t alive = 0, na = 0;
    for (uint32_t g = 0; g < ng; g++) {
      const uint32_t cnt = gl_block_into(R, kb0 + g, s_r + 128u * g, lane, to.status);
      const uint64_t bstart = 128ull * (kb0 + g);
      na = 128u * g + cnt;  // every block but r's last is full
#pragma unroll
      for (int j = 0; j < 4; j++) {
        const uint64_t pos = bstart + 32 * j + lane;
        if (pos >= p0 && pos < p1 && (uint32_t)(32 * j + lane) < cnt) alive |= 1u << (4 * g + j);
      }
    }
    __syncwarp();
    bool merged = false;
    if (MERGE && merge_span != 0u && na > 0u && F.nblocks > 0u) {
      const int64_t kl = warp_ubound(F.first, F.nblocks, s_r[na - 1], lane);
      if (kl < 0) {  // the whole run is below f's first value
        alive = 0;
        merged = true;
      } else {
        const int64_t kf = warp_ubound(F.first, F.nblocks, s_r[0], lane);
        if ((uint64_t)(kl - imax64(kf, 0) + 1) <= (uint64_t)merge_span * ng) {
          s_hit[lane] = 0u;
          __syncwarp();
          merge_run_hits(F, s_r, na, kf, kl, s_f, s_hit, lane, to.status);
          alive = alive_and_hits(alive, ng, s_hit, lane);
          __syncwarp();
          merged = true;
        }
      }
    }
    FWin win = fwin_empty();
    for (uint32_t g = 0; g < ng && !merged; g++) {
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
      gl_membership_win(F, v, valid, hit, lo, hi, s_f, win, lane, dense_max, to.status);
#pragma unroll
      for (int j = 0; j < 4; j++)
        if (valid[j] && !hit[j]) alive &= ~(1u << (4 * g + j));
    }
    scount = compact_alive(s_r, ng, alive, lane);  // the survivors, in order
  }
  tile_emit_buf(s_r, scount, t, t == ntiles - 1, cp, to, s_wcnt, s_base);
}

__global__ void __launch_bounds__(kIxThreads)
    sorted_pair_kernel(const uint32_t *__restrict__ r, uint32_t nr, const uint32_t *__restrict__ f,
                       uint32_t nf, Compaction cp, TileOut to, uint32_t ntiles, uint32_t dense_max) {
  __shared__ uint32_t s_f[kIxWarps][kIxDenseMax * 128];
  __shared__ uint32_t s_wcnt[kIxWarps], s_base[1], s_tile;
  if (threadIdx.x == 0) s_tile = atomicAdd(cp.ticket, 1u);
  __syncthreads();
  const uint32_t t = s_tile;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
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

inline size_t up256(size_t v) { return (v + 255) & ~(size_t)255; }

uint32_t pair_tiles(uint64_t nr, uint32_t vpw = 128) {
  const uint64_t chunks = (nr + vpw - 1) / vpw;
  return (uint32_t)std::max<uint64_t>(1, (chunks + kIxWarps - 1) / kIxWarps);
}

// Values of the shorter list per warp.  Very skewed pairs (every value
// probes a block of its own, ratio >= 128) with too few values to fill the
// GPU: down to 8 (more warps, fewer probes each).  Otherwise runs of g <= 8
// blocks per warp: among the g that keep at least 16 warps per SM busy, the
// one whose CTAs fill the `resident` CTA slots most evenly (the last wave
// least empty; the larger g on a tie), else g = 1 (slices of a block measured
// slower here: for m = 2^18 against 2^22, 61 us with whole blocks, 76 us
// with 64 values per warp, 120 us with 8).
uint32_t pair_vpw(uint64_t nr, uint64_t nf, uint64_t resident) {
  if (nr == 0) return 128;
  if (nf >= 128 * nr) {
    const uint64_t want_warps = 16ull * device_sm_count() * 8;
    uint32_t vpw = 128;
    while (vpw > 8 && (nr + vpw - 1) / vpw < want_warps) vpw >>= 1;
    return vpw;
  }
  const uint64_t want_warps = 16ull * device_sm_count();
  uint32_t best = 1;
  double best_fill = -1.0;
  for (uint32_t g = kPairGroups; g >= 1; g--) {
    const uint64_t warps = (nr + 128ull * g - 1) / (128ull * g);
    if (warps < want_warps) continue;
    const uint64_t tiles = (warps + kIxWarps - 1) / kIxWarps;
    const uint64_t waves = (tiles + resident - 1) / resident;
    const double fill = (double)tiles / (double)(waves * resident);
    if (fill > best_fill + 1e-9) {
      best_fill = fill;
      best = g;
    }
  }
  return 128u * best;
}

// Per device (bit d: device d): the kernel's shared-memory limit was raised
// and its resident CTAs per SM are in g_pair_per_sm[d].
std::mutex g_pair_mu;
uint64_t g_pair_smem_set = 0;
int g_pair_per_sm[64];
constexpr size_t pair_smem(bool merge) { return sizeof(uint32_t) * pair_warp_words(merge) * kIxWarps; }

}  // namespace

size_t intersect_scratch_bytes(size_t na, size_t nb, int layout, int mode) {
  const size_t nr = std::min(na, nb), nf = std::max(na, nb);
  const size_t comp = up256(compaction_bytes(pair_tiles(nr, 8)));
  if (mode == BP_MODE_FUSED) return comp;
  size_t dec = 0;
  if (layout == BP_LAYOUT_PAPER) dec = up256(pl_scratch_bytes(bp_fmt::units_of(nf, 0), 1));
  return comp + up256(4 * nr + 16) + up256(4 * nf + 16) + dec;
}

int launch_intersect_pair(const uint8_t *da, size_t a_bytes, size_t na, const uint8_t *db,
                          size_t b_bytes, size_t nb, int layout, int mode, uint32_t *out,
                          size_t out_cap, uint32_t *count, void *scratch, size_t scratch_bytes,
                          uint32_t *status, cudaStream_t s) {
  const bool swap = nb < na;
  PairArgs a;
  a.r_enc = swap ? db : da;
  a.r_bytes = swap ? b_bytes : a_bytes;
  a.nr = (uint32_t)(swap ? nb : na);
  a.f_enc = swap ? da : db;
  a.f_bytes = swap ? a_bytes : b_bytes;
  a.nf = (uint32_t)(swap ? na : nb);
  uint8_t *sp = static_cast<uint8_t *>(scratch);
  const Compaction cp = compaction_at(sp);
  TileOut to{out, out_cap, count, status};
  const Tuning &tu = tuning();
  if (mode == BP_MODE_FUSED) {
    int dev = 0, per_sm = 1;  // resident CTAs of fused_pair_kernel per SM
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return BP_ERR_CUDA;
    auto *const kern = tu.merge_span ? fused_pair_kernel<true> : fused_pair_kernel<false>;
    {
      std::lock_guard<std::mutex> g(g_pair_mu);
      if (!((g_pair_smem_set >> dev) & 1u)) {
        if (cudaFuncSetAttribute(fused_pair_kernel<false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)pair_smem(false)) != cudaSuccess ||
            cudaFuncSetAttribute(fused_pair_kernel<true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)pair_smem(true)) != cudaSuccess)
          return BP_ERR_CUDA;
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fused_pair_kernel<false>,
                                                          kIxThreads, pair_smem(false)) !=
                cudaSuccess ||
            n < 1)
          n = 1;
        g_pair_per_sm[dev] = n;
        g_pair_smem_set |= 1ull << dev;
      }
      per_sm = g_pair_per_sm[dev];
    }
    const uint32_t vpw = pair_vpw(a.nr, a.nf, (uint64_t)per_sm * device_sm_count());
    const uint32_t ft = pair_tiles(a.nr, vpw);
    if (cudaMemsetAsync(sp, 0, compaction_bytes(ft), s) != cudaSuccess) return BP_ERR_CUDA;
    kern<<<ft, kIxThreads, pair_smem(tu.merge_span != 0u), s>>>(a, cp, to, ft,
                                           std::min<uint32_t>(tu.dense_blocks, kIxDenseMax), vpw,
                                           tu.merge_span);
    return cudaPeekAtLastError() == cudaSuccess ? BP_OK : BP_ERR_CUDA;
  }
  // unfused: decode both lists into scratch, then intersect the arrays
  const uint32_t ntiles = pair_tiles(a.nr);
  if (cudaMemsetAsync(sp, 0, compaction_bytes(ntiles), s) != cudaSuccess) return BP_ERR_CUDA;
  size_t off = up256(compaction_bytes(pair_tiles(a.nr, 8)));
  uint32_t *dr = reinterpret_cast<uint32_t *>(sp + off);
  off += up256(4ull * a.nr + 16);
  uint32_t *df = reinterpret_cast<uint32_t *>(sp + off);
  off += up256(4ull * a.nf + 16);
  void *dsc = sp + off;
  const size_t dsc_bytes = scratch_bytes - off;
  int rc;
  for (int which = 0; which < 2; which++) {
    const uint8_t *enc = which ? a.f_enc : a.r_enc;
    const uint64_t bytes = which ? a.f_bytes : a.r_bytes;
    const uint32_t n = which ? a.nf : a.nr;
    uint32_t *dst = which ? df : dr;
    const ListSrc src = single_list(bytes, n, layout);
    const uint64_t units = bp_fmt::units_of(n, layout);
    rc = layout == BP_LAYOUT_GPU
             ? launch_gl_decode(enc, src, units, dst, n, nullptr, status, s)
             : launch_pl_decode(enc, src, units, dst, n, nullptr, dsc, dsc_bytes, status, s);
    if (rc != BP_OK) return rc;
  }
  sorted_pair_kernel<<<ntiles, kIxThreads, 0, s>>>(dr, a.nr, df, a.nf, cp, to, ntiles,
                                                   std::min<uint32_t>(tu.dense_blocks, kIxDenseMax));
  return cudaPeekAtLastError() == cudaSuccess ? BP_OK : BP_ERR_CUDA;
}

}  // namespace bp
