// intersect.cu -- bp_intersect_pair: sorted intersection of two compressed
// lists (Section 6; the result is output-to-input safe in the paper's sense
// because each output value comes from the shorter list, in order).
//
//  fused (both GL): the shorter list r is decoded block by block in
//      registers; candidate blocks of the longer list f are located through
//      f's skip headers and decoded into shared memory only where needed;
//      nothing decoded is written back to HBM.
//  unfused (any layout): both lists are decoded into scratch, then the
//      decoded arrays are intersected by the same warp-level regimes.
// Output: ballot/popc inside warps, a CTA scan, and a decoupled look-back
// across CTAs, so the result is written once, sorted, in a single pass.
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

// vpw: values of the shorter list per warp (8..128, a power of two).  Warps
// that share an r block each decode it and take their slice.
__global__ void __launch_bounds__(kIxThreads)
    fused_pair_kernel(PairArgs a, Compaction cp, TileOut to, uint32_t ntiles, uint32_t dense_max,
                      uint32_t vpw) {
  __shared__ uint32_t s_r[kIxWarps][128];
  __shared__ uint32_t s_f[kIxWarps][kIxDenseMax * 128];
  __shared__ uint32_t s_wcnt[kIxWarps], s_base[1], s_tile;
  if (threadIdx.x == 0) s_tile = atomicAdd(cp.ticket, 1u);
  __syncthreads();
  const uint32_t t = s_tile;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;

  GlView R, F;
  const bool okR = gl_view(a.r_enc, a.r_bytes, R) && R.n == a.nr;
  const bool okF = gl_view(a.f_enc, a.f_bytes, F) && F.n == a.nf;
  if ((!okR || !okF) && threadIdx.x == 0 && t == 0) set_status(to.status, BP_ERR_CORRUPT);

  uint32_t v[4] = {0, 0, 0, 0};
  bool valid[4] = {false, false, false, false}, hit[4] = {false, false, false, false};
  const uint64_t p0 = ((uint64_t)t * kIxWarps + w) * vpw;  // first r position of this warp
  if (okR && okF && p0 < a.nr) {
    const uint32_t kb = (uint32_t)(p0 >> 7), s0 = (uint32_t)(p0 & 127u);
    const uint32_t cnt = gl_block_into(R, kb, s_r[w], lane, to.status);
    __syncwarp();
    const uint32_t end = min(cnt, s0 + vpw);
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const uint32_t pos = s0 + 32u * k + lane;
      valid[k] = pos < end;
      v[k] = valid[k] ? s_r[w][pos] : 0u;
    }
    if (end > s0)
      gl_membership(F, v, valid, hit, s_r[w][s0], s_r[w][end - 1], s_f[w], lane, dense_max,
                    to.status);
  }
  tile_emit(v, hit, t, t == ntiles - 1, cp, to, s_wcnt, s_base);
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

// Values of the shorter list per warp: 128, unless the lists are so skewed
// that every value probes a block of its own (ratio >= 128) and there are
// too few values to fill the GPU -- then down to 8 (more warps, fewer
// probes each).
uint32_t pair_vpw(uint64_t nr, uint64_t nf) {
  if (nr == 0 || nf < 128 * nr) return 128;
  const uint64_t want_warps = 16ull * device_sm_count() * 8;
  uint32_t vpw = 128;
  while (vpw > 8 && (nr + vpw - 1) / vpw < want_warps) vpw >>= 1;
  return vpw;
}

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
    const uint32_t vpw = pair_vpw(a.nr, a.nf);
    const uint32_t ft = pair_tiles(a.nr, vpw);
    if (cudaMemsetAsync(sp, 0, compaction_bytes(ft), s) != cudaSuccess) return BP_ERR_CUDA;
    fused_pair_kernel<<<ft, kIxThreads, 0, s>>>(
        a, cp, to, ft, std::min<uint32_t>(tu.dense_blocks, kIxDenseMax), vpw);
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
