// decode_pl.cu -- decoding of the paper's S4-BP128-D4 layout (PL).
//
// Three launches per call (all lists of a batch at once):
//  1. pl_walk: one warp per list follows the meta-block chain (Section 4.3:
//     16 width bytes, then 16 blocks of 16b bytes each; then leftover blocks
//     with one width byte each) and records every block's byte offset and
//     width.  Work unit u of a list: its block u - unit_base, and one last
//     unit for the varint tail.
//  2. pl_decode: tiles of 32 units; each warp unpacks 4 blocks (Algorithm 1,
//     4-lane interleave), the D4 seed of every block -- the column sums of
//     all earlier blocks of its list, starting from (0,0,0,0) (Section 5) --
//     comes from a segmented scan inside the tile and a decoupled look-back
//     over earlier tiles, then the values are stored (or summed).
//  3. pl_tail: one warp per list decodes the fewer than 128 final integers
//     (varint of D1 gaps, Section 4.1) after the last packed value.
#include "decode.h"
#include "pl_block.cuh"

namespace bp {

namespace {

constexpr int kThreads = 256;
constexpr int kTileUnits = 32;  // 8 warps x 4 units
constexpr uint64_t kOffMask = (1ull << 56) - 1;
constexpr uint32_t kBadWidth = 0xFF;
constexpr uint32_t kSpinLimit = 1u << 22;

struct PlScratch {
  uint64_t *boffw;   // [units] byte offset | width << 56 (tail unit: tail offset)
  uint32_t *ticket;  // tile ticket counter (zeroed per call)
  uint32_t *flags;   // [ntiles] 0 none, 1|head<<2 aggregate, 2 inclusive (zeroed per call)
  uint4 *agg;        // [ntiles]
  uint4 *incl;       // [ntiles]
  uint32_t *lastval; // [count] last packed value of each list
};

__host__ __device__ inline size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

struct PlLayout {
  size_t boffw, ticket, flags, agg, incl, lastval, total;
};

__host__ __device__ inline PlLayout pl_layout(uint64_t units, uint32_t count) {
  const uint64_t ntiles = (units + kTileUnits - 1) / kTileUnits;
  PlLayout L;
  L.boffw = 0;
  L.ticket = align256(8 * units);
  L.flags = L.ticket + 16;  // ticket and flags are cleared together
  L.agg = align256(L.flags + 4 * ntiles);
  L.incl = L.agg + 16 * ntiles;
  L.lastval = align256(L.incl + 16 * ntiles);
  L.total = align256(L.lastval + 4 * (size_t)count);
  return L;
}

__device__ __forceinline__ uint32_t rd_u32(const uint8_t *p) {
  return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}

// ---- 1. meta-block walk -------------------------------------------------------

__global__ void __launch_bounds__(kThreads)
    pl_walk_kernel(const uint8_t *__restrict__ data, ListSrc src, PlScratch sc,
                   uint64_t out_cap, bool sum, uint32_t *status) {
  const int lane = threadIdx.x & 31;
  const uint32_t warp = (blockIdx.x * kThreads + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * kThreads) >> 5;
  for (uint32_t li = warp; li < src.count; li += nwarps) {
    const bp_list L = src.get(li);
    const uint8_t *enc = data + L.enc_offset;
    const uint64_t bytes = L.enc_bytes;
    const uint64_t U0 = L.unit_base;
    const uint32_t nb = L.n / 128u, meta = nb / 16u;
    if (!sum && L.out_offset + L.n > out_cap) {
      if (lane == 0) set_status(status, BP_ERR_CAPACITY);
      for (uint32_t j = lane; j <= nb; j += 32) sc.boffw[U0 + j] = (uint64_t)kBadWidth << 56;
      continue;
    }
    bool ok = bytes >= 16 && (L.enc_offset & 15u) == 0;
    uint32_t tail_bytes = 0;
    if (ok) {
      ok = rd_u32(enc) == L.n && rd_u32(enc + 4) == 0u && rd_u32(enc + 12) == 0u;
      tail_bytes = rd_u32(enc + 8);
    }
    uint64_t pos = 16;
    uint32_t k = 0;  // blocks recorded so far
    for (uint32_t m = 0; ok && m < meta; m++) {
      if (pos + 16 > bytes) {
        ok = false;
        break;
      }
      const uint32_t w = lane < 16 ? enc[pos + lane] : 0u;
      if (__any_sync(kFull, w > 32u)) {
        ok = false;
        break;
      }
      uint32_t incl = 16u * w;
#pragma unroll
      for (int dd = 1; dd < 16; dd <<= 1) {
        const uint32_t t = __shfl_up_sync(kFull, incl, dd);
        if (lane >= dd) incl += t;
      }
      const uint64_t next = pos + 16 + __shfl_sync(kFull, incl, 15);
      if (next > bytes) {  // the meta-block runs past the stream
        ok = false;
        break;
      }
      const uint64_t blk_off = pos + 16 + (incl - 16u * w);
      if (lane < 16) sc.boffw[U0 + k + lane] = blk_off | ((uint64_t)w << 56);
      pos = next;
      k += 16;
    }
    for (; ok && k < nb; k++) {
      if (pos + 1 > bytes) {
        ok = false;
        break;
      }
      const uint32_t w = enc[pos];
      if (w > 32u || pos + 1 + 16ull * w > bytes) {
        ok = false;
        break;
      }
      if (lane == 0) sc.boffw[U0 + k] = (pos + 1) | ((uint64_t)w << 56);
      pos += 1 + 16ull * w;
    }
    if (ok && pos + tail_bytes != bytes) ok = false;
    if (ok) {
      if (lane == 0) sc.boffw[U0 + nb] = pos;
    } else {
      if (lane == 0) set_status(status, BP_ERR_CORRUPT);
      for (uint32_t j = k + lane; j <= nb; j += 32) sc.boffw[U0 + j] = (uint64_t)kBadWidth << 56;
    }
  }
}

// ---- 2. decode with decoupled look-back ------------------------------------------

__device__ __forceinline__ uint32_t ld_flag(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_flag(uint32_t *p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ uint32_t comp(const uint4 &v, int s) {
  return s == 0 ? v.x : s == 1 ? v.y : s == 2 ? v.z : v.w;
}

template <bool SUM>
__global__ void __launch_bounds__(kThreads, 4)
    pl_decode_kernel(const uint8_t *__restrict__ data, ListSrc src, uint64_t total_units,
                     uint32_t *__restrict__ out, uint64_t *sums, PlScratch sc, uint32_t *status) {
  __shared__ uint32_t s_tile;
  __shared__ uint32_t s_wsum[8][4];  // warp aggregate per column
  __shared__ uint32_t s_whead[8];
  __shared__ uint4 s_E;

  if (threadIdx.x == 0) s_tile = atomicAdd(sc.ticket, 1u);
  __syncthreads();
  const uint64_t t = s_tile;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int s = lane >> 3, c = lane & 7;

  uint32_t xv[4][4];   // local running sums down the lane's 4 rows, per unit
  uint32_t cex[4];     // exclusive sum over lanes c' < c of the column, per unit
  uint32_t cs[4];      // column total of the block (own column), per unit
  bool head[4], isblk[4];
  uint32_t lst[4], kb[4];

#pragma unroll
  for (int i = 0; i < 4; i++) {
    const uint64_t u = t * kTileUnits + 4u * w + i;
    head[i] = false;
    isblk[i] = false;
    cs[i] = 0;
    cex[i] = 0;
    lst[i] = 0xFFFFFFFFu;
    kb[i] = 0;
#pragma unroll
    for (int j = 0; j < 4; j++) xv[i][j] = 0;
    if (u >= total_units) continue;
    const uint32_t li = src.find(u);
    const bp_list L = src.get(li);
    const uint64_t k = u - L.unit_base;
    const uint32_t nb = L.n / 128u;
    lst[i] = li;
    kb[i] = (uint32_t)k;
    head[i] = (k == 0);
    if (k >= nb) continue;
    const uint64_t e = sc.boffw[u];
    const uint32_t b = (uint32_t)(e >> 56);
    if (b > 32u) continue;  // list marked bad by the walk: nothing is stored
    isblk[i] = true;
    uint32_t d[4];
    pl_block_deltas((int)b, data + L.enc_offset + (e & kOffMask), lane, d);
    xv[i][0] = d[0];
    xv[i][1] = d[0] + d[1];
    xv[i][2] = xv[i][1] + d[2];
    xv[i][3] = xv[i][2] + d[3];
    uint32_t incl = xv[i][3];
#pragma unroll
    for (int dd = 1; dd < 8; dd <<= 1) {
      const uint32_t v = __shfl_up_sync(kFull, incl, dd, 8);
      if (c >= dd) incl += v;
    }
    cex[i] = incl - xv[i][3];
    cs[i] = __shfl_sync(kFull, incl, (lane & ~7) | 7);
  }

  // segmented scan of the 4 units inside the warp (heads restart at zero)
  uint32_t pw[4];  // exclusive within warp
  uint32_t r = 0;
  bool whead = false;
#pragma unroll
  for (int i = 0; i < 4; i++) {
    if (head[i]) {
      r = 0;
      whead = true;
    }
    pw[i] = r;
    r += cs[i];
  }
  if (c == 0) s_wsum[w][s] = r;
  if (lane == 0) s_whead[w] = whead ? 1u : 0u;
  __syncthreads();

  // exclusive within tile for this warp, and whether a head came before it
  uint32_t W = 0;
  bool head_before = false;
  for (int v = 0; v < w; v++) {
    if (s_whead[v]) {
      W = s_wsum[v][s];
      head_before = true;
    } else {
      W += s_wsum[v][s];
    }
  }

  if (threadIdx.x == 0) {
    uint4 tail = make_uint4(0, 0, 0, 0);
    bool th = false;
    for (int v = 0; v < 8; v++) {
      if (s_whead[v]) {
        tail = make_uint4(s_wsum[v][0], s_wsum[v][1], s_wsum[v][2], s_wsum[v][3]);
        th = true;
      } else {
        tail.x += s_wsum[v][0];
        tail.y += s_wsum[v][1];
        tail.z += s_wsum[v][2];
        tail.w += s_wsum[v][3];
      }
    }
    uint4 E = make_uint4(0, 0, 0, 0);
    if (t > 0) {
      // publish the aggregate, then look back
      sc.agg[t] = tail;
      __threadfence();
      st_flag(sc.flags + t, 1u | (th ? 4u : 0u));
      for (int64_t j = (int64_t)t - 1; j >= 0; j--) {
        uint32_t f = 0, spins = 0;
        while ((f = ld_flag(sc.flags + j)) == 0u) {
          if (++spins > kSpinLimit) break;
          __nanosleep(64);
        }
        if (f == 0u) {
          set_status(status, BP_ERR_TIMEOUT);
          break;
        }
        if (f == 2u) {
          const uint4 v = __ldcg(sc.incl + j);
          E.x += v.x; E.y += v.y; E.z += v.z; E.w += v.w;
          break;
        }
        const uint4 v = __ldcg(sc.agg + j);
        E.x += v.x; E.y += v.y; E.z += v.z; E.w += v.w;
        if (f & 4u) break;
      }
    }
    uint4 inc = tail;
    if (!th) {
      inc.x += E.x; inc.y += E.y; inc.z += E.z; inc.w += E.w;
    }
    sc.incl[t] = inc;
    __threadfence();
    st_flag(sc.flags + t, 2u);
    s_E = E;
  }
  __syncthreads();
  const uint32_t Es = comp(s_E, s);

  // seeds and output (list changes are warp-uniform, so sums reduce per warp)
  auto flush = [&](uint64_t &a, uint32_t li) {
#pragma unroll
    for (int dd = 16; dd > 0; dd >>= 1) a += __shfl_down_sync(kFull, a, dd);
    if (lane == 0 && a) atomicAdd(reinterpret_cast<unsigned long long *>(sums + li), a);
    a = 0;
  };
  uint64_t acc = 0;
  uint32_t acc_list = 0xFFFFFFFFu;
  bool head_in_warp = false;
#pragma unroll
  for (int i = 0; i < 4; i++) {
    if (lst[i] == 0xFFFFFFFFu) continue;
    if (head[i]) head_in_warp = true;
    uint32_t seed = pw[i];
    if (!head_in_warp) {
      seed += W;
      if (!head_before) seed += Es;
    }
    if (head[i]) seed = 0;
    const bp_list L = src.get(lst[i]);
    if (!isblk[i]) {
      // tail unit: its seed's column 3 is the last packed value of the list
      if (kb[i] == L.n / 128u && s == 3 && c == 0) sc.lastval[lst[i]] = seed;
      continue;
    }
    const uint32_t base = seed + cex[i];
    if (SUM) {
      if (acc_list != lst[i]) {
        if (acc_list != 0xFFFFFFFFu) flush(acc, acc_list);
        acc_list = lst[i];
      }
#pragma unroll
      for (int j = 0; j < 4; j++) acc += base + xv[i][j];
    } else {
      uint32_t *o = out + L.out_offset + 128ull * kb[i] + 16 * c + s;
#pragma unroll
      for (int j = 0; j < 4; j++) o[4 * j] = base + xv[i][j];
    }
  }
  if (SUM && acc_list != 0xFFFFFFFFu) flush(acc, acc_list);
}

// ---- 3. varint tail ----------------------------------------------------------------

template <bool SUM>
__global__ void __launch_bounds__(kThreads)
    pl_tail_kernel(const uint8_t *__restrict__ data, ListSrc src, uint32_t *__restrict__ out,
                   uint64_t *sums, PlScratch sc, uint32_t *status) {
  __shared__ uint8_t s_bytes[8][640];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint32_t warp = (blockIdx.x * kThreads + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * kThreads) >> 5;
  for (uint32_t li = warp; li < src.count; li += nwarps) {
    const bp_list L = src.get(li);
    const uint32_t nb = L.n / 128u, np = 128u * nb, nt = L.n - np;
    const uint64_t e = sc.boffw[L.unit_base + nb];
    if (nt == 0 || (e >> 56) == kBadWidth) continue;
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

PlScratch carve(void *scratch, uint64_t units, uint32_t count) {
  const PlLayout L = pl_layout(units, count);
  uint8_t *b = static_cast<uint8_t *>(scratch);
  PlScratch sc;
  sc.boffw = reinterpret_cast<uint64_t *>(b + L.boffw);
  sc.ticket = reinterpret_cast<uint32_t *>(b + L.ticket);
  sc.flags = reinterpret_cast<uint32_t *>(b + L.flags);
  sc.agg = reinterpret_cast<uint4 *>(b + L.agg);
  sc.incl = reinterpret_cast<uint4 *>(b + L.incl);
  sc.lastval = reinterpret_cast<uint32_t *>(b + L.lastval);
  return sc;
}

}  // namespace

size_t pl_scratch_bytes(uint64_t total_units, uint32_t count) {
  return pl_layout(total_units, count).total;
}

int launch_pl_decode(const uint8_t *data, const ListSrc &src, uint64_t total_units,
                     uint32_t *out, uint64_t out_cap, uint64_t *sums, void *scratch,
                     size_t scratch_bytes, uint32_t *status, cudaStream_t s) {
  if (total_units == 0 || src.count == 0) return BP_OK;
  if (!scratch || scratch_bytes < pl_scratch_bytes(total_units, src.count)) return BP_ERR_SCRATCH;
  const PlLayout L = pl_layout(total_units, src.count);
  const PlScratch sc = carve(scratch, total_units, src.count);
  const uint64_t ntiles = (total_units + kTileUnits - 1) / kTileUnits;
  if (cudaMemsetAsync(static_cast<uint8_t *>(scratch) + L.ticket, 0, L.agg - L.ticket, s) !=
      cudaSuccess)
    return BP_ERR_CUDA;
  const int wgrid = (int)std::min<uint64_t>((src.count + 7) / 8, 4096);
  pl_walk_kernel<<<wgrid, kThreads, 0, s>>>(data, src, sc, out_cap, sums != nullptr, status);
  if (sums) {
    pl_decode_kernel<true><<<(unsigned)ntiles, kThreads, 0, s>>>(data, src, total_units, out, sums,
                                                                 sc, status);
    pl_tail_kernel<true><<<wgrid, kThreads, 0, s>>>(data, src, out, sums, sc, status);
  } else {
    pl_decode_kernel<false><<<(unsigned)ntiles, kThreads, 0, s>>>(data, src, total_units, out,
                                                                  sums, sc, status);
    pl_tail_kernel<false><<<wgrid, kThreads, 0, s>>>(data, src, out, sums, sc, status);
  }
  return cudaPeekAtLastError() == cudaSuccess ? BP_OK : BP_ERR_CUDA;
}

}  // namespace bp
