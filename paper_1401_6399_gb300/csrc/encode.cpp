// encode.cpp -- host encoder for the S4-BP128-D4 paper layout and the GPU
// layout, plus stream-header parsing and batch planning (C ABI in bp128.h).
//
// Section 4.3 (container), Section 4.2 / Fig. 2 (4-lane interleave),
// Section 5 (D4 differential coding), Section 4.1 (varint tail).
#include <algorithm>
#include <cstring>
#include <thread>
#include <vector>

#include "../../include/bp128.h"
#include "format.h"

namespace {

inline unsigned width_of(uint32_t v) { return v ? 32u - (unsigned)__builtin_clz(v) : 0u; }

inline void put_le32(uint8_t *p, uint32_t v) { std::memcpy(p, &v, 4); }

// Section 5: the index of the earlier value that x[g] is coded against --
// D4 g-4, DM the last value of the previous 4-vector, D2 g-2, D1 g-1 --
// negative when the value lies before the list (or block).
inline int64_t ref_index(int kind, int64_t g) {
  switch (kind) {
    case BP_DELTA_DM: return 4 * (g / 4) - 1;
    case BP_DELTA_D2: return g - 2;
    case BP_DELTA_D1: return g - 1;
    default: return g - 4;
  }
}

// Run f(lo, hi) over [0, count) split into `nthreads` contiguous ranges.
template <class F>
void parallel_ranges(size_t count, int nthreads, F f) {
  if (nthreads <= 1 || count < 4096) {
    f(size_t(0), count);
    return;
  }
  const size_t nt = std::min<size_t>((size_t)nthreads, 256);
  std::vector<std::thread> th;
  const size_t step = (count + nt - 1) / nt;
  for (size_t t = 0; t < nt; t++) {
    const size_t lo = t * step, hi = std::min(count, lo + step);
    if (lo >= hi) break;
    th.emplace_back([=] { f(lo, hi); });
  }
  for (auto &x : th) x.join();
}

// ---- paper layout ---------------------------------------------------------

// Pack 128 D4 deltas of one block in the 4-lane interleave (Fig. 2):
// integer n -> lane n%4, slot n/4, lane word k at block word 4k+lane.
void pack_s4(const uint32_t *d, unsigned b, uint32_t *w) {
  std::memset(w, 0, 16 * b);
  if (!b) return;
  for (unsigned lane = 0; lane < 4; lane++) {
    unsigned bit = 0;
    for (unsigned slot = 0; slot < 32; slot++, bit += b) {
      const uint32_t v = d[4 * slot + lane];
      const unsigned k = bit >> 5, o = bit & 31;
      w[4 * k + lane] |= v << o;
      if (o + b > 32) w[4 * (k + 1) + lane] |= v >> (32 - o);
    }
  }
}

// Delta of list position g (the values before the list are 0).
inline uint32_t pl_delta(int kind, const uint32_t *x, size_t g) {
  const int64_t j = ref_index(kind, (int64_t)g);
  return x[g] - (j >= 0 ? x[j] : 0u);
}

int encode_paper(const uint32_t *x, size_t n, int kind, uint8_t *out, size_t cap,
                 size_t *out_bytes, int nthreads) {
  const size_t nb = n / 128, np = nb * 128, meta = nb / 16;
  std::vector<uint8_t> widths(nb);
  parallel_ranges(nb, nthreads, [&](size_t lo, size_t hi) {
    for (size_t k = lo; k < hi; k++) {
      uint32_t m = 0;
      for (unsigned i = 0; i < 128; i++) m |= pl_delta(kind, x, 128 * k + i);
      widths[k] = (uint8_t)width_of(m);  // OR has the same width as the max
    }
  });
  // byte offset of every block
  std::vector<size_t> boff(nb + 1);
  size_t pos = bp_fmt::kPaperHeader;
  for (size_t k = 0; k < nb; k++) {
    if (k < 16 * meta) {
      if (k % 16 == 0) pos += 16;
    } else {
      pos += 1;
    }
    boff[k] = pos;
    pos += 16 * (size_t)widths[k];
  }
  const size_t body_end = pos;
  // tail: varint of D1 gaps
  uint8_t tailbuf[128 * 5];
  size_t tail = 0;
  uint32_t prev = np ? x[np - 1] : 0u;
  for (size_t i = np; i < n; i++) {
    uint32_t g = x[i] - prev;
    prev = x[i];
    while (g >= 128u) {
      tailbuf[tail++] = (uint8_t)(g & 127u);
      g >>= 7;
    }
    tailbuf[tail++] = (uint8_t)(g | 128u);
  }
  if (body_end + tail > cap) return BP_ERR_CAPACITY;

  put_le32(out + 0, (uint32_t)n);
  put_le32(out + 4, 0u);
  put_le32(out + 8, (uint32_t)tail);
  put_le32(out + 12, (uint32_t)kind);
  for (size_t m = 0; m < meta; m++) std::memcpy(out + boff[16 * m] - 16, &widths[16 * m], 16);
  for (size_t k = 16 * meta; k < nb; k++) out[boff[k] - 1] = widths[k];
  parallel_ranges(nb, nthreads, [&](size_t lo, size_t hi) {
    uint32_t d[128], w[128];
    for (size_t k = lo; k < hi; k++) {
      for (unsigned i = 0; i < 128; i++) d[i] = pl_delta(kind, x, 128 * k + i);
      pack_s4(d, widths[k], w);
      std::memcpy(out + boff[k], w, 16 * (size_t)widths[k]);
    }
  });
  std::memcpy(out + body_end, tailbuf, tail);
  *out_bytes = body_end + tail;
  return BP_OK;
}

// ---- GPU layout -------------------------------------------------------------

// Column-major packing: delta of position 4t+s at bit b*(32s+t).
void pack_gl(const uint32_t *d, unsigned b, uint32_t *w) {
  std::memset(w, 0, 16 * b);
  if (!b) return;
  unsigned bit = 0;
  for (unsigned s = 0; s < 4; s++)
    for (unsigned t = 0; t < 32; t++, bit += b) {
      const uint32_t v = d[4 * t + s];
      const unsigned k = bit >> 5, o = bit & 31;
      w[k] |= v << o;
      if (o + b > 32) w[k + 1] |= v >> (32 - o);
    }
}

// Deltas of block k, the values before the block being F = x[128k]; a
// short last block is padded so that every missing delta is zero.
void gl_deltas(const uint32_t *x, size_t n, size_t k, int kind, uint32_t *d) {
  const size_t base = 128 * k;
  const unsigned cnt = (unsigned)std::min<size_t>(128, n - base);
  const uint32_t F = x[base];
  uint32_t xx[128];
  for (unsigned i = 0; i < 128; i++) {
    const int64_t j = ref_index(kind, i);
    const uint32_t ref = j >= 0 ? xx[j] : F;
    xx[i] = i < cnt ? x[base + i] : ref;
    d[i] = xx[i] - ref;
  }
}

int encode_gpu(const uint32_t *x, size_t n, int kind, uint8_t *out, size_t cap,
               size_t *out_bytes, int nthreads) {
  const bp_fmt::GlGeometry g = bp_fmt::gl_geometry(n);
  std::vector<uint8_t> widths(g.nblocks);
  parallel_ranges(g.nblocks, nthreads, [&](size_t lo, size_t hi) {
    uint32_t d[128];
    for (size_t k = lo; k < hi; k++) {
      gl_deltas(x, n, k, kind, d);
      uint32_t m = 0;
      for (unsigned i = 0; i < 128; i++) m |= d[i];
      widths[k] = (uint8_t)width_of(m);
    }
  });
  std::vector<uint64_t> woff(g.nblocks + 1);
  uint64_t w = 0;
  for (size_t k = 0; k < g.nblocks; k++) {
    woff[k] = w;
    w += 4 * (uint64_t)widths[k];
  }
  woff[g.nblocks] = w;
  if (w > 0xFFFFFFFFull) return BP_ERR_ARG;
  const size_t total = g.off_payload + 4 * (size_t)w;
  if (total > cap) return BP_ERR_CAPACITY;

  std::memset(out, 0, g.off_payload);
  uint32_t hdr[16] = {bp_fmt::kGlMagic, 1u, (uint32_t)n, (uint32_t)g.nblocks,
                      (uint32_t)g.nsuper, (uint32_t)w, (uint32_t)g.off_first,
                      (uint32_t)g.off_sbo, (uint32_t)g.off_bw,
                      (uint32_t)g.off_payload, (uint32_t)(total & 0xFFFFFFFFu),
                      (uint32_t)((uint64_t)total >> 32), (uint32_t)kind, 0, 0, 0};
  std::memcpy(out, hdr, 64);
  for (size_t q = 0; q <= g.nsuper; q++)
    put_le32(out + g.off_sbo + 4 * q, (uint32_t)woff[std::min(32 * q, g.nblocks)]);
  std::memcpy(out + g.off_bw, widths.data(), g.nblocks);
  parallel_ranges(g.nblocks, nthreads, [&](size_t lo, size_t hi) {
    uint32_t d[128], wb[128];
    for (size_t k = lo; k < hi; k++) {
      put_le32(out + g.off_first + 4 * k, x[128 * k]);
      gl_deltas(x, n, k, kind, d);
      pack_gl(d, widths[k], wb);
      std::memcpy(out + g.off_payload + 4 * woff[k], wb, 16 * (size_t)widths[k]);
    }
  });
  *out_bytes = total;
  return BP_OK;
}

// Exact GL size of list x[0..n) (needs its block widths).
size_t gl_size(const uint32_t *x, size_t n) {
  const bp_fmt::GlGeometry g = bp_fmt::gl_geometry(n);
  uint64_t w = 0;
  uint32_t d[128];
  for (size_t k = 0; k < g.nblocks; k++) {
    gl_deltas(x, n, k, BP_DELTA_D4, d);
    uint32_t m = 0;
    for (unsigned i = 0; i < 128; i++) m |= d[i];
    w += 4 * width_of(m);
  }
  return g.off_payload + 4 * (size_t)w;
}

// ---- S4-FastPFOR, GPU layout (GP) ------------------------------------------

struct PforBlock {
  uint8_t bp, w, c;  // low width b', high width b - b', exceptions
};

// Section 4.4: b' in [0, b] minimizing 128 b' + c(b') (b - b' + 8), the
// largest on a tie; c(b') from a histogram of the deltas' widths.
PforBlock pfor_choose(const uint32_t *d) {
  unsigned hist[33] = {0};
  for (unsigned i = 0; i < 128; i++) hist[width_of(d[i])]++;
  unsigned b = 32;
  while (b > 0 && hist[b] == 0) b--;
  unsigned above = 0;  // deltas wider than the candidate b'
  uint64_t best_cost = ~0ull;
  PforBlock best{0, 0, 0};
  for (int bp = (int)b; bp >= 0; bp--) {
    const uint64_t cost = 128ull * (unsigned)bp + (uint64_t)above * (b - (unsigned)bp + 8);
    if (cost < best_cost) {  // strictly lower: a tie keeps the larger b'
      best_cost = cost;
      best = PforBlock{(uint8_t)bp, (uint8_t)(b - (unsigned)bp), (uint8_t)above};
    }
    above += hist[bp];
  }
  if (best.c == 0) best.w = 0;
  return best;
}

// Words of a page: the low bits, the position bytes and the high bits of its
// blocks, the last two padded to a word, the page to 4 words.
uint64_t gp_page_words(const std::vector<PforBlock> &m, size_t k0, size_t k1) {
  uint64_t low = 0, ne = 0, hbits = 0;
  for (size_t k = k0; k < k1; k++) {
    low += 4ull * m[k].bp;
    ne += m[k].c;
    hbits += (uint64_t)m[k].c * m[k].w;
  }
  return (low + (ne + 3) / 4 + (hbits + 31) / 32 + 3) & ~3ull;
}

// OR v (w bits) into the little-endian bit string at `words`, bit `bit`.
void put_field(uint8_t *words, uint64_t bit, uint32_t v, unsigned w) {
  uint8_t *p = words + 4 * (bit >> 5);
  const unsigned o = (unsigned)(bit & 31);
  uint32_t cur;
  std::memcpy(&cur, p, 4);
  cur |= v << o;
  std::memcpy(p, &cur, 4);
  if (o + w > 32) {
    std::memcpy(&cur, p + 4, 4);
    cur |= v >> (32 - o);
    std::memcpy(p + 4, &cur, 4);
  }
}

int encode_pfor(const uint32_t *x, size_t n, int kind, uint8_t *out, size_t cap,
                size_t *out_bytes, int nthreads) {
  const bp_fmt::GpGeometry g = bp_fmt::gp_geometry(n);
  std::vector<PforBlock> meta(g.nblocks);
  parallel_ranges(g.nblocks, nthreads, [&](size_t lo, size_t hi) {
    uint32_t d[128];
    for (size_t k = lo; k < hi; k++) {
      gl_deltas(x, n, k, kind, d);
      meta[k] = pfor_choose(d);
    }
  });
  std::vector<uint64_t> poff(g.npages + 1);
  uint64_t w = 0;
  for (size_t p = 0; p < g.npages; p++) {
    poff[p] = w;
    w += gp_page_words(meta, 32 * p, std::min(g.nblocks, 32 * p + 32));
  }
  poff[g.npages] = w;
  if (w > 0xFFFFFFFFull) return BP_ERR_ARG;
  const size_t total = g.off_payload + 4 * (size_t)w;
  if (total > cap) return BP_ERR_CAPACITY;

  std::memset(out, 0, total);
  const uint32_t hdr[16] = {bp_fmt::kGpMagic, 3u, (uint32_t)n, (uint32_t)g.nblocks,
                            (uint32_t)g.npages, (uint32_t)w, (uint32_t)g.off_first,
                            (uint32_t)g.off_spo, (uint32_t)g.off_meta,
                            (uint32_t)g.off_payload, (uint32_t)(total & 0xFFFFFFFFu),
                            (uint32_t)((uint64_t)total >> 32), (uint32_t)kind, 0, 0, 0};
  std::memcpy(out, hdr, 64);
  for (size_t p = 0; p <= g.npages; p++) put_le32(out + g.off_spo + 4 * p, (uint32_t)poff[p]);
  for (size_t k = 0; k < g.nblocks; k++) {
    out[g.off_meta + 4 * k + 0] = meta[k].bp;
    out[g.off_meta + 4 * k + 1] = meta[k].w;
    out[g.off_meta + 4 * k + 2] = meta[k].c;
  }
  parallel_ranges(g.npages, nthreads, [&](size_t lo, size_t hi) {
    uint32_t d[128], lowd[128], wb[128];
    std::vector<uint8_t> pos;
    std::vector<uint32_t> high, hw;
    for (size_t p = lo; p < hi; p++) {
      const size_t k0 = 32 * p, k1 = std::min(g.nblocks, k0 + 32);
      uint8_t *page = out + g.off_payload + 4 * poff[p];
      uint64_t wl = 0;
      pos.clear();
      high.clear();
      hw.clear();
      for (size_t k = k0; k < k1; k++) {
        put_le32(out + g.off_first + 4 * k, x[128 * k]);
        gl_deltas(x, n, k, kind, d);
        const PforBlock m = meta[k];
        const uint32_t mask = m.bp >= 32 ? 0xFFFFFFFFu : (1u << m.bp) - 1u;
        for (unsigned i = 0; i < 128; i++) {
          lowd[i] = d[i] & mask;
          if (d[i] & ~mask) {  // an exception (only when b' < b)
            pos.push_back((uint8_t)i);
            high.push_back(d[i] >> m.bp);
            hw.push_back(m.w);
          }
        }
        pack_gl(lowd, m.bp, wb);
        std::memcpy(page + 4 * wl, wb, 16 * (size_t)m.bp);
        wl += 4ull * m.bp;
      }
      if (!pos.empty()) std::memcpy(page + 4 * wl, pos.data(), pos.size());
      uint8_t *hbase = page + 4 * (wl + (pos.size() + 3) / 4);
      uint64_t bit = 0;
      for (size_t e = 0; e < high.size(); e++) {
        put_field(hbase, bit, high[e], hw[e]);
        bit += hw[e];
      }
    }
  });
  *out_bytes = total;
  return BP_OK;
}

}  // namespace

extern "C" {

size_t bp_index_bound(const uint64_t *offs, uint32_t count) {
  size_t total = 0;
  for (uint32_t i = 0; i < count; i++)
    total += bp_fmt::up16(bp_encode_bound(offs[i + 1] - offs[i], BP_LAYOUT_GPU));
  return total;
}

int bp_index_encode(const uint32_t *values, const uint64_t *offs, uint32_t count, uint8_t *out,
                    size_t cap, bp_list *lists, size_t *out_bytes, int nthreads) {
  if (!values || !offs || !out || !lists || !out_bytes) return BP_ERR_ARG;
  std::vector<size_t> sizes(count);
  std::vector<int> bad(count, 0);
  parallel_ranges(count, nthreads, [&](size_t lo, size_t hi) {
    for (size_t i = lo; i < hi; i++) {
      const uint32_t *x = values + offs[i];
      const size_t n = offs[i + 1] - offs[i];
      if (n > bp_fmt::kMaxList) bad[i] = BP_ERR_ARG;
      for (size_t j = 1; j < n && !bad[i]; j++)
        if (x[j] <= x[j - 1]) bad[i] = BP_ERR_UNSORTED;
      if (!bad[i]) sizes[i] = gl_size(x, n);
    }
  });
  size_t pos = 0;
  for (uint32_t i = 0; i < count; i++) {
    if (bad[i]) return bad[i];
    lists[i] = bp_list{pos, sizes[i], offs[i], 0, (uint32_t)(offs[i + 1] - offs[i]),
                       (uint32_t)BP_LAYOUT_GPU, 0};
    pos += bp_fmt::up16(sizes[i]);
  }
  if (pos > cap) return BP_ERR_CAPACITY;
  bp_plan_lists(lists, count);
  std::vector<int> rc(count, BP_OK);
  parallel_ranges(count, nthreads, [&](size_t lo, size_t hi) {
    for (size_t i = lo; i < hi; i++) {
      size_t got = 0;
      const size_t n = offs[i + 1] - offs[i];
      rc[i] = encode_gpu(values + offs[i], n, BP_DELTA_D4, out + lists[i].enc_offset,
                         bp_encode_bound(n, BP_LAYOUT_GPU), &got, 1);
      if (rc[i] == BP_OK && got != sizes[i]) rc[i] = BP_ERR_ARG;
      const size_t pad = bp_fmt::up16(sizes[i]) - sizes[i];
      if (pad) std::memset(out + lists[i].enc_offset + sizes[i], 0, pad);
    }
  });
  for (uint32_t i = 0; i < count; i++)
    if (rc[i] != BP_OK) return rc[i];
  *out_bytes = pos;
  return BP_OK;
}

size_t bp_index_hybrid_bound(const uint64_t *offs, uint32_t count, uint32_t universe,
                             uint32_t B) {
  if (!offs) return 0;
  const size_t bm = bp_fmt::kBitmapHeader + 4 * bp_fmt::bitmap_words(universe);
  size_t total = 0;
  for (uint32_t i = 0; i < count; i++) {
    const uint64_t n = offs[i + 1] - offs[i];
    total += (B && n * B >= universe) ? bm
                                      : bp_fmt::up16(bp_encode_bound(n, BP_LAYOUT_GPU));
  }
  return total;
}

int bp_index_encode_hybrid(const uint32_t *values, const uint64_t *offs, uint32_t count,
                           uint32_t universe, uint32_t B, uint8_t *out, size_t cap,
                           bp_list *lists, size_t *out_bytes, int nthreads) {
  if (!values || !offs || !out || !lists || !out_bytes || universe == 0) return BP_ERR_ARG;
  const uint64_t words = bp_fmt::bitmap_words(universe);
  const size_t bm_bytes = bp_fmt::kBitmapHeader + 4 * words;
  std::vector<size_t> sizes(count);
  std::vector<uint8_t> is_bm(count, 0);
  std::vector<int> bad(count, 0);
  parallel_ranges(count, nthreads, [&](size_t lo, size_t hi) {
    for (size_t i = lo; i < hi; i++) {
      const uint32_t *x = values + offs[i];
      const size_t n = offs[i + 1] - offs[i];
      if (n > bp_fmt::kMaxList) bad[i] = BP_ERR_ARG;
      for (size_t j = 1; j < n && !bad[i]; j++)
        if (x[j] <= x[j - 1]) bad[i] = BP_ERR_UNSORTED;
      if (bad[i]) continue;
      if (B && (uint64_t)n * B >= universe) {
        if (n && x[n - 1] >= universe) bad[i] = BP_ERR_ARG;
        is_bm[i] = 1;
        sizes[i] = bm_bytes;
      } else {
        sizes[i] = gl_size(x, n);
      }
    }
  });
  size_t pos = 0;
  for (uint32_t i = 0; i < count; i++) {
    if (bad[i]) return bad[i];
    lists[i] = bp_list{pos, sizes[i], offs[i], 0, (uint32_t)(offs[i + 1] - offs[i]),
                       is_bm[i] ? (uint32_t)BP_LAYOUT_BITMAP : (uint32_t)BP_LAYOUT_GPU, 0};
    pos += bp_fmt::up16(sizes[i]);
  }
  if (pos > cap) return BP_ERR_CAPACITY;
  std::vector<int> rc(count, BP_OK);
  parallel_ranges(count, nthreads, [&](size_t lo, size_t hi) {
    for (size_t i = lo; i < hi; i++) {
      const size_t n = offs[i + 1] - offs[i];
      uint8_t *o = out + lists[i].enc_offset;
      if (is_bm[i]) {
        std::memset(o, 0, bm_bytes);
        put_le32(o + 0, bp_fmt::kBitmapMagic);
        put_le32(o + 4, (uint32_t)BP_LAYOUT_BITMAP);
        put_le32(o + 8, (uint32_t)n);
        put_le32(o + 12, (uint32_t)words);
        uint8_t *bits = o + bp_fmt::kBitmapHeader;
        for (size_t j = 0; j < n; j++) {
          const uint32_t v = values[offs[i] + j];
          bits[v >> 3] |= (uint8_t)(1u << (v & 7));  // little endian: bit v%32 of word v/32
        }
      } else {
        size_t got = 0;
        rc[i] = encode_gpu(values + offs[i], n, BP_DELTA_D4, o, bp_encode_bound(n, BP_LAYOUT_GPU),
                           &got, 1);
        if (rc[i] == BP_OK && got != sizes[i]) rc[i] = BP_ERR_ARG;
      }
      const size_t pad = bp_fmt::up16(sizes[i]) - sizes[i];
      if (pad) std::memset(o + sizes[i], 0, pad);
    }
  });
  for (uint32_t i = 0; i < count; i++)
    if (rc[i] != BP_OK) return rc[i];
  *out_bytes = pos;
  return BP_OK;
}

size_t bp_encode_bound(size_t n, int layout) {
  if (layout == BP_LAYOUT_PAPER) return bp_fmt::pl_bound(n);
  if (layout == BP_LAYOUT_GPU) {
    const bp_fmt::GlGeometry g = bp_fmt::gl_geometry(n);
    return g.off_payload + 512 * g.nblocks;
  }
  if (layout == BP_LAYOUT_PFOR) return bp_fmt::gp_bound(n);
  return 0;
}

int bp_encode(const uint32_t *in, size_t n, int layout, uint8_t *out,
              size_t cap, size_t *out_bytes, int nthreads) {
  return bp_encode_kind(in, n, layout, BP_DELTA_D4, out, cap, out_bytes, nthreads);
}

int bp_encode_kind(const uint32_t *in, size_t n, int layout, int delta, uint8_t *out,
                   size_t cap, size_t *out_bytes, int nthreads) {
  if (!out || !out_bytes || (n && !in)) return BP_ERR_ARG;
  if (layout != BP_LAYOUT_PAPER && layout != BP_LAYOUT_GPU && layout != BP_LAYOUT_PFOR)
    return BP_ERR_ARG;
  const bool any_order = (delta & BP_ENCODE_ANY_ORDER) != 0;
  delta &= ~BP_ENCODE_ANY_ORDER;
  if (delta < BP_DELTA_D4 || delta > BP_DELTA_D1) return BP_ERR_ARG;
  if (n > bp_fmt::kMaxList) return BP_ERR_ARG;
  for (size_t i = 1; i < n && !any_order; i++)
    if (in[i] <= in[i - 1]) return BP_ERR_UNSORTED;
  if (cap < bp_encode_bound(n, layout)) return BP_ERR_CAPACITY;
  if (layout == BP_LAYOUT_PFOR) return encode_pfor(in, n, delta, out, cap, out_bytes, nthreads);
  return layout == BP_LAYOUT_PAPER ? encode_paper(in, n, delta, out, cap, out_bytes, nthreads)
                                   : encode_gpu(in, n, delta, out, cap, out_bytes, nthreads);
}

int bp_stream_info(const uint8_t *enc, size_t enc_bytes, uint32_t *n_out,
                   int *layout_out) {
  if (!enc || !n_out || !layout_out) return BP_ERR_ARG;
  uint32_t h[16];
  if (enc_bytes < 16) return BP_ERR_CORRUPT;
  std::memcpy(h, enc, 16);
  if (h[1] == 0u && h[3] <= (uint32_t)BP_DELTA_D1) {
    *n_out = h[0];
    *layout_out = BP_LAYOUT_PAPER;
    return BP_OK;
  }
  if (enc_bytes < 64) return BP_ERR_CORRUPT;
  std::memcpy(h, enc, 64);
  if (h[0] == bp_fmt::kGlMagic && h[1] == 1u) {
    const bp_fmt::GlGeometry g = bp_fmt::gl_geometry(h[2]);
    const uint64_t total = (uint64_t)h[10] | ((uint64_t)h[11] << 32);
    if (h[3] != g.nblocks || h[4] != g.nsuper || h[9] != g.off_payload ||
        total != g.off_payload + 4ull * h[5] || total > enc_bytes)
      return BP_ERR_CORRUPT;
    if (h[12] > (uint32_t)BP_DELTA_D1) return BP_ERR_CORRUPT;
    *n_out = h[2];
    *layout_out = BP_LAYOUT_GPU;
    return BP_OK;
  }
  if (h[0] == bp_fmt::kGpMagic && h[1] == 3u) {
    const bp_fmt::GpGeometry g = bp_fmt::gp_geometry(h[2]);
    const uint64_t total = (uint64_t)h[10] | ((uint64_t)h[11] << 32);
    if (h[3] != g.nblocks || h[4] != g.npages || h[6] != g.off_first || h[7] != g.off_spo ||
        h[8] != g.off_meta || h[9] != g.off_payload || total != g.off_payload + 4ull * h[5] ||
        total > enc_bytes || h[12] > (uint32_t)BP_DELTA_D1)
      return BP_ERR_CORRUPT;
    *n_out = h[2];
    *layout_out = BP_LAYOUT_PFOR;
    return BP_OK;
  }
  return BP_ERR_CORRUPT;
}

int bp_stream_kind(const uint8_t *enc, size_t enc_bytes, int *delta_out) {
  uint32_t n = 0;
  int layout = 0;
  if (!delta_out) return BP_ERR_ARG;
  const int rc = bp_stream_info(enc, enc_bytes, &n, &layout);
  if (rc != BP_OK) return rc;
  uint32_t w;
  std::memcpy(&w, enc + (layout == BP_LAYOUT_PAPER ? 12 : 48), 4);
  *delta_out = (int)w;
  return BP_OK;
}

uint64_t bp_plan_lists(bp_list *lists, uint32_t count) {
  uint64_t u = 0;
  for (uint32_t i = 0; i < count; i++) {
    lists[i].unit_base = u;
    u += bp_fmt::units_of(lists[i].n, (int)lists[i].layout);
  }
  return u;
}

const char *bp_status_string(int status) {
  switch (status) {
    case BP_OK: return "ok";
    case BP_ERR_ARG: return "invalid argument";
    case BP_ERR_UNSORTED: return "input not strictly increasing";
    case BP_ERR_CORRUPT: return "corrupt compressed stream";
    case BP_ERR_CAPACITY: return "output buffer too small";
    case BP_ERR_CUDA: return "CUDA error";
    case BP_ERR_TIMEOUT: return "device wait timed out";
    case BP_ERR_SCRATCH: return "scratch buffer too small";
    default: return "unknown status";
  }
}

}  // extern "C"
