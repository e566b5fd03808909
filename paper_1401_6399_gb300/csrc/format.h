// format.h -- geometry of the two stream layouts, shared by the host encoder
// and the CUDA kernels of this library (host/device inline functions only).
#pragma once
#include <stddef.h>
#include <stdint.h>

#ifdef __CUDACC__
#define BP_HD __host__ __device__ __forceinline__
#else
#define BP_HD inline
#endif

namespace bp_fmt {

constexpr uint32_t kGlMagic = 0x344C4742u;  // "BGL4"
constexpr size_t kPaperHeader = 16;         // {n, 0, tail_bytes, 0}
constexpr size_t kGlHeader = 64;
constexpr size_t kMaxList = 0x7FFFFFFFull;  // integers per list
constexpr uint32_t kBitmapMagic = 0x314D5042u;  // "BPM1"
constexpr size_t kBitmapHeader = 16;           // {magic, layout 2, n, words}

// Words of the bitmap of a universe of u values (a multiple of 4).
BP_HD uint64_t bitmap_words(uint64_t universe) { return ((universe + 31) / 32 + 3) & ~3ull; }

BP_HD size_t up16(size_t v) { return (v + 15) & ~(size_t)15; }

struct GlGeometry {
  size_t nblocks, nsuper, off_first, off_sbo, off_bw, off_payload;
};

BP_HD GlGeometry gl_geometry(size_t n) {
  GlGeometry g;
  g.nblocks = (n + 127) / 128;
  g.nsuper = (g.nblocks + 31) / 32;
  g.off_first = kGlHeader;
  g.off_sbo = g.off_first + up16(4 * g.nblocks);
  g.off_bw = g.off_sbo + up16(4 * (g.nsuper + 1));
  g.off_payload = g.off_bw + up16(g.nblocks);
  return g;
}

// S4-FastPFOR in the GPU layout (GP): GL's blocks and pages of 32 blocks,
// with a 4-byte meta entry {b', b - b', exceptions, 0} per block instead of
// a width byte, and each page's exception positions and high bits after its
// low bits.
constexpr uint32_t kGpMagic = 0x34504742u;  // "BGP4"

struct GpGeometry {
  size_t nblocks, npages, off_first, off_spo, off_meta, off_payload;
};

BP_HD GpGeometry gp_geometry(size_t n) {
  GpGeometry g;
  g.nblocks = (n + 127) / 128;
  g.npages = (g.nblocks + 31) / 32;
  g.off_first = kGlHeader;
  g.off_spo = g.off_first + up16(4 * g.nblocks);
  g.off_meta = g.off_spo + up16(4 * (g.npages + 1));
  g.off_payload = g.off_meta + up16(4 * g.nblocks);
  return g;
}

// Largest GP stream: no block costs more bits than unpatched (128 b <= 4096
// bits), and a page adds less than 5 words of padding.
BP_HD uint64_t gp_bound(uint64_t n) {
  const GpGeometry g = gp_geometry(n);
  return g.off_payload + 512ull * g.nblocks + 32ull * g.npages;
}

// Largest PL stream of n integers: every block at width 32 plus its width
// byte, and five bytes per varint of the tail.
BP_HD uint64_t pl_bound(uint64_t n) {
  const uint64_t nb = n / 128;
  return kPaperHeader + (nb / 16) * 16 + nb % 16 + nb * 512 + (n % 128) * 5;
}

// Work units of a list in a batch: GL and GP -> groups of 32 blocks; PL ->
// one unit per 128-integer block plus one for the varint tail.
BP_HD uint64_t units_of(uint64_t n, int layout) {
  if (layout == 1 || layout == 3) return ((n + 127) / 128 + 31) / 32;
  return n / 128 + 1;
}

}  // namespace bp_fmt
