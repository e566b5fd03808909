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

// Largest PL stream of n integers: every block at width 32 plus its width
// byte, and five bytes per varint of the tail.
BP_HD uint64_t pl_bound(uint64_t n) {
  const uint64_t nb = n / 128;
  return kPaperHeader + (nb / 16) * 16 + nb % 16 + nb * 512 + (n % 128) * 5;
}

// Work units of a list in a batch: GL -> groups of 32 blocks; PL -> one
// unit per 128-integer block plus one for the varint tail.
BP_HD uint64_t units_of(uint64_t n, int layout) {
  if (layout == 1) return ((n + 127) / 128 + 31) / 32;
  return n / 128 + 1;
}

}  // namespace bp_fmt
