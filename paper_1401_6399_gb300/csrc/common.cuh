// common.cuh -- device helpers shared by the kernels of this library.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/bp128.h"
#include "format.h"

namespace bp {

constexpr unsigned kFull = 0xFFFFFFFFu;

// First error wins; later calls leave the word alone.
__device__ __forceinline__ void set_status(uint32_t *st, uint32_t code) {
  if (st) atomicCAS(st, 0u, code);
}

__host__ __device__ constexpr int gcd_c(int a, int b) { return b == 0 ? a : gcd_c(b, a % b); }

__device__ __forceinline__ uint32_t ld_nc(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.global.nc.L1::no_allocate.u32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}

__device__ __forceinline__ uint32_t low_mask(int b) {
  return b >= 32 ? 0xFFFFFFFFu : ((1u << b) - 1u);
}

// A GL stream as seen from the device after its header has been checked.
struct GlView {
  uint32_t n, nblocks, nsuper, pw;
  uint32_t kind;  // differential coding (0 D4, 1 DM, 2 D2, 3 D1)
  const uint32_t *first;
  const uint32_t *sbo;
  const uint8_t *bw;
  const uint32_t *payload;
};

// Parse and check a GL header (64 bytes at enc).  Returns false if the header
// is inconsistent with its own n or with enc_bytes.
__device__ __forceinline__ bool gl_view(const uint8_t *enc, uint64_t enc_bytes, GlView &v) {
  if (enc_bytes < bp_fmt::kGlHeader || (reinterpret_cast<uintptr_t>(enc) & 15u) != 0) return false;
  const uint4 *h4 = reinterpret_cast<const uint4 *>(enc);
  const uint4 a = __ldg(h4 + 0), b = __ldg(h4 + 1), c = __ldg(h4 + 2), d = __ldg(h4 + 3);
  if (a.x != bp_fmt::kGlMagic || a.y != 1u) return false;
  const bp_fmt::GlGeometry g = bp_fmt::gl_geometry(a.z);
  const uint64_t total = (uint64_t)c.z | ((uint64_t)c.w << 32);
  if (a.w != g.nblocks || b.x != g.nsuper || b.z != g.off_first || b.w != g.off_sbo ||
      c.x != g.off_bw || c.y != g.off_payload || total != g.off_payload + 4ull * b.y ||
      total > enc_bytes || d.x > 3u)
    return false;
  v.n = a.z;
  v.kind = d.x;
  v.nblocks = a.w;
  v.nsuper = b.x;
  v.pw = b.y;
  v.first = reinterpret_cast<const uint32_t *>(enc + g.off_first);
  v.sbo = reinterpret_cast<const uint32_t *>(enc + g.off_sbo);
  v.bw = enc + g.off_bw;
  v.payload = reinterpret_cast<const uint32_t *>(enc + g.off_payload);
  return true;
}

// Launch geometry: a persistent grid of `per_sm` resident CTAs on every SM.
int device_sm_count();

}  // namespace bp
