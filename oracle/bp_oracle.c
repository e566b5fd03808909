/*
 * bp_oracle.c -- scalar reference for S4-BP128-D4 and sorted intersections.
 *
 * TEST INFRASTRUCTURE ONLY (see bp_oracle.h).  Plain scalar C, written from
 * the paper's definitions; no blocking, fusion or reordering beyond what
 * those definitions state.  Nothing here is tuned.
 *
 * Paper references: Section 4.1 (varint, Fig. 1b), Section 4.2 (bit packing,
 * Figs. 1c and 2), Section 4.3 (S4-BP128 container), Section 5 (differential
 * coding, Algorithm 1), Section 6 (intersections, Algorithms 2-4).
 */
#include "bp_oracle.h"

#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* little helpers on byte streams (portable little-endian access)          */
/* ------------------------------------------------------------------------ */

static uint32_t rd32(const uint8_t *p) {
  return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) |
         ((uint32_t)p[3] << 24);
}

static void wr32(uint8_t *p, uint32_t v) {
  p[0] = (uint8_t)v;
  p[1] = (uint8_t)(v >> 8);
  p[2] = (uint8_t)(v >> 16);
  p[3] = (uint8_t)(v >> 24);
}

static uint32_t low_mask(unsigned b) {
  return b >= 32 ? 0xFFFFFFFFu : ((1u << b) - 1u);
}

/* ------------------------------------------------------------------------ */
/* Section 4.3: the bit width b is the smallest value such that all the    */
/* integers of the block are smaller than 2^b; 0 <= b <= 32.               */
/* ------------------------------------------------------------------------ */

unsigned orc_bits(uint32_t v) {
  unsigned b = 0;
  while (b < 32 && (v >> b) != 0) b++;
  return b;
}

unsigned orc_max_bits(const uint32_t *v, size_t n) {
  unsigned b = 0;
  for (size_t i = 0; i < n; i++) {
    unsigned c = orc_bits(v[i]);
    if (c > b) b = c;
  }
  return b;
}

/* ------------------------------------------------------------------------ */
/* Section 4.2, Fig. 1c: consecutive packing, least significant bit first.  */
/* Written one bit at a time so that it reads as the definition.           */
/* ------------------------------------------------------------------------ */

void orc_pack_scalar(const uint32_t *in, size_t n, unsigned b, uint8_t *out) {
  size_t nbytes = (n * (size_t)b + 7) / 8;
  memset(out, 0, nbytes);
  for (size_t i = 0; i < n; i++) {
    for (unsigned k = 0; k < b; k++) {
      size_t p = i * (size_t)b + k;
      if ((in[i] >> k) & 1u) out[p / 8] |= (uint8_t)(1u << (p % 8));
    }
  }
}

void orc_unpack_scalar(const uint8_t *in, size_t n, unsigned b, uint32_t *out) {
  for (size_t i = 0; i < n; i++) {
    uint32_t v = 0;
    for (unsigned k = 0; k < b; k++) {
      size_t p = i * (size_t)b + k;
      if ((in[p / 8] >> (p % 8)) & 1u) v |= 1u << k;
    }
    out[i] = v;
  }
}

/* ------------------------------------------------------------------------ */
/* Section 4.2, Fig. 2: the 4-lane interleaved layout.  Integer n of the    */
/* block is the (n div 4)-th value of lane n mod 4; lane s holds its values */
/* at b bits each, least significant bit first, in the words y[4k+s].  A    */
/* value that does not fit in the rest of word k continues at the low bits */
/* of word k+1 of the same lane.                                           */
/* ------------------------------------------------------------------------ */

void orc_s4_pack128(const uint32_t in[128], unsigned b, uint32_t *out) {
  for (unsigned w = 0; w < 4 * b; w++) out[w] = 0;
  if (b == 0) return;
  const uint32_t m = low_mask(b);
  for (unsigned n = 0; n < 128; n++) {
    const unsigned s = n % 4, j = n / 4;
    const unsigned p = j * b, k = p / 32, o = p % 32;
    const uint32_t v = in[n] & m;
    out[4 * k + s] |= v << o;
    if (o + b > 32) out[4 * (k + 1) + s] |= v >> (32 - o);
  }
}

/* Algorithm 1.  For each lane word k = 0..b-1, extract every value that    */
/* lies wholly inside the word at offset i, then the one that straddles    */
/* into word k+1 (joined from the high bits of word k and the low bits of  */
/* word k+1), and apply the prefix function P to each 4-vector.  The seed  */
/* v starts at (0,0,0,0) for a stream and becomes the last vector decoded. */
/* Reading for b = 0 (where the printed loop produces nothing): all 128    */
/* values are 0, so each vector is P((0,0,0,0), v).                        */

static void apply_p(int kind, uint32_t t[4], uint32_t v[4]) {
  if (kind == ORC_P_DM) {
    /* Section 5, DM: copy the last component of the previous vector to all
     * four components and add */
    const uint32_t last = v[3];
    for (int s = 0; s < 4; s++) t[s] += last;
  } else if (kind == ORC_P_D2 || kind == ORC_P_D1) {
    /* Section 5, D2: shift the deltas by two integers and add them to
     * themselves, then add (v2, v3, v2, v3) */
    uint32_t u[4] = {t[0], t[1], t[0] + t[2], t[1] + t[3]};
    if (kind == ORC_P_D2) {
      t[0] = u[0] + v[2];
      t[1] = u[1] + v[3];
      t[2] = u[2] + v[2];
      t[3] = u[3] + v[3];
    } else {
      /* D1: shift that result by one integer and add it to itself, then add
       * the last component of the previous vector to all components */
      const uint32_t w[4] = {u[0], u[0] + u[1], u[1] + u[2], u[2] + u[3]};
      for (int s = 0; s < 4; s++) t[s] = w[s] + v[3];
    }
  }
  for (int s = 0; s < 4; s++) {
    if (kind == ORC_P_D4) t[s] += v[s]; /* P(t,v) = t + v, Section 5 */
    v[s] = t[s];
  }
}

void orc_s4_unpack128(const uint32_t *y, unsigned b, int kind, uint32_t v[4],
                      uint32_t out[128]) {
  unsigned produced = 0;
  uint32_t t[4];
  if (b == 0) {
    for (unsigned r = 0; r < 32; r++) {
      for (int s = 0; s < 4; s++) t[s] = 0;
      apply_p(kind, t, v);
      for (int s = 0; s < 4; s++) out[produced++] = t[s];
    }
    return;
  }
  const uint32_t M = low_mask(b);
  unsigned i = 0;
  for (unsigned k = 0; k < b; k++) {
    while (i + b <= 32) {
      for (int s = 0; s < 4; s++) t[s] = (y[4 * k + s] >> i) & M;
      apply_p(kind, t, v);
      for (int s = 0; s < 4; s++) out[produced++] = t[s];
      i += b;
    }
    if (i < 32) {
      /* straddle: high 32-i bits from word k, the rest from word k+1 */
      for (int s = 0; s < 4; s++) {
        uint32_t z = (y[4 * (k + 1) + s] << (32 - i)) & M;
        t[s] = (y[4 * k + s] >> i) | z;
      }
      apply_p(kind, t, v);
      for (int s = 0; s < 4; s++) out[produced++] = t[s];
      i = i + b - 32;
    } else {
      i = 0;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Section 5: D4 differential coding, delta_i = x_i - x_{i-4}, taken with    */
/* the seed (0,0,0,0) in front of the list; arithmetic is modulo 2^32.      */
/* ------------------------------------------------------------------------ */

void orc_d4_deltas(const uint32_t *x, size_t n, uint32_t *d) {
  for (size_t i = 0; i < n; i++) d[i] = x[i] - (i >= 4 ? x[i - 4] : 0u);
}

void orc_d4_prefix(const uint32_t *d, size_t n, uint32_t *x) {
  for (size_t i = 0; i < n; i++) x[i] = d[i] + (i >= 4 ? x[i - 4] : 0u);
}

/* The value x[i] is coded against, for each kind of Section 5; positions
 * before 0 hold `seed`.  DM: the last value of the previous 4-vector. */
static uint32_t delta_ref(int kind, const uint32_t *x, size_t i, uint32_t seed) {
  long long j;
  switch (kind) {
    case ORC_DELTA_DM: j = 4 * (long long)(i / 4) - 1; break;
    case ORC_DELTA_D2: j = (long long)i - 2; break;
    case ORC_DELTA_D1: j = (long long)i - 1; break;
    default: j = (long long)i - 4; break;
  }
  return j >= 0 ? x[j] : seed;
}

void orc_deltas(int kind, const uint32_t *x, size_t n, uint32_t seed, uint32_t *d) {
  for (size_t i = 0; i < n; i++) d[i] = x[i] - delta_ref(kind, x, i, seed);
}

void orc_prefix(int kind, const uint32_t *d, size_t n, uint32_t seed, uint32_t *x) {
  for (size_t i = 0; i < n; i++) x[i] = d[i] + delta_ref(kind, x, i, seed);
}

/* ------------------------------------------------------------------------ */
/* Section 4.1, Fig. 1b: varint.  Seven payload bits per byte, least        */
/* significant group first; the last byte of an integer has its high bit   */
/* set, the others have it clear.                                          */
/* ------------------------------------------------------------------------ */

size_t orc_varint_encode(const uint32_t *in, size_t n, uint8_t *out) {
  size_t k = 0;
  for (size_t i = 0; i < n; i++) {
    uint32_t v = in[i];
    while (v >= 128u) {
      out[k++] = (uint8_t)(v & 127u);
      v >>= 7;
    }
    out[k++] = (uint8_t)(v | 128u);
  }
  return k;
}

int orc_varint_decode(const uint8_t *in, size_t nbytes, size_t n,
                      uint32_t *out, size_t *used) {
  size_t k = 0;
  for (size_t i = 0; i < n; i++) {
    uint64_t v = 0;
    unsigned shift = 0;
    for (;;) {
      if (k >= nbytes) return ORC_ECORRUPT;
      if (shift > 28) return ORC_ECORRUPT; /* more than 5 bytes */
      uint8_t c = in[k++];
      v |= (uint64_t)(c & 127u) << shift;
      shift += 7;
      if (c & 128u) break;
    }
    if (v > 0xFFFFFFFFull) return ORC_ECORRUPT;
    out[i] = (uint32_t)v;
  }
  if (used) *used = k;
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Section 4.3: the S4-BP128 container, paper layout (PL).                  */
/* Readings where the paper is silent: a 16-byte header {n, 0, tail_bytes,  */
/* 0}; the varint tail codes D1 gaps from the previous integer.             */
/* ------------------------------------------------------------------------ */

static int is_sorted_distinct(const uint32_t *x, size_t n) {
  for (size_t i = 1; i < n; i++)
    if (x[i] <= x[i - 1]) return 0;
  return 1;
}

size_t orc_pl_bound(size_t n) {
  size_t nb = n / 128;
  return 16 + (nb / 16) * 16 + (nb % 16) + nb * 512 + (n % 128) * 5;
}

int orc_pl_encode(const uint32_t *x, size_t n, uint8_t *out, size_t cap,
                  size_t *out_bytes) {
  return orc_pl_encode_kind(x, n, ORC_DELTA_D4, out, cap, out_bytes);
}

int orc_pl_encode_kind(const uint32_t *x, size_t n, int kind, uint8_t *out,
                       size_t cap, size_t *out_bytes) {
  if ((!x && n) || !out || !out_bytes) return ORC_EARG;
  if (kind < ORC_DELTA_D4 || kind > ORC_DELTA_D1) return ORC_EARG;
  if (n > 0xFFFFFFFFull) return ORC_EARG;
  if (!is_sorted_distinct(x, n)) return ORC_EARG;
  if (cap < orc_pl_bound(n)) return ORC_ECAPACITY;

  const size_t nb = n / 128, np = nb * 128, meta = nb / 16;
  uint32_t *d = (uint32_t *)malloc((np ? np : 1) * sizeof(uint32_t));
  if (!d) return ORC_EARG;
  if (kind == ORC_DELTA_D4) orc_d4_deltas(x, np, d);
  else orc_deltas(kind, x, np, 0u, d);

  size_t pos = 16;
  uint32_t words[128];
  for (size_t m = 0; m < meta; m++) {
    unsigned w[16];
    for (unsigned j = 0; j < 16; j++) {
      w[j] = orc_max_bits(d + (16 * m + j) * 128, 128);
      out[pos++] = (uint8_t)w[j];
    }
    for (unsigned j = 0; j < 16; j++) {
      orc_s4_pack128(d + (16 * m + j) * 128, w[j], words);
      for (unsigned q = 0; q < 4 * w[j]; q++, pos += 4) wr32(out + pos, words[q]);
    }
  }
  for (size_t blk = meta * 16; blk < nb; blk++) {
    unsigned w = orc_max_bits(d + blk * 128, 128);
    out[pos++] = (uint8_t)w;
    orc_s4_pack128(d + blk * 128, w, words);
    for (unsigned q = 0; q < 4 * w; q++, pos += 4) wr32(out + pos, words[q]);
  }
  free(d);

  /* varint tail of D1 gaps */
  const size_t nt = n - np;
  uint32_t gaps[128];
  uint32_t prev = np ? x[np - 1] : 0u;
  for (size_t i = 0; i < nt; i++) {
    gaps[i] = x[np + i] - prev;
    prev = x[np + i];
  }
  size_t tail = orc_varint_encode(gaps, nt, out + pos);
  pos += tail;

  wr32(out + 0, (uint32_t)n);
  wr32(out + 4, 0u);
  wr32(out + 8, (uint32_t)tail);
  wr32(out + 12, (uint32_t)kind);
  *out_bytes = pos;
  return ORC_OK;
}

int orc_stream_count(const uint8_t *in, size_t nbytes, size_t *n_out) {
  if (!in || !n_out) return ORC_EARG;
  if (nbytes >= 16 && rd32(in + 4) == 0u) {
    *n_out = rd32(in);
    return ORC_OK;
  }
  if (nbytes >= 64 && (rd32(in + 4) == 1u || rd32(in + 4) == 3u)) {
    *n_out = rd32(in + 8);
    return ORC_OK;
  }
  return ORC_ECORRUPT;
}

static int pl_block(const uint8_t *in, size_t nbytes, size_t *pos, unsigned w,
                    int pkind, uint32_t v[4], uint32_t *out) {
  uint32_t y[128];
  if (w > 32) return ORC_ECORRUPT;
  if (*pos + 16 * (size_t)w > nbytes) return ORC_ECORRUPT;
  for (unsigned q = 0; q < 4 * w; q++) y[q] = rd32(in + *pos + 4 * q);
  *pos += 16 * (size_t)w;
  orc_s4_unpack128(y, w, pkind, v, out);
  return ORC_OK;
}

/* Prefix function of Algorithm 1 for a kind of differential coding. */
static int prefix_kind(uint32_t kind) {
  switch (kind) {
    case ORC_DELTA_DM: return ORC_P_DM;
    case ORC_DELTA_D2: return ORC_P_D2;
    case ORC_DELTA_D1: return ORC_P_D1;
    default: return ORC_P_D4;
  }
}

int orc_pl_decode(const uint8_t *in, size_t nbytes, uint32_t *out, size_t cap,
                  size_t *n_out) {
  if (!in || !n_out) return ORC_EARG;
  if (nbytes < 16) return ORC_ECORRUPT;
  const size_t n = rd32(in);
  const uint32_t kind = rd32(in + 12);
  if (rd32(in + 4) != 0u || kind > ORC_DELTA_D1) return ORC_ECORRUPT;
  const int pkind = prefix_kind(kind);
  const size_t tail = rd32(in + 8);
  *n_out = n;
  if (n > cap) return ORC_ECAPACITY;
  if (n && !out) return ORC_EARG;

  const size_t nb = n / 128, np = nb * 128, meta = nb / 16;
  uint32_t v[4] = {0, 0, 0, 0};
  size_t pos = 16;
  int rc;
  for (size_t m = 0; m < meta; m++) {
    if (pos + 16 > nbytes) return ORC_ECORRUPT;
    unsigned w[16];
    for (unsigned j = 0; j < 16; j++) w[j] = in[pos + j];
    pos += 16;
    for (unsigned j = 0; j < 16; j++) {
      rc = pl_block(in, nbytes, &pos, w[j], pkind, v, out + (16 * m + j) * 128);
      if (rc) return rc;
    }
  }
  for (size_t blk = meta * 16; blk < nb; blk++) {
    if (pos + 1 > nbytes) return ORC_ECORRUPT;
    unsigned w = in[pos++];
    rc = pl_block(in, nbytes, &pos, w, pkind, v, out + blk * 128);
    if (rc) return rc;
  }
  if (pos + tail != nbytes) return ORC_ECORRUPT;
  size_t used = 0;
  rc = orc_varint_decode(in + pos, tail, n - np, out + np, &used);
  if (rc) return rc;
  if (used != tail) return ORC_ECORRUPT;
  uint32_t prev = np ? out[np - 1] : 0u;
  for (size_t i = np; i < n; i++) {
    out[i] += prev;
    prev = out[i];
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* GPU layout (GL).  Not part of the paper: the same codec (128-integer    */
/* blocks, one bit width per block, D4 deltas), with a per-block skip      */
/* header so that any block decodes on its own.                            */
/*                                                                          */
/* header, 16 little-endian u32 words:                                      */
/*   0 magic 0x344C4742   1 layout tag 1     2 n          3 nblocks        */
/*   4 nsuper             5 payload words    6 off_first  7 off_sbo        */
/*   8 off_bw             9 off_payload     10 total bytes (low)           */
/*  11 total bytes (high) 12..15 zero                                      */
/* sections, each starting on a 16-byte boundary:                           */
/*   first[nblocks] u32, sbo[nsuper+1] u32, bw[nblocks] u8, payload words  */
/* ------------------------------------------------------------------------ */

#define GL_MAGIC 0x344C4742u

static size_t up16(size_t v) { return (v + 15) & ~(size_t)15; }

static void gl_offsets(size_t nblocks, size_t nsuper, size_t *off_first,
                       size_t *off_sbo, size_t *off_bw, size_t *off_payload) {
  *off_first = 64;
  *off_sbo = *off_first + up16(4 * nblocks);
  *off_bw = *off_sbo + up16(4 * (nsuper + 1));
  *off_payload = *off_bw + up16(nblocks);
}

size_t orc_gl_bound(size_t n) {
  size_t nb = (n + 127) / 128, ns = (nb + 31) / 32;
  size_t a, b, c, p;
  gl_offsets(nb, ns, &a, &b, &c, &p);
  return p + nb * 512;
}

/* One block: the 128 values x[0..cnt) padded so that every missing delta is
 * zero, D4 deltas against the seed (F,F,F,F), F = x[0]; other kinds of
 * Section 5 likewise against F. */
static void gl_block_deltas(const uint32_t *x, unsigned cnt, int kind, uint32_t d[128]) {
  uint32_t xx[128];
  const uint32_t F = x[0];
  if (kind != ORC_DELTA_D4) {
    for (unsigned i = 0; i < 128; i++) xx[i] = i < cnt ? x[i] : delta_ref(kind, xx, i, F);
    orc_deltas(kind, xx, 128, F, d);
    return;
  }
  for (unsigned i = 0; i < 128; i++) {
    if (i < cnt) xx[i] = x[i];
    else xx[i] = (i >= 4) ? xx[i - 4] : F;
  }
  for (unsigned i = 0; i < 128; i++) d[i] = xx[i] - (i >= 4 ? xx[i - 4] : F);
}

static void put_bits(uint32_t *w, size_t pos, uint32_t v, unsigned b) {
  for (unsigned k = 0; k < b; k++)
    if ((v >> k) & 1u) w[(pos + k) / 32] |= 1u << ((pos + k) % 32);
}

static uint32_t get_bits(const uint32_t *w, size_t pos, unsigned b) {
  if (b == 0) return 0;
  const size_t k = pos / 32;
  const unsigned o = (unsigned)(pos % 32);
  uint64_t v = (uint64_t)w[k] >> o;
  if (o + b > 32) v |= (uint64_t)w[k + 1] << (32 - o);
  return (uint32_t)v & low_mask(b);
}

int orc_gl_encode(const uint32_t *x, size_t n, uint8_t *out, size_t cap,
                  size_t *out_bytes) {
  return orc_gl_encode_kind(x, n, ORC_DELTA_D4, out, cap, out_bytes);
}

int orc_gl_encode_kind(const uint32_t *x, size_t n, int kind, uint8_t *out,
                       size_t cap, size_t *out_bytes) {
  if ((!x && n) || !out || !out_bytes) return ORC_EARG;
  if (kind < ORC_DELTA_D4 || kind > ORC_DELTA_D1) return ORC_EARG;
  if (n > 0x7FFFFFFFull) return ORC_EARG;
  if (!is_sorted_distinct(x, n)) return ORC_EARG;
  if (cap < orc_gl_bound(n)) return ORC_ECAPACITY;

  const size_t nb = (n + 127) / 128, ns = (nb + 31) / 32;
  size_t off_first, off_sbo, off_bw, off_payload;
  gl_offsets(nb, ns, &off_first, &off_sbo, &off_bw, &off_payload);
  memset(out, 0, off_payload);

  size_t wpos = 0; /* payload word offset */
  uint32_t d[128], words[128];
  for (size_t k = 0; k < nb; k++) {
    const unsigned cnt = (unsigned)((n - 128 * k) < 128 ? (n - 128 * k) : 128);
    gl_block_deltas(x + 128 * k, cnt, kind, d);
    const unsigned b = orc_max_bits(d, 128);
    if (k % 32 == 0) wr32(out + off_sbo + 4 * (k / 32), (uint32_t)wpos);
    wr32(out + off_first + 4 * k, x[128 * k]);
    out[off_bw + k] = (uint8_t)b;
    for (unsigned q = 0; q < 4 * b; q++) words[q] = 0;
    for (unsigned t = 0; t < 32; t++)
      for (unsigned s = 0; s < 4; s++)
        put_bits(words, (size_t)b * (32 * s + t), d[4 * t + s], b);
    for (unsigned q = 0; q < 4 * b; q++)
      wr32(out + off_payload + 4 * (wpos + q), words[q]);
    wpos += 4 * b;
  }
  wr32(out + off_sbo + 4 * ns, (uint32_t)wpos);
  const size_t total = off_payload + 4 * wpos;

  uint32_t hdr[16] = {GL_MAGIC,
                      1u,
                      (uint32_t)n,
                      (uint32_t)nb,
                      (uint32_t)ns,
                      (uint32_t)wpos,
                      (uint32_t)off_first,
                      (uint32_t)off_sbo,
                      (uint32_t)off_bw,
                      (uint32_t)off_payload,
                      (uint32_t)(total & 0xFFFFFFFFu),
                      (uint32_t)((uint64_t)total >> 32),
                      (uint32_t)kind,
                      0,
                      0,
                      0};
  for (int i = 0; i < 16; i++) wr32(out + 4 * i, hdr[i]);
  *out_bytes = total;
  return ORC_OK;
}

int orc_gl_info(const uint8_t *in, size_t nbytes, uint32_t info[8]) {
  if (!in || !info) return ORC_EARG;
  if (nbytes < 64) return ORC_ECORRUPT;
  if (rd32(in) != GL_MAGIC || rd32(in + 4) != 1u) return ORC_ECORRUPT;
  const size_t n = rd32(in + 8), nb = rd32(in + 12), ns = rd32(in + 16);
  const size_t pw = rd32(in + 20);
  if (nb != (n + 127) / 128 || ns != (nb + 31) / 32) return ORC_ECORRUPT;
  size_t a, b, c, p;
  gl_offsets(nb, ns, &a, &b, &c, &p);
  if (rd32(in + 24) != a || rd32(in + 28) != b || rd32(in + 32) != c ||
      rd32(in + 36) != p)
    return ORC_ECORRUPT;
  const uint64_t total = (uint64_t)rd32(in + 40) | ((uint64_t)rd32(in + 44) << 32);
  if (total != p + 4 * pw || total > nbytes) return ORC_ECORRUPT;
  info[0] = (uint32_t)n;
  info[1] = (uint32_t)nb;
  info[2] = (uint32_t)ns;
  info[3] = (uint32_t)pw;
  info[4] = (uint32_t)a;
  info[5] = (uint32_t)b;
  info[6] = (uint32_t)c;
  info[7] = (uint32_t)p;
  return ORC_OK;
}

int orc_gl_decode(const uint8_t *in, size_t nbytes, uint32_t *out, size_t cap,
                  size_t *n_out) {
  uint32_t info[8];
  if (!n_out) return ORC_EARG;
  int rc = orc_gl_info(in, nbytes, info);
  if (rc) return rc;
  const size_t n = info[0], nb = info[1], ns = info[2], pw = info[3];
  *n_out = n;
  if (n > cap) return ORC_ECAPACITY;
  if (n && !out) return ORC_EARG;
  const uint8_t *first = in + info[4], *sbo = in + info[5], *bw = in + info[6];
  const uint32_t kind = rd32(in + 48);
  if (kind > ORC_DELTA_D1) return ORC_ECORRUPT;

  uint32_t *payload = (uint32_t *)malloc((pw + 1) * sizeof(uint32_t));
  if (!payload) return ORC_EARG;
  for (size_t q = 0; q < pw; q++) payload[q] = rd32(in + info[7] + 4 * q);
  payload[pw] = 0;

  rc = ORC_OK;
  for (size_t sb = 0; sb < ns && rc == ORC_OK; sb++) {
    size_t wpos = rd32(sbo + 4 * sb);
    for (size_t k = 32 * sb; k < nb && k < 32 * sb + 32; k++) {
      const unsigned b = bw[k];
      if (b > 32 || wpos + 4 * (size_t)b > pw) {
        rc = ORC_ECORRUPT;
        break;
      }
      const uint32_t F = rd32(first + 4 * k);
      uint32_t x[128];
      if (kind == ORC_DELTA_D4) {
        for (unsigned t = 0; t < 32; t++)
          for (unsigned s = 0; s < 4; s++) {
            uint32_t delta = get_bits(payload + wpos, (size_t)b * (32 * s + t), b);
            uint32_t prev = (t == 0) ? F : x[4 * (t - 1) + s];
            x[4 * t + s] = prev + delta;
          }
      } else {
        uint32_t d[128];
        for (unsigned t = 0; t < 32; t++)
          for (unsigned s = 0; s < 4; s++)
            d[4 * t + s] = get_bits(payload + wpos, (size_t)b * (32 * s + t), b);
        orc_prefix((int)kind, d, 128, F, x);
      }
      const size_t cnt = (n - 128 * k) < 128 ? (n - 128 * k) : 128;
      for (size_t i = 0; i < cnt; i++) out[128 * k + i] = x[i];
      wpos += 4 * (size_t)b;
    }
    if (rc == ORC_OK && rd32(sbo + 4 * (sb + 1)) != wpos) rc = ORC_ECORRUPT;
  }
  free(payload);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* S4-FastPFOR (Section 4.4, Fig. 3) in a GPU layout (GP).  Not the        */
/* paper's byte format: blocks of 128 deltas (any kind of Section 5, each  */
/* block restarting from its first value F as in GL) are bit packed at a   */
/* width b' <= b, the deltas >= 2^b' are exceptions whose positions (one   */
/* byte each) and b - b' high bits are stored per page of 32 blocks.       */
/*                                                                          */
/* header, 16 little-endian u32 words:                                      */
/*   0 magic 0x34504742   1 layout tag 3     2 n          3 nblocks        */
/*   4 npages             5 payload words    6 off_first  7 off_spo        */
/*   8 off_meta           9 off_payload     10 total bytes (low)           */
/*  11 total bytes (high) 12 kind            13..15 zero                   */
/* sections, each starting on a 16-byte boundary:                           */
/*   first[nblocks] u32, spo[npages+1] u32 (payload word offset of every   */
/*   page, then the total), meta[nblocks] of 4 bytes {b', b - b', c, 0}    */
/*   (c = number of exceptions), payload words.                             */
/* page p (blocks 32p ..): the low b' bits of every block, 4 b' words per   */
/*   block in GL's column order; then the exception positions, c bytes per  */
/*   block in ascending order, zero-padded to a word; then the high bits,   */
/*   b - b' per exception, blocks and exceptions in order, least           */
/*   significant bit first, zero-padded to a word; then zero words to a     */
/*   multiple of 4.                                                         */
/* ------------------------------------------------------------------------ */

#define GP_MAGIC 0x34504742u

static void gp_offsets(size_t nblocks, size_t npages, size_t *off_first,
                       size_t *off_spo, size_t *off_meta, size_t *off_payload) {
  *off_first = 64;
  *off_spo = *off_first + up16(4 * nblocks);
  *off_meta = *off_spo + up16(4 * (npages + 1));
  *off_payload = *off_meta + up16(4 * nblocks);
}

size_t orc_gp_bound(size_t n) {
  size_t nb = (n + 127) / 128, np = (nb + 31) / 32;
  size_t a, b, c, p;
  gp_offsets(nb, np, &a, &b, &c, &p);
  /* a block never costs more bits than at b' = b (128 b <= 4096); a page
   * adds less than 5 words of padding (positions, high bits, 4-word end) */
  return p + nb * 512 + np * 32;
}

/* Section 4.4: b is the width of the largest delta; b' in [0, b] minimizes
 * 128 b' + c(b') (b - b' + 8), c(b') = number of deltas >= 2^b'.  Where
 * several b' tie, the largest is taken (fewer exceptions; the paper does
 * not say). */
void orc_pfor_choose(const uint32_t d[128], unsigned *b_out, unsigned *bp_out,
                     unsigned *c_out) {
  const unsigned b = orc_max_bits(d, 128);
  unsigned best = b, best_c = 0;
  uint64_t best_cost = 128ull * b;
  for (unsigned bp = 0; bp < b; bp++) {
    unsigned c = 0;
    for (unsigned i = 0; i < 128; i++)
      if (orc_bits(d[i]) > bp) c++;
    const uint64_t cost = 128ull * bp + (uint64_t)c * (b - bp + 8);
    if (cost < best_cost) {
      best_cost = cost;
      best = bp;
      best_c = c;
    }
  }
  /* ties: a later (larger) b' with the same cost wins */
  for (unsigned bp = best + 1; bp <= b; bp++) {
    unsigned c = 0;
    for (unsigned i = 0; i < 128; i++)
      if (orc_bits(d[i]) > bp) c++;
    if (128ull * bp + (uint64_t)c * (b - bp + 8) == best_cost) {
      best = bp;
      best_c = c;
    }
  }
  *b_out = b;
  *bp_out = best;
  *c_out = best_c;
}

int orc_gp_encode_kind(const uint32_t *x, size_t n, int kind, uint8_t *out,
                       size_t cap, size_t *out_bytes) {
  if ((!x && n) || !out || !out_bytes) return ORC_EARG;
  if (kind < ORC_DELTA_D4 || kind > ORC_DELTA_D1) return ORC_EARG;
  if (n > 0x7FFFFFFFull) return ORC_EARG;
  if (!is_sorted_distinct(x, n)) return ORC_EARG;
  if (cap < orc_gp_bound(n)) return ORC_ECAPACITY;

  const size_t nb = (n + 127) / 128, np = (nb + 31) / 32;
  size_t off_first, off_spo, off_meta, off_payload;
  gp_offsets(nb, np, &off_first, &off_spo, &off_meta, &off_payload);
  memset(out, 0, cap);

  size_t wpos = 0; /* payload word offset */
  uint32_t d[128];
  for (size_t p = 0; p < np; p++) {
    wr32(out + off_spo + 4 * p, (uint32_t)wpos);
    const size_t k0 = 32 * p, k1 = (k0 + 32 < nb) ? k0 + 32 : nb;
    /* pass over the page's blocks: low bits, then collect the exceptions */
    uint8_t pos[32 * 128];
    uint32_t high[32 * 128];
    unsigned hw[32 * 128];
    size_t ne = 0;
    for (size_t k = k0; k < k1; k++) {
      const unsigned cnt = (unsigned)((n - 128 * k) < 128 ? (n - 128 * k) : 128);
      gl_block_deltas(x + 128 * k, cnt, kind, d);
      unsigned b, bp, c;
      orc_pfor_choose(d, &b, &bp, &c);
      wr32(out + off_first + 4 * k, x[128 * k]);
      out[off_meta + 4 * k + 0] = (uint8_t)bp;
      out[off_meta + 4 * k + 1] = (uint8_t)(b - bp);
      out[off_meta + 4 * k + 2] = (uint8_t)c;
      uint32_t words[128];
      for (unsigned q = 0; q < 4 * bp; q++) words[q] = 0;
      for (unsigned t = 0; t < 32; t++)
        for (unsigned s = 0; s < 4; s++)
          put_bits(words, (size_t)bp * (32 * s + t), d[4 * t + s] & low_mask(bp), bp);
      for (unsigned q = 0; q < 4 * bp; q++)
        wr32(out + off_payload + 4 * (wpos + q), words[q]);
      wpos += 4 * bp;
      for (unsigned i = 0; i < 128; i++)
        if (orc_bits(d[i]) > bp) {
          pos[ne] = (uint8_t)i;
          high[ne] = d[i] >> bp; /* bp < b <= 32 here */
          hw[ne] = b - bp;
          ne++;
        }
    }
    for (size_t e = 0; e < ne; e++) out[off_payload + 4 * wpos + e] = pos[e];
    wpos += (ne + 3) / 4;
    size_t hbits = 0;
    for (size_t e = 0; e < ne; e++) hbits += hw[e];
    uint32_t *hwords = (uint32_t *)calloc((hbits + 31) / 32 + 1, sizeof(uint32_t));
    if (!hwords) return ORC_EARG;
    size_t bit = 0;
    for (size_t e = 0; e < ne; e++) {
      put_bits(hwords, bit, high[e], hw[e]);
      bit += hw[e];
    }
    for (size_t q = 0; q < (hbits + 31) / 32; q++)
      wr32(out + off_payload + 4 * (wpos + q), hwords[q]);
    free(hwords);
    wpos += (hbits + 31) / 32;
    wpos = (wpos + 3) & ~(size_t)3;
  }
  wr32(out + off_spo + 4 * np, (uint32_t)wpos);
  const size_t total = off_payload + 4 * wpos;
  const uint32_t hdr[16] = {GP_MAGIC,
                            3u,
                            (uint32_t)n,
                            (uint32_t)nb,
                            (uint32_t)np,
                            (uint32_t)wpos,
                            (uint32_t)off_first,
                            (uint32_t)off_spo,
                            (uint32_t)off_meta,
                            (uint32_t)off_payload,
                            (uint32_t)(total & 0xFFFFFFFFu),
                            (uint32_t)((uint64_t)total >> 32),
                            (uint32_t)kind,
                            0,
                            0,
                            0};
  for (int i = 0; i < 16; i++) wr32(out + 4 * i, hdr[i]);
  *out_bytes = total;
  return ORC_OK;
}

int orc_gp_decode(const uint8_t *in, size_t nbytes, uint32_t *out, size_t cap,
                  size_t *n_out) {
  if (!in || !n_out) return ORC_EARG;
  if (nbytes < 64) return ORC_ECORRUPT;
  if (rd32(in) != GP_MAGIC || rd32(in + 4) != 3u) return ORC_ECORRUPT;
  const size_t n = rd32(in + 8), nb = rd32(in + 12), np = rd32(in + 16);
  const size_t pw = rd32(in + 20);
  const uint32_t kind = rd32(in + 48);
  if (nb != (n + 127) / 128 || np != (nb + 31) / 32 || kind > ORC_DELTA_D1)
    return ORC_ECORRUPT;
  size_t off_first, off_spo, off_meta, off_payload;
  gp_offsets(nb, np, &off_first, &off_spo, &off_meta, &off_payload);
  if (rd32(in + 24) != off_first || rd32(in + 28) != off_spo ||
      rd32(in + 32) != off_meta || rd32(in + 36) != off_payload)
    return ORC_ECORRUPT;
  const uint64_t total = (uint64_t)rd32(in + 40) | ((uint64_t)rd32(in + 44) << 32);
  if (total != off_payload + 4 * pw || total > nbytes) return ORC_ECORRUPT;
  *n_out = n;
  if (n > cap) return ORC_ECAPACITY;
  if (n && !out) return ORC_EARG;

  uint32_t *payload = (uint32_t *)malloc((pw + 1) * sizeof(uint32_t));
  if (!payload) return ORC_EARG;
  for (size_t q = 0; q < pw; q++) payload[q] = rd32(in + off_payload + 4 * q);
  payload[pw] = 0;
  int rc = ORC_OK;
  for (size_t p = 0; p < np && rc == ORC_OK; p++) {
    const size_t k0 = 32 * p, k1 = (k0 + 32 < nb) ? k0 + 32 : nb;
    const size_t page = rd32(in + off_spo + 4 * p), page_end = rd32(in + off_spo + 4 * (p + 1));
    /* where the page's positions and high bits start */
    size_t low = 0, ne = 0, hbits = 0;
    for (size_t k = k0; k < k1; k++) {
      const unsigned bp = in[off_meta + 4 * k], w = in[off_meta + 4 * k + 1];
      const unsigned c = in[off_meta + 4 * k + 2];
      if (bp + w > 32 || (w == 0) != (c == 0) || c > 128) {
        rc = ORC_ECORRUPT;
        break;
      }
      low += 4 * bp;
      ne += c;
      hbits += (size_t)c * w;
    }
    const size_t pos_w = page + low, high_w = pos_w + (ne + 3) / 4;
    const size_t end = (high_w + (hbits + 31) / 32 + 3) & ~(size_t)3;
    if (rc || end != page_end || page_end > pw) {
      rc = ORC_ECORRUPT;
      break;
    }
    const uint8_t *posb = in + off_payload + 4 * pos_w;
    size_t wpos = page, e = 0, bit = 0;
    for (size_t k = k0; k < k1; k++) {
      const unsigned bp = in[off_meta + 4 * k], w = in[off_meta + 4 * k + 1];
      const unsigned c = in[off_meta + 4 * k + 2];
      uint32_t d[128];
      /* unpack b' bits, patch the exceptions, then the prefix (Section 4.4:
       * unpacking, patching and the prefix sum in that order) */
      for (unsigned t = 0; t < 32; t++)
        for (unsigned s = 0; s < 4; s++)
          d[4 * t + s] = get_bits(payload + wpos, (size_t)bp * (32 * s + t), bp);
      for (unsigned i = 0; i < c; i++, e++) {
        const unsigned q = posb[e];
        if (q > 127) {
          rc = ORC_ECORRUPT;
          break;
        }
        d[q] |= get_bits(payload + high_w, bit, w) << bp;
        bit += w;
      }
      if (rc) break;
      uint32_t x[128];
      orc_prefix((int)kind, d, 128, rd32(in + off_first + 4 * k), x);
      const size_t cnt = (n - 128 * k) < 128 ? (n - 128 * k) : 128;
      for (size_t i = 0; i < cnt; i++) out[128 * k + i] = x[i];
      wpos += 4 * (size_t)bp;
    }
  }
  free(payload);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Section 6: intersections of sorted lists of distinct integers.          */
/* ------------------------------------------------------------------------ */

size_t orc_intersect_merge(const uint32_t *a, size_t na, const uint32_t *b,
                           size_t nb, uint32_t *out) {
  size_t i = 0, j = 0, k = 0;
  while (i < na && j < nb) {
    if (a[i] < b[j]) i++;
    else if (a[i] > b[j]) j++;
    else {
      uint32_t v = a[i];
      out[k++] = v;
      i++;
      j++;
    }
  }
  return k;
}

/* Galloping: for each value of the short list r, probe the long list f at
 * the next position, then twice as far each time, until a value >= r_i is
 * seen; then binary search between the last two probes for the first value
 * >= r_i, and advance there. */
size_t orc_intersect_gallop(const uint32_t *a, size_t na, const uint32_t *b,
                            size_t nb, uint32_t *out) {
  const uint32_t *r = na <= nb ? a : b, *f = na <= nb ? b : a;
  const size_t nr = na <= nb ? na : nb, nf = na <= nb ? nb : na;
  size_t j = 0, k = 0;
  for (size_t i = 0; i < nr && j < nf; i++) {
    const uint32_t ri = r[i];
    if (f[j] < ri) {
      size_t lo = j, step = 1; /* invariant: f[lo] < ri */
      size_t hi = j + step;
      while (hi < nf && f[hi] < ri) {
        lo = hi;
        step *= 2;
        hi = j + step;
      }
      if (hi > nf) hi = nf; /* hi == nf means "past the end" */
      /* first index in (lo, hi] with f >= ri, or nf */
      size_t L = lo + 1, H = hi;
      while (L < H) {
        size_t mid = L + (H - L) / 2;
        if (f[mid] < ri) L = mid + 1;
        else H = mid;
      }
      j = L;
      if (j >= nf) break;
    }
    if (f[j] == ri) {
      out[k++] = ri;
      j++;
    }
  }
  return k;
}

static int any_equal(const uint32_t *F, unsigned T, uint32_t r) {
  int hit = 0;
  for (unsigned t = 0; t < T; t++) hit |= (F[t] == r);
  return hit;
}

/* Algorithm 2 (V1): advance in the long list by whole T-blocks until the
 * last value of the block is >= r_i, then compare r_i with all T values. */
size_t orc_intersect_v1(const uint32_t *r, size_t nr, const uint32_t *f,
                        size_t nf, unsigned T, uint32_t *out) {
  const size_t nfp = nf / T * T;
  size_t j = 0, k = 0, i = 0;
  for (; i < nr; i++) {
    while (j < nfp && f[j + T - 1] < r[i]) j += T;
    if (j >= nfp) break;
    if (any_equal(f + j, T, r[i])) out[k++] = r[i];
  }
  /* scalar completion over the part of f beyond the last whole block */
  return k + orc_intersect_merge(r + i, nr - i, f + nfp, nf - nfp, out + k);
}

/* Algorithm 3 (V3): skip by 4T-blocks, pick one T-block of the four with two
 * comparisons, compare r_i with its T values.  The printed indices of the
 * second and fourth choices are read as contiguous T-blocks. */
size_t orc_intersect_v3(const uint32_t *r, size_t nr, const uint32_t *f,
                        size_t nf, unsigned T, uint32_t *out) {
  const size_t Q = 4 * (size_t)T, nfp = nf / Q * Q;
  size_t j = 0, k = 0, i = 0;
  for (; i < nr; i++) {
    const uint32_t ri = r[i];
    while (j < nfp && f[j + Q - 1] < ri) j += Q;
    if (j >= nfp) break;
    const uint32_t *F;
    if (f[j + 2 * T - 1] >= ri) F = (f[j + T - 1] >= ri) ? f + j : f + j + T;
    else F = (f[j + 3 * T - 1] >= ri) ? f + j + 2 * T : f + j + 3 * T;
    if (any_equal(F, T, ri)) out[k++] = ri;
  }
  return k + orc_intersect_merge(r + i, nr - i, f + nfp, nf - nfp, out + k);
}

/* Algorithm 4 (SIMD Galloping): find by sequential search the smallest delta
 * in 0, T, 2T, 4T, ... (the last candidate clamped to the last whole T-block)
 * with f[j+delta+T-1] >= r_i, then by binary search the smallest multiple of
 * T in [delta/2, delta] with the same property; compare r_i with that
 * T-block. */
size_t orc_intersect_simd_gallop(const uint32_t *r, size_t nr,
                                 const uint32_t *f, size_t nf, unsigned T,
                                 uint32_t *out) {
  const size_t nfp = nf / T * T;
  size_t j = 0, k = 0, i = 0;
  for (; i < nr; i++) {
    const uint32_t ri = r[i];
    if (j >= nfp) break;
    const size_t last = nfp - T - j; /* largest admissible delta */
    size_t delta = 0;
    int found = 0;
    for (size_t cand = 0;; cand = (cand == 0) ? T : 2 * cand) {
      size_t c = cand > last ? last : cand;
      if (f[j + c + T - 1] >= ri) {
        delta = c;
        found = 1;
        break;
      }
      if (c == last) break;
    }
    if (!found) break;
    size_t lo = (delta / 2 + T - 1) / T, hi = delta / T; /* in units of T */
    while (lo < hi) {
      size_t mid = lo + (hi - lo) / 2;
      if (f[j + mid * T + T - 1] >= ri) hi = mid;
      else lo = mid + 1;
    }
    j += lo * T;
    if (any_equal(f + j, T, ri)) out[k++] = ri;
  }
  return k + orc_intersect_merge(r + i, nr - i, f + nfp, nf - nfp, out + k);
}

size_t orc_intersect_hybrid(const uint32_t *a, size_t na, const uint32_t *b,
                            size_t nb, uint32_t *out) {
  const uint32_t *r = na <= nb ? a : b, *f = na <= nb ? b : a;
  const size_t nr = na <= nb ? na : nb, nf = na <= nb ? nb : na;
  if (nr == 0) return 0;
  if (nf < 50 * nr) return orc_intersect_v1(r, nr, f, nf, 8, out);
  if (nf < 1000 * nr) return orc_intersect_v3(r, nr, f, nf, 32, out);
  return orc_intersect_simd_gallop(r, nr, f, nf, 32, out);
}

/* Set-vs-Set: lists in order of non-decreasing cardinality, the running
 * result intersected with each next list (written back in place). */
size_t orc_svs(const uint32_t *const *lists, const size_t *lens, size_t k,
               uint32_t *out) {
  if (k == 0) return 0;
  size_t *ord = (size_t *)malloc(k * sizeof(size_t));
  if (!ord) return 0;
  for (size_t i = 0; i < k; i++) ord[i] = i;
  for (size_t i = 1; i < k; i++) { /* insertion sort by length, stable */
    size_t t = ord[i], p = i;
    while (p > 0 && lens[ord[p - 1]] > lens[t]) {
      ord[p] = ord[p - 1];
      p--;
    }
    ord[p] = t;
  }
  size_t n = lens[ord[0]];
  memcpy(out, lists[ord[0]], n * sizeof(uint32_t));
  for (size_t i = 1; i < k && n > 0; i++)
    n = orc_intersect_merge(out, n, lists[ord[i]], lens[ord[i]], out);
  free(ord);
  return n;
}
