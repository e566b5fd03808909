/*
 * bp_oracle.h -- scalar reference implementation of S4-BP128-D4 coding and
 * sorted-list intersection (Lemire, Boytsov, Kurz, "SIMD Compression and the
 * Intersection of Sorted Integers", arXiv 1401.6399).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the oracle that the CUDA path is
 * checked against.  It is plain, slow, obviously-correct scalar C.  It shares
 * no code, header, table or helper with the CUDA library; only tests/, the
 * smoke check and the CPU-baseline leg of the benchmark may load it.
 *
 * Every function cites the passage of the paper it follows.  Where the paper
 * is silent the reading taken is stated next to the function.
 *
 * Error convention: functions returning int give 0 on success and a positive
 * ORC_E* code on failure.
 */
#ifndef BP_ORACLE_H
#define BP_ORACLE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  ORC_OK = 0,
  ORC_EARG = 1,      /* bad argument (null pointer, unsorted list, ...) */
  ORC_ECORRUPT = 3,  /* malformed stream (width > 32, truncated, ...)   */
  ORC_ECAPACITY = 4  /* output buffer too small                         */
};

/* ---- bit widths (Section 4.3) ------------------------------------------ */

/* Smallest b such that v < 2^b (0 for v == 0); range 0..32. */
unsigned orc_bits(uint32_t v);
/* Smallest b such that every v[i] < 2^b. */
unsigned orc_max_bits(const uint32_t *v, size_t n);

/* ---- bit packing (Section 4.2) ----------------------------------------- */

/* Consecutive (scalar) layout of Fig. 1c: value i occupies bits
 * [i*b, (i+1)*b) of a little-endian bit string, least significant bit first.
 * out receives ceil(n*b/8) bytes (zeroed first). */
void orc_pack_scalar(const uint32_t *in, size_t n, unsigned b, uint8_t *out);
void orc_unpack_scalar(const uint8_t *in, size_t n, unsigned b, uint32_t *out);

/* 4-lane interleaved layout of Fig. 2: integer n of the 128-block goes to
 * lane n mod 4, slot n div 4; lane s is a b-bit-per-value LSB-first stream
 * over the words y[4k+s], k = 0..b-1.  out receives 4*b words. */
void orc_s4_pack128(const uint32_t in[128], unsigned b, uint32_t *out);

/* Algorithm 1: unpack 128 integers from 4*b words with an integrated prefix
 * function P.  kind = ORC_P_NONE gives P(t,v) = t (plain unpack);
 * kind = ORC_P_D4 gives P(t,v) = t + v (D4, Section 5).  v is the 4-int
 * seed vector, updated in place to the last 4 outputs. */
enum { ORC_P_NONE = 0, ORC_P_D4 = 1, ORC_P_DM = 2, ORC_P_D2 = 3, ORC_P_D1 = 4 };
/* ORC_P_DM, ORC_P_D2, ORC_P_D1 apply the vector prefix steps Section 5 gives
 * for DM, D2 and D1 (v: the previous output vector). */
void orc_s4_unpack128(const uint32_t *y, unsigned b, int kind, uint32_t v[4],
                      uint32_t out[128]);

/* ---- differential coding (Section 5) ------------------------------------ */

/* D4 deltas: d[i] = x[i] - x[i-4] (mod 2^32) with x[-4..-1] = 0. */
void orc_d4_deltas(const uint32_t *x, size_t n, uint32_t *d);
/* Inverse: x[i] = d[i] + x[i-4]. */
void orc_d4_prefix(const uint32_t *d, size_t n, uint32_t *x);

/* The four kinds of differential coding of Section 5, as stored in stream
 * headers: D4 d[i] = x[i] - x[i-4]; DM d[4t+s] = x[4t+s] - x[4t-1] (every
 * 4-vector minus the last value of the previous one); D2 d[i] = x[i] - x[i-2];
 * D1 d[i] = x[i] - x[i-1].  Positions before x[0] hold `seed`. */
enum { ORC_DELTA_D4 = 0, ORC_DELTA_DM = 1, ORC_DELTA_D2 = 2, ORC_DELTA_D1 = 3 };
void orc_deltas(int kind, const uint32_t *x, size_t n, uint32_t seed, uint32_t *d);
/* Inverse of orc_deltas. */
void orc_prefix(int kind, const uint32_t *d, size_t n, uint32_t seed, uint32_t *x);

/* ---- varint (Section 4.1, Fig. 1b) --------------------------------------- */

/* 7-bit groups, least significant group first; the byte that ends an integer
 * has its most significant bit set.  Returns bytes written (<= 5n). */
size_t orc_varint_encode(const uint32_t *in, size_t n, uint8_t *out);
/* Decodes exactly n integers from at most nbytes bytes; *used = bytes read. */
int orc_varint_decode(const uint8_t *in, size_t nbytes, size_t n,
                      uint32_t *out, size_t *used);

/* ---- S4-BP128-D4 container, paper layout "PL" (Section 4.3) ------------- *
 * header   16 bytes: u32 n, u32 layout tag (0), u32 tail_bytes, u32 kind of
 *          differential coding (ORC_DELTA_*, 0 = D4)
 * then     floor(nb/16) meta-blocks: 16 width bytes, then 16 packed blocks
 * then     nb mod 16 leftover blocks: 1 width byte, then the packed block
 * then     the n mod 128 remaining integers as varint of D1 gaps from the
 *          previous integer (0 before the first)
 * where nb = floor(n/128) and blocks hold D4 (or DM, D2, D1) deltas carried
 * across blocks. */
size_t orc_pl_bound(size_t n);
int orc_pl_encode(const uint32_t *x, size_t n, uint8_t *out, size_t cap,
                  size_t *out_bytes);
int orc_pl_encode_kind(const uint32_t *x, size_t n, int kind, uint8_t *out,
                       size_t cap, size_t *out_bytes);
/* Reads n from the header; fails with ORC_ECAPACITY if n > cap. */
int orc_pl_decode(const uint8_t *in, size_t nbytes, uint32_t *out, size_t cap,
                  size_t *n_out);
/* n stored in a PL or GL header (no validation beyond the size). */
int orc_stream_count(const uint8_t *in, size_t nbytes, size_t *n_out);

/* ---- GPU layout "GL" (not in the paper; our format) -------------------- *
 * header 64 bytes (see bp_oracle.c); per block k of 128 integers:
 *   first[k] = x[128k]; D4 restarts at each block with seed (F,F,F,F),
 *   F = first[k]; the last block is padded with zero deltas;
 *   bw[k] = bit width; the block's 4*bw[k] words hold the 128 deltas in
 *   column-major order: delta of in-block position 4t+s (row t, column s)
 *   at bit bw*(32s+t) of the block's LSB-first bit string;
 *   sbo[q] = word offset of block 32q in the payload (q <= nsuper).
 * Header word 12 holds the kind of differential coding (ORC_DELTA_*); for
 * DM, D2 and D1 the block's deltas are taken the same way against the seed
 * F, and padding again makes the missing deltas zero. */
size_t orc_gl_bound(size_t n);
int orc_gl_encode(const uint32_t *x, size_t n, uint8_t *out, size_t cap,
                  size_t *out_bytes);
int orc_gl_encode_kind(const uint32_t *x, size_t n, int kind, uint8_t *out,
                       size_t cap, size_t *out_bytes);
int orc_gl_decode(const uint8_t *in, size_t nbytes, uint32_t *out, size_t cap,
                  size_t *n_out);
/* Header fields of a GL stream: nblocks, offsets of first[], sbo[], bw[],
 * payload (bytes from the start of the stream). */
int orc_gl_info(const uint8_t *in, size_t nbytes, uint32_t info[8]);

/* ---- S4-FastPFOR in a GPU layout, GP (Section 4.4, Fig. 3) --------------- *
 * Blocks of 128 deltas as in GL (any kind, restarting from the block's first
 * value F); each block is bit packed at a width b' <= b and the deltas
 * >= 2^b' are exceptions: their in-block positions (a byte each) and their
 * b - b' high bits are stored after the low bits of each page of 32 blocks.
 * Layout: bp_oracle.c.  Decoding unpacks, patches, then takes the prefix. */
size_t orc_gp_bound(size_t n);
/* The widths of one block of deltas (Section 4.4): b = orc_max_bits, b' the
 * minimizer of 128 b' + c(b') (b - b' + 8) (largest b' on a tie), c = c(b'),
 * the number of deltas >= 2^b'. */
void orc_pfor_choose(const uint32_t d[128], unsigned *b, unsigned *bp, unsigned *c);
int orc_gp_encode_kind(const uint32_t *x, size_t n, int kind, uint8_t *out,
                       size_t cap, size_t *out_bytes);
int orc_gp_decode(const uint8_t *in, size_t nbytes, uint32_t *out, size_t cap,
                  size_t *n_out);

/* ---- intersections (Section 6) ------------------------------------------- */

/* Textbook merge ("scalar"), O(m+n).  out may alias the shorter input. */
size_t orc_intersect_merge(const uint32_t *a, size_t na, const uint32_t *b,
                           size_t nb, uint32_t *out);
/* Galloping (exponential) search of each element of the shorter list. */
size_t orc_intersect_gallop(const uint32_t *a, size_t na, const uint32_t *b,
                            size_t nb, uint32_t *out);
/* Algorithm 2 (V1), Algorithm 3 (V3) and Algorithm 4 (SIMD Galloping) with
 * T-wide comparisons emulated by scalar loops; any part of the long list
 * beyond a multiple of T (or 4T) is finished with the merge. */
size_t orc_intersect_v1(const uint32_t *r, size_t nr, const uint32_t *f,
                        size_t nf, unsigned T, uint32_t *out);
size_t orc_intersect_v3(const uint32_t *r, size_t nr, const uint32_t *f,
                        size_t nf, unsigned T, uint32_t *out);
size_t orc_intersect_simd_gallop(const uint32_t *r, size_t nr,
                                 const uint32_t *f, size_t nf, unsigned T,
                                 uint32_t *out);
/* The hybrid of Section 6.2.1: V1 (T=8) below ratio 50, V3 (T=32) below
 * 1000, SIMD Galloping (T=32) above. */
size_t orc_intersect_hybrid(const uint32_t *a, size_t na, const uint32_t *b,
                            size_t nb, uint32_t *out);
/* Set-vs-Set over k lists: order by cardinality, intersect the two
 * smallest, then the result with each next list.  out needs the length of
 * the shortest list. */
size_t orc_svs(const uint32_t *const *lists, const size_t *lens, size_t k,
               uint32_t *out);

#ifdef __cplusplus
}
#endif
#endif
