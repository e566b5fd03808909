/*
 * gen.c -- seeded synthetic inputs shaped like the paper's workloads.
 *
 * This module holds no coding or intersection arithmetic: it only draws
 * sorted lists of distinct uint32 values and query term sets.  Both the
 * oracle and the CUDA path consume its output.
 *
 * Random numbers: xoshiro256** seeded through splitmix64 (Blackman and
 * Vigna), written from the published definitions.  Bounded draws use
 * Lemire's multiply-and-reject method, so results are exact and identical
 * on every platform.  No floating point is used.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  uint64_t s[4];
} rng_t;

static uint64_t splitmix64(uint64_t *x) {
  uint64_t z = (*x += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

static void rng_seed(rng_t *r, uint64_t seed) {
  uint64_t x = seed;
  for (int i = 0; i < 4; i++) r->s[i] = splitmix64(&x);
}

static inline uint64_t rotl(uint64_t x, int k) {
  return (x << k) | (x >> (64 - k));
}

static uint64_t rng_next(rng_t *r) {
  uint64_t *s = r->s;
  const uint64_t out = rotl(s[1] * 5, 7) * 9;
  const uint64_t t = s[1] << 17;
  s[2] ^= s[0];
  s[3] ^= s[1];
  s[1] ^= s[2];
  s[0] ^= s[3];
  s[2] ^= t;
  s[3] = rotl(s[3], 45);
  return out;
}

/* uniform integer in [0, range), range >= 1 */
static uint64_t below(rng_t *r, uint64_t range) {
  uint64_t x = rng_next(r);
  __uint128_t m = (__uint128_t)x * range;
  uint64_t l = (uint64_t)m;
  if (l < range) {
    uint64_t t = (0 - range) % range;
    while (l < t) {
      x = rng_next(r);
      m = (__uint128_t)x * range;
      l = (uint64_t)m;
    }
  }
  return (uint64_t)(m >> 64);
}

static int cmp_u32(const void *a, const void *b) {
  uint32_t x = *(const uint32_t *)a, y = *(const uint32_t *)b;
  return (x > y) - (x < y);
}

/* ---- uniform sample without replacement ------------------------------- */

/* n distinct values of [lo, hi), ascending.  Dense ranges use a bitmap
 * (marking the complement when n > half the range); sparse ones use
 * Floyd's algorithm with an open-addressing set, then a sort. */
static int uniform_into(rng_t *r, uint64_t n, uint64_t lo, uint64_t hi,
                        uint32_t *out) {
  const uint64_t R = hi - lo;
  if (n == 0) return 0;
  if (n > R) return 1;
  if (R <= (1ull << 31) && (n * 64 >= R || R <= (1ull << 22))) {
    const int flip = n * 2 > R;
    const uint64_t want = flip ? R - n : n;
    uint64_t *bm = (uint64_t *)calloc((R + 63) / 64, 8);
    if (!bm) return 2;
    uint64_t have = 0;
    while (have < want) {
      uint64_t v = below(r, R);
      uint64_t bit = 1ull << (v & 63);
      if (!(bm[v >> 6] & bit)) {
        bm[v >> 6] |= bit;
        have++;
      }
    }
    uint64_t k = 0;
    const uint64_t nw = (R + 63) / 64;
    for (uint64_t w = 0; w < nw; w++) {
      uint64_t bits = flip ? ~bm[w] : bm[w];
      if (w == nw - 1 && (R & 63)) bits &= (1ull << (R & 63)) - 1;
      while (bits) {
        out[k++] = (uint32_t)(lo + 64 * w + (uint64_t)__builtin_ctzll(bits));
        bits &= bits - 1;
      }
    }
    free(bm);
    return 0;
  }
  uint64_t cap = 16;
  while (cap < 2 * n) cap *= 2;
  uint64_t *tab = (uint64_t *)malloc(cap * 8);
  if (!tab) return 2;
  memset(tab, 0xFF, cap * 8);
  uint64_t k = 0;
  for (uint64_t j = R - n; j < R; j++) {
    uint64_t t = below(r, j + 1);
    /* insert t, or j if t is present */
    for (int pass = 0; pass < 2; pass++) {
      uint64_t v = pass ? j : t;
      uint64_t h = (v * 0x9E3779B97F4A7C15ull) & (cap - 1);
      int present = 0;
      while (tab[h] != ~0ull) {
        if (tab[h] == v) {
          present = 1;
          break;
        }
        h = (h + 1) & (cap - 1);
      }
      if (!present) {
        tab[h] = v;
        out[k++] = (uint32_t)(lo + v);
        break;
      }
    }
  }
  free(tab);
  qsort(out, n, sizeof(uint32_t), cmp_u32);
  return 0;
}

int wl_uniform(uint64_t n, uint64_t lo, uint64_t hi, uint64_t seed,
               uint32_t *out) {
  rng_t r;
  rng_seed(&r, seed);
  if (hi > (1ull << 32) || lo > hi) return 1;
  return uniform_into(&r, n, lo, hi, out);
}

/* ---- clustered generator ------------------------------------------------ *
 * Recursive interval splitting.  A node (n values in [lo, hi)) whose range
 * is at most 2n wide, or that is 24 levels deep, draws its values uniformly.
 * Otherwise, with probability 1/2 it narrows to a random sub-interval of
 * random width in [2n, hi-lo) (a cluster), and with probability 1/2 it cuts
 * the range at a uniform point and gives each side a share of n in
 * proportion to its width (randomised rounding), then recurses on both.  The
 * result has runs of small gaps separated by occasional large ones.
 */
static int clustered_rec(rng_t *r, uint64_t n, uint64_t lo, uint64_t hi,
                         int depth, uint32_t *out) {
  if (n == 0) return 0;
  const uint64_t R = hi - lo;
  if (R <= 2 * n || depth >= 24) return uniform_into(r, n, lo, hi, out);
  if (rng_next(r) & 1) {
    const uint64_t L = 2 * n + below(r, R - 2 * n);
    const uint64_t lo2 = lo + below(r, R - L + 1);
    return clustered_rec(r, n, lo2, lo2 + L, depth + 1, out);
  }
  const uint64_t c = lo + 1 + below(r, R - 1);
  const __uint128_t num = (__uint128_t)n * (c - lo);
  uint64_t nl = (uint64_t)(num / R);
  const uint64_t rem = (uint64_t)(num % R);
  if (below(r, R) < rem) nl++;
  if (nl > c - lo) nl = c - lo;
  if (n - nl > hi - c) nl = n - (hi - c);
  int rc = clustered_rec(r, nl, lo, c, depth + 1, out);
  if (rc) return rc;
  return clustered_rec(r, n - nl, c, hi, depth + 1, out + nl);
}

int wl_clustered(uint64_t n, uint64_t lo, uint64_t hi, uint64_t seed,
                 uint32_t *out) {
  rng_t r;
  rng_seed(&r, seed);
  if (hi > (1ull << 32) || lo > hi || n > hi - lo) return 1;
  return clustered_rec(&r, n, lo, hi, 0, out);
}

/* ---- many lists in parallel --------------------------------------------- */

typedef struct {
  int kind; /* 0 uniform, 1 clustered */
  uint64_t lo, hi, seed_base;
  const uint64_t *lens, *offs;
  uint32_t *out;
  uint64_t count;
  volatile uint64_t next; /* shared work counter */
  pthread_mutex_t mu;
  int rc;
} many_job;

static void *many_worker(void *arg) {
  many_job *j = (many_job *)arg;
  for (;;) {
    pthread_mutex_lock(&j->mu);
    uint64_t i = j->next++;
    pthread_mutex_unlock(&j->mu);
    if (i >= j->count) break;
    int rc = j->kind ? wl_clustered(j->lens[i], j->lo, j->hi, j->seed_base + i,
                                    j->out + j->offs[i])
                     : wl_uniform(j->lens[i], j->lo, j->hi, j->seed_base + i,
                                  j->out + j->offs[i]);
    if (rc) {
      pthread_mutex_lock(&j->mu);
      j->rc = rc;
      pthread_mutex_unlock(&j->mu);
    }
  }
  return NULL;
}

/* List i gets lens[i] values at out + offs[i], drawn with seed seed_base+i. */
int wl_many(int kind, uint64_t count, const uint64_t *lens,
            const uint64_t *offs, uint64_t lo, uint64_t hi, uint64_t seed_base,
            int nthreads, uint32_t *out) {
  many_job j;
  memset(&j, 0, sizeof j);
  j.kind = kind;
  j.lo = lo;
  j.hi = hi;
  j.seed_base = seed_base;
  j.lens = lens;
  j.offs = offs;
  j.out = out;
  j.count = count;
  pthread_mutex_init(&j.mu, NULL);
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  pthread_t th[256];
  for (int t = 0; t < nthreads; t++) pthread_create(&th[t], NULL, many_worker, &j);
  for (int t = 0; t < nthreads; t++) pthread_join(th[t], NULL);
  pthread_mutex_destroy(&j.mu);
  return j.rc;
}

/* ---- short list of a pair with a planted overlap ------------------------- *
 * k values drawn without replacement from f (nf sorted values), plus m-k
 * values of [0, U) that are not in f, sorted.  U <= 2^32. */
int wl_pair_short(const uint32_t *f, uint64_t nf, uint64_t m, uint64_t k,
                  uint64_t U, uint64_t seed, uint32_t *out) {
  rng_t r;
  rng_seed(&r, seed);
  if (k > m || k > nf || U > (1ull << 32) || m - k > U - nf) return 1;
  uint32_t *idx = (uint32_t *)malloc((k ? k : 1) * 4);
  if (!idx) return 2;
  int rc = uniform_into(&r, k, 0, nf, idx);
  if (rc) {
    free(idx);
    return rc;
  }
  uint64_t *bm = (uint64_t *)calloc((U + 63) / 64, 8);
  if (!bm) {
    free(idx);
    return 2;
  }
  for (uint64_t i = 0; i < nf; i++) bm[f[i] >> 6] |= 1ull << (f[i] & 63);
  for (uint64_t i = 0; i < k; i++) out[i] = f[idx[i]];
  free(idx);
  uint64_t have = k;
  while (have < m) {
    uint64_t v = below(&r, U);
    uint64_t bit = 1ull << (v & 63);
    if (!(bm[v >> 6] & bit)) {
      bm[v >> 6] |= bit;
      out[have++] = (uint32_t)v;
    }
  }
  free(bm);
  qsort(out, m, sizeof(uint32_t), cmp_u32);
  return 0;
}

/* ---- conjunctive queries ------------------------------------------------- *
 * nq queries.  Term count t (t = tmin + i) with probability weight[i] / sum;
 * terms drawn without replacement with probability proportional to the
 * length of their list (cum[] holds the running sum of lengths, cum[T-1] the
 * total).  terms[] receives the term ids, term_off[q] the start of query q
 * (nq+1 entries).  Capacity of terms[] must be nq * (tmin + nw - 1). */
int wl_queries(uint64_t nq, const uint64_t *cum, uint64_t T, uint32_t tmin,
               const uint32_t *weight, uint32_t nw, uint64_t seed,
               uint32_t *terms, uint64_t *term_off) {
  rng_t r;
  rng_seed(&r, seed);
  uint64_t wsum = 0;
  for (uint32_t i = 0; i < nw; i++) wsum += weight[i];
  if (wsum == 0 || T == 0) return 1;
  const uint64_t total = cum[T - 1];
  uint64_t pos = 0;
  for (uint64_t q = 0; q < nq; q++) {
    term_off[q] = pos;
    uint64_t u = below(&r, wsum), acc = 0;
    uint32_t cnt = tmin;
    for (uint32_t i = 0; i < nw; i++) {
      acc += weight[i];
      if (u < acc) {
        cnt = tmin + i;
        break;
      }
    }
    if (cnt > T) cnt = (uint32_t)T;
    for (uint32_t t = 0; t < cnt;) {
      uint64_t v = below(&r, total);
      uint64_t a = 0, b = T - 1; /* first i with cum[i] > v */
      while (a < b) {
        uint64_t mid = a + (b - a) / 2;
        if (cum[mid] > v) b = mid;
        else a = mid + 1;
      }
      int dup = 0;
      for (uint32_t s = 0; s < t; s++) dup |= (terms[pos + s] == (uint32_t)a);
      if (!dup) terms[pos + t++] = (uint32_t)a;
    }
    pos += cnt;
  }
  term_off[nq] = pos;
  return 0;
}
