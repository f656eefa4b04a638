/*
 * Seeded synthetic column generator for the delta-to-main merge.
 *
 * This file produces INPUTS only: sorted main dictionaries, main code
 * vectors (uniform or Zipf over dictionary ranks), the LSB-first bit
 * packing of those codes, and delta partitions stored as an
 * insertion-order dictionary plus uint32 row codes.  It holds none of the
 * merge arithmetic (no dictionary merge, no translation table, no
 * re-encode); both the CUDA path and the CPU oracle consume what it writes.
 *
 * Randomness is counter based: element i of a stream with seed s is
 * splitmix64's output function applied to s + (i+1)*0x9E3779B97F4A7C15
 * (Steele, Lea, Flood, "Fast splittable pseudorandom number generators",
 * OOPSLA 2014), so every element is a pure function of (seed, i) and the
 * bulk loops split over threads without changing the result.
 *
 * The paper's experiments draw values uniformly at random (Section 7);
 * dictionaries here are stratified-uniform: key i is uniform inside the
 * i-th of m equal slices of the value range, which makes the dictionary
 * sorted and duplicate free by construction.  Zipf ranks are drawn by
 * inversion of the exact discrete CDF with a guide table (Chen and Asau,
 * 1974) and mapped to codes through a seeded Fisher-Yates permutation, so
 * hot codes are scattered over the dictionary.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GOLDEN 0x9E3779B97F4A7C15ULL

static inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* i-th output of the stream with the given seed */
static inline uint64_t rnd(uint64_t seed, uint64_t i) { return mix64(seed + (i + 1) * GOLDEN); }

/* derived stream seed: independent streams for different purposes */
uint64_t synth_subseed(uint64_t seed, uint64_t tag) { return mix64(seed ^ mix64(tag + 0x5851F42D4C957F2DULL)); }

/* uniform integer in [0, n) (multiply-high; bias below 2^-64 * n) */
static inline uint64_t below(uint64_t r, uint64_t n) {
  return (uint64_t)(((unsigned __int128)r * (unsigned __int128)n) >> 64);
}

/* uniform double in [0, 1) with 53 random bits */
static inline double unit(uint64_t r) { return (double)(r >> 11) * (1.0 / 9007199254740992.0); }

/* ------------------------------------------------------------------ */
/* keys: w = 4 (uint32), 8 (uint64), 16 ({uint64 hi, uint64 lo})       */
/* ------------------------------------------------------------------ */

typedef struct { uint64_t hi, lo; } k128;

static inline int key_cmp(uint32_t w, const void* a, const void* b) {
  if (w == 4) {
    uint32_t x = *(const uint32_t*)a, y = *(const uint32_t*)b;
    return (x > y) - (x < y);
  }
  if (w == 8) {
    uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
    return (x > y) - (x < y);
  }
  const k128* x = (const k128*)a;
  const k128* y = (const k128*)b;
  if (x->hi != y->hi) return x->hi > y->hi ? 1 : -1;
  return (x->lo > y->lo) - (x->lo < y->lo);
}

/* true if key is present in the sorted array arr[0..n) */
static int sorted_contains(uint32_t w, const void* arr, uint64_t n, const void* key) {
  uint64_t lo = 0, hi = n;
  const char* base = (const char*)arr;
  while (lo < hi) {
    uint64_t mid = lo + (hi - lo) / 2;
    int c = key_cmp(w, base + mid * w, key);
    if (c == 0) return 1;
    if (c < 0) lo = mid + 1; else hi = mid;
  }
  return 0;
}

/*
 * m sorted, distinct keys of width w.  Slice width = floor(range / m);
 * key i = i * slice + uniform(slice).  For w = 16 the slices stratify the
 * hi word and lo is uniform.  Returns -1 when m exceeds the key space.
 */
int synth_dict(uint64_t seed, uint32_t w, uint64_t m, void* out) {
  if (m == 0) return 0;
  if (w == 4) {
    if (m > (1ULL << 32)) return -1;
    uint64_t slice = (1ULL << 32) / m;
    uint32_t* o = (uint32_t*)out;
    for (uint64_t i = 0; i < m; ++i) o[i] = (uint32_t)(i * slice + below(rnd(seed, i), slice));
    return 0;
  }
  uint64_t slice = (m == 1) ? UINT64_MAX : (UINT64_MAX / m);
  if (w == 8) {
    uint64_t* o = (uint64_t*)out;
    for (uint64_t i = 0; i < m; ++i) o[i] = i * slice + below(rnd(seed, i), slice);
    return 0;
  }
  if (w == 16) {
    k128* o = (k128*)out;
    uint64_t s2 = synth_subseed(seed, 16);
    for (uint64_t i = 0; i < m; ++i) {
      o[i].hi = i * slice + below(rnd(seed, i), slice);
      o[i].lo = rnd(s2, i);
    }
    return 0;
  }
  return -1;
}

/* ------------------------------------------------------------------ */
/* code distributions                                                  */
/* ------------------------------------------------------------------ */

typedef struct {
  uint64_t m;
  int zipf;
  double* cdf;      /* cdf[r] = P(rank <= r), ranks 0..m-1 (rank 0 is the most frequent) */
  uint64_t* guide;  /* guide[g] = first rank r with cdf[r] > g / m */
  uint32_t* perm;   /* rank -> code */
} sampler;

/* Zipf(s) over m ranks: P(rank r) proportional to (r+1)^-s. */
static int sampler_init(sampler* S, uint64_t seed, uint64_t m, int zipf, double s) {
  memset(S, 0, sizeof(*S));
  S->m = m;
  S->zipf = zipf;
  if (!zipf || m == 0) return 0;
  S->cdf = (double*)malloc(sizeof(double) * m);
  S->guide = (uint64_t*)malloc(sizeof(uint64_t) * (m + 1));
  S->perm = (uint32_t*)malloc(sizeof(uint32_t) * m);
  if (!S->cdf || !S->guide || !S->perm) return -1;
  double acc = 0.0;
  for (uint64_t r = 0; r < m; ++r) {
    acc += pow((double)(r + 1), -s);
    S->cdf[r] = acc;
  }
  for (uint64_t r = 0; r < m; ++r) S->cdf[r] /= acc;
  S->cdf[m - 1] = 1.0;
  uint64_t r = 0;
  for (uint64_t g = 0; g <= m; ++g) {
    double t = (double)g / (double)m;
    while (r < m - 1 && S->cdf[r] <= t) ++r;
    S->guide[g] = r;
  }
  /* Fisher-Yates: rank -> code permutation */
  uint64_t ps = synth_subseed(seed, 0x7065726DULL);
  for (uint64_t i = 0; i < m; ++i) S->perm[i] = (uint32_t)i;
  for (uint64_t i = m - 1; i > 0; --i) {
    uint64_t j = below(rnd(ps, i), i + 1);
    uint32_t t = S->perm[i];
    S->perm[i] = S->perm[j];
    S->perm[j] = t;
  }
  return 0;
}

static void sampler_free(sampler* S) {
  free(S->cdf);
  free(S->guide);
  free(S->perm);
  memset(S, 0, sizeof(*S));
}

static inline uint32_t sampler_draw(const sampler* S, uint64_t r) {
  if (!S->zipf) return (uint32_t)below(r, S->m);
  double u = unit(r);
  uint64_t g = (uint64_t)(u * (double)S->m);
  if (g > S->m) g = S->m;
  uint64_t k = S->guide[g];
  while (k < S->m - 1 && S->cdf[k] <= u) ++k;
  return S->perm[k];
}

typedef struct {
  const sampler* S;
  uint64_t seed, begin, end;
  uint32_t* out;
} codes_job;

static void* codes_worker(void* p) {
  codes_job* J = (codes_job*)p;
  for (uint64_t i = J->begin; i < J->end; ++i) J->out[i] = sampler_draw(J->S, rnd(J->seed, i));
  return NULL;
}

/*
 * n codes in [0, m): dist 0 = uniform, dist 1 = Zipf(s) over ranks mapped
 * through a seeded permutation.  nthreads splits the index range; the
 * output does not depend on it.
 */
int synth_codes(uint64_t seed, uint64_t m, uint64_t n, int dist, double s, uint32_t* out, int nthreads) {
  if (n == 0) return 0;
  if (m == 0) return -1;
  sampler S;
  if (sampler_init(&S, seed, m, dist == 1, s) != 0) { sampler_free(&S); return -2; }
  uint64_t cs = synth_subseed(seed, 0x636F6465ULL);
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 64) nthreads = 64;
  pthread_t th[64];
  codes_job jobs[64];
  uint64_t chunk = (n + nthreads - 1) / nthreads;
  int started = 0;
  for (int t = 0; t < nthreads; ++t) {
    uint64_t b = (uint64_t)t * chunk, e = b + chunk;
    if (b >= n) break;
    if (e > n) e = n;
    jobs[t] = (codes_job){&S, cs, b, e, out};
    if (nthreads == 1) { codes_worker(&jobs[t]); continue; }
    pthread_create(&th[t], NULL, codes_worker, &jobs[t]);
    ++started;
  }
  for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
  sampler_free(&S);
  return 0;
}

/* ------------------------------------------------------------------ */
/* packing: code i occupies stream bits [i*b, (i+1)*b), LSB first;     */
/* stream bit k is bit (k mod 32) of 32-bit word k/32 (little endian); */
/* the buffer is a whole number of 16-byte units, zero padded.         */
/* ------------------------------------------------------------------ */

uint64_t synth_packed_words(uint64_t n, uint32_t b) {
  uint64_t bits = n * (uint64_t)b;
  return ((bits + 127) / 128) * 4;
}

typedef struct {
  const uint32_t* codes;
  uint64_t n, g0, g1;
  uint32_t b;
  uint32_t* words;
  uint64_t nwords;
} pack_job;

/* groups of 32 codes own exactly b words, so groups pack independently */
static void* pack_worker(void* p) {
  pack_job* J = (pack_job*)p;
  uint32_t b = J->b;
  for (uint64_t g = J->g0; g < J->g1; ++g) {
    uint64_t bit = 0;
    uint64_t wbase = g * b;
    for (uint32_t k = 0; k < b && wbase + k < J->nwords; ++k) J->words[wbase + k] = 0;
    for (uint32_t j = 0; j < 32; ++j, bit += b) {
      uint64_t i = g * 32 + j;
      if (i >= J->n) break;
      uint64_t c = J->codes[i];
      if (b < 32) c &= ((1ULL << b) - 1);
      uint64_t wi = wbase + (bit >> 5);
      uint32_t sh = (uint32_t)(bit & 31);
      uint64_t v = c << sh;
      J->words[wi] |= (uint32_t)v;
      if (sh + b > 32) J->words[wi + 1] |= (uint32_t)(v >> 32);
    }
  }
  return NULL;
}

int synth_pack(const uint32_t* codes, uint64_t n, uint32_t b, uint32_t* words, int nthreads) {
  uint64_t nwords = synth_packed_words(n, b);
  memset(words, 0, nwords * 4);
  if (b == 0 || n == 0) return 0;
  if (b > 32) return -1;
  uint64_t ng = (n + 31) / 32;
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 64) nthreads = 64;
  pthread_t th[64];
  pack_job jobs[64];
  uint64_t chunk = (ng + nthreads - 1) / nthreads;
  int started = 0;
  for (int t = 0; t < nthreads; ++t) {
    uint64_t b0 = (uint64_t)t * chunk, e = b0 + chunk;
    if (b0 >= ng) break;
    if (e > ng) e = ng;
    jobs[t] = (pack_job){codes, n, b0, e, b, words, nwords};
    if (nthreads == 1) { pack_worker(&jobs[t]); continue; }
    pthread_create(&th[t], NULL, pack_worker, &jobs[t]);
    ++started;
  }
  for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
  return 0;
}

/* ------------------------------------------------------------------ */
/* delta partition                                                     */
/* ------------------------------------------------------------------ */

/* open-addressing map from a w-byte key to its insertion index */
typedef struct {
  uint32_t w;
  uint64_t cap;     /* power of two */
  uint64_t* slot;   /* index + 1, 0 = empty */
  const char* keys; /* key storage indexed by insertion index */
} keymap;

static inline uint64_t key_hash(uint32_t w, const void* k) {
  if (w == 4) return mix64(*(const uint32_t*)k);
  if (w == 8) return mix64(*(const uint64_t*)k);
  const k128* x = (const k128*)k;
  return mix64(x->hi ^ mix64(x->lo));
}

static int keymap_init(keymap* M, uint32_t w, uint64_t expected, const char* keys) {
  M->w = w;
  M->cap = 16;
  while (M->cap < expected * 2 + 16) M->cap <<= 1;
  M->slot = (uint64_t*)calloc(M->cap, sizeof(uint64_t));
  M->keys = keys;
  return M->slot ? 0 : -1;
}

/* returns the slot holding key (existing) or the empty slot to use */
static uint64_t* keymap_find(keymap* M, const void* key) {
  uint64_t mask = M->cap - 1;
  uint64_t h = key_hash(M->w, key) & mask;
  for (;;) {
    uint64_t* s = &M->slot[h];
    if (*s == 0) return s;
    if (memcmp(M->keys + (*s - 1) * M->w, key, M->w) == 0) return s;
    h = (h + 1) & mask;
  }
}

static void random_key(uint32_t w, uint64_t seed, uint64_t i, void* out) {
  if (w == 4) *(uint32_t*)out = (uint32_t)rnd(seed, i);
  else if (w == 8) *(uint64_t*)out = rnd(seed, i);
  else {
    k128* k = (k128*)out;
    k->hi = rnd(seed, 2 * i);
    k->lo = rnd(seed, 2 * i + 1);
  }
}

/*
 * Delta partition of nd rows against the sorted main dictionary um[0..m).
 *
 * Each row is "fresh" with probability f_new, else it resamples a main
 * value U_M[c] with c drawn from the code distribution (dist, s); passing
 * the seed the main codes were drawn with (code_seed) reuses their
 * rank -> code permutation, so values hot in the main are hot here too.
 *   pool == 0 : every fresh row carries its own new value;
 *   pool  > 0 : fresh rows draw uniformly from `pool` new values.
 * New values are uniform keys absent from U_M and from each other.
 * The delta dictionary lists distinct values in first-occurrence order
 * and dcodes[r] is the row's index in it.  ddict must hold nd keys;
 * *d_out receives the dictionary length.
 */
int synth_delta(uint64_t seed, uint64_t code_seed, uint32_t w, const void* um, uint64_t m, uint64_t nd,
                double f_new, uint64_t pool, int dist, double s, void* ddict, uint64_t* d_out,
                uint32_t* dcodes) {
  *d_out = 0;
  if (nd == 0) return 0;
  if (w != 4 && w != 8 && w != 16) return -1;
  uint64_t rs = synth_subseed(seed, 0x726F7773ULL);   /* row kind */
  uint64_t ns = synth_subseed(seed, 0x6E657776ULL);   /* new-value keys */
  uint64_t ps = synth_subseed(seed, 0x706F6F6CULL);   /* pool picks */
  uint64_t n_fresh = 0;
  for (uint64_t r = 0; r < nd; ++r) n_fresh += (m == 0) || (unit(rnd(rs, r)) < f_new);
  uint64_t n_new = pool ? pool : n_fresh;
  if (n_fresh == 0) n_new = 0;

  /* new values: uniform, rejected when in U_M or already drawn */
  char* newv = (char*)malloc((n_new ? n_new : 1) * w);
  keymap NM;
  if (!newv || keymap_init(&NM, w, n_new, newv) != 0) { free(newv); return -2; }
  uint64_t drawn = 0;
  for (uint64_t t = 0; drawn < n_new; ++t) {
    char* k = newv + drawn * w;
    random_key(w, ns, t, k);
    if (sorted_contains(w, um, m, k)) continue;
    uint64_t* sl = keymap_find(&NM, k);
    if (*sl) continue;
    *sl = drawn + 1;
    ++drawn;
  }
  free(NM.slot);

  sampler S;
  if (m > 0 && sampler_init(&S, code_seed, m, dist == 1, s) != 0) {
    sampler_free(&S);
    free(newv);
    return -3;
  }
  uint64_t cs = synth_subseed(seed, 0x72657361ULL);
  keymap DM;
  if (keymap_init(&DM, w, nd < (1u << 24) ? nd : (1u << 24), (const char*)ddict) != 0) {
    if (m > 0) sampler_free(&S);
    free(newv);
    return -2;
  }
  uint64_t d = 0, next_new = 0;
  char kbuf[16];
  for (uint64_t r = 0; r < nd; ++r) {
    int fresh = (m == 0) || (unit(rnd(rs, r)) < f_new);
    if (fresh) {
      uint64_t idx = pool ? below(rnd(ps, r), pool) : next_new++;
      memcpy(kbuf, newv + idx * w, w);
    } else {
      uint32_t c = sampler_draw(&S, rnd(cs, r));
      memcpy(kbuf, (const char*)um + (uint64_t)c * w, w);
    }
    uint64_t* sl = keymap_find(&DM, kbuf);
    if (*sl == 0) {
      if (d * 2 + 16 > DM.cap) {
        /* grow: rehash existing entries */
        uint64_t oc = DM.cap;
        uint64_t* os = DM.slot;
        DM.cap <<= 1;
        DM.slot = (uint64_t*)calloc(DM.cap, sizeof(uint64_t));
        if (!DM.slot) { free(os); if (m > 0) sampler_free(&S); free(newv); return -2; }
        for (uint64_t q = 0; q < oc; ++q)
          if (os[q]) *keymap_find(&DM, (const char*)ddict + (os[q] - 1) * w) = os[q];
        free(os);
        sl = keymap_find(&DM, kbuf);
      }
      memcpy((char*)ddict + d * w, kbuf, w);
      *sl = d + 1;
      dcodes[r] = (uint32_t)d;
      ++d;
    } else {
      dcodes[r] = (uint32_t)(*sl - 1);
    }
  }
  free(DM.slot);
  if (m > 0) sampler_free(&S);
  free(newv);
  *d_out = d;
  return 0;
}
