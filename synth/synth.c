/*
 * Seeded synthetic hypergraph generators.
 *
 * This file holds input generation only: random net sizes, random pin
 * choices and random weights.  It contains none of the partitioner's
 * arithmetic and is shared, as input, by the CPU oracle and by the CUDA
 * library.  Everything is a pure function of the 64-bit stream seed passed
 * in, so both sides see identical hypergraphs.
 *
 * Random source: xoshiro256** (Blackman and Vigna, "Scrambled linear
 * pseudorandom number generators", 2018), its 256-bit state filled from the
 * seed with SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
 * number generators", OOPSLA 2014), as the xoshiro authors recommend.
 *
 * Portable C99 plus unsigned __int128 (gcc on x86_64 and aarch64).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  uint64_t s[4];
} rng_t;

static uint64_t splitmix_next(uint64_t* x) {
  uint64_t z = (*x += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

static inline uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static void rng_seed(rng_t* r, uint64_t seed) {
  uint64_t x = seed;
  for (int i = 0; i < 4; ++i) r->s[i] = splitmix_next(&x);
}

static uint64_t rng_next(rng_t* r) {
  uint64_t* s = r->s;
  const uint64_t result = rotl(s[1] * 5, 7) * 9;
  const uint64_t t = s[1] << 17;
  s[2] ^= s[0];
  s[3] ^= s[1];
  s[1] ^= s[2];
  s[0] ^= s[3];
  s[2] ^= t;
  s[3] = rotl(s[3], 45);
  return result;
}

/* uniform double in [0, 1) with 53 random bits */
static double rng_unif(rng_t* r) { return (double)(rng_next(r) >> 11) * 0x1.0p-53; }

/* uniform integer in [0, bound) by the multiply-high map (bound >= 1) */
static uint64_t rng_below(rng_t* r, uint64_t bound) {
  return (uint64_t)(((unsigned __int128)rng_next(r) * bound) >> 64);
}

/* ---- exported: the raw streams, so tests can pin the generator itself ---- */

uint64_t syn_splitmix64_first(uint64_t seed) {
  uint64_t x = seed;
  return splitmix_next(&x);
}

void syn_xoshiro_stream(uint64_t seed, int64_t count, uint64_t* out) {
  rng_t r;
  rng_seed(&r, seed);
  for (int64_t i = 0; i < count; ++i) out[i] = rng_next(&r);
}

/* ---- net sizes ---- */

/* size = base + G, G = number of failures before the first success of a
 * Bernoulli(prob) sequence, the whole size capped at cap. */
void syn_sizes_geometric(uint64_t seed, int64_t m, double prob, int32_t base, int32_t cap,
                         int32_t* out) {
  rng_t r;
  rng_seed(&r, seed);
  const double lq = log1p(-prob);
  for (int64_t i = 0; i < m; ++i) {
    double u = 1.0 - rng_unif(&r); /* (0, 1] */
    double g = floor(log(u) / lq);
    int64_t s = (int64_t)base + (int64_t)g;
    if (s > cap) s = cap;
    out[i] = (int32_t)s;
  }
}

/* discrete Zipf: P(size = x) proportional to x^-s on the integers [lo, hi],
 * drawn by inverse transform over the tabulated CDF */
void syn_sizes_zipf(uint64_t seed, int64_t m, double s, int32_t lo, int32_t hi, int32_t* out) {
  rng_t r;
  rng_seed(&r, seed);
  const int32_t span = hi - lo + 1;
  double* cdf = (double*)malloc(sizeof(double) * (size_t)span);
  double acc = 0.0;
  for (int32_t i = 0; i < span; ++i) {
    acc += pow((double)(lo + i), -s);
    cdf[i] = acc;
  }
  for (int64_t i = 0; i < m; ++i) {
    double u = rng_unif(&r) * acc;
    int32_t a = 0, b = span - 1; /* first index with cdf > u */
    while (a < b) {
      int32_t mid = a + (b - a) / 2;
      if (cdf[mid] > u) b = mid; else a = mid + 1;
    }
    out[i] = lo + a;
  }
  free(cdf);
}

/* continuous power law, density proportional to x^-alpha on [lo, hi],
 * by inverse transform, rounded down to an integer */
void syn_sizes_powerlaw(uint64_t seed, int64_t m, double alpha, double lo, double hi,
                        int32_t* out) {
  rng_t r;
  rng_seed(&r, seed);
  const double a1 = 1.0 - alpha;
  const double l = pow(lo, a1), h = pow(hi, a1);
  for (int64_t i = 0; i < m; ++i) {
    double u = rng_unif(&r);
    double x = pow(l + u * (h - l), 1.0 / a1);
    int64_t v = (int64_t)floor(x);
    if (v < (int64_t)lo) v = (int64_t)lo;
    if (v > (int64_t)hi) v = (int64_t)hi;
    out[i] = (int32_t)v;
  }
}

/* ---- pins ---- */

/* Pins of every net drawn uniformly from [0, n) without repeats inside a net.
 * offsets has m+1 entries; every net size must be <= n. */
int syn_pins_uniform(uint64_t seed, int32_t n, int64_t m, const int64_t* offsets,
                     int32_t* pins) {
  rng_t r;
  rng_seed(&r, seed);
  int64_t* stamp = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  if (!stamp) return -1;
  for (int32_t v = 0; v < n; ++v) stamp[v] = -1;
  for (int64_t e = 0; e < m; ++e) {
    const int64_t b = offsets[e], en = offsets[e + 1];
    if (en - b > n) { free(stamp); return -2; }
    for (int64_t q = b; q < en; ++q) {
      int32_t v;
      do { v = (int32_t)rng_below(&r, (uint64_t)n); } while (stamp[v] == e);
      stamp[v] = e;
      pins[q] = v;
    }
  }
  free(stamp);
  return 0;
}

/* Preferential pin choice: every new pin is, with probability n/(n + P) where
 * P counts the pins of all earlier nets, a "fresh" node (the next node of a
 * seeded random permutation that has not been used yet; once all nodes have
 * been used, a uniform node); otherwise it copies a uniformly chosen pin of
 * an earlier net.  A node already in the current net is redrawn.  Copying
 * gives a heavy-tailed node-degree distribution; drawing fresh nodes first
 * leaves (with high probability) no node of degree zero. */
int syn_pins_preferential(uint64_t seed, int32_t n, int64_t m, const int64_t* offsets,
                          int32_t* pins) {
  rng_t r;
  rng_seed(&r, seed);
  int64_t* stamp = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  int32_t* perm = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  if (!stamp || !perm) { free(stamp); free(perm); return -1; }
  for (int32_t v = 0; v < n; ++v) { stamp[v] = -1; perm[v] = v; }
  for (int32_t v = n - 1; v > 0; --v) { /* Fisher-Yates */
    int32_t j = (int32_t)rng_below(&r, (uint64_t)v + 1);
    int32_t t = perm[v]; perm[v] = perm[j]; perm[j] = t;
  }
  int32_t next_fresh = 0;
  for (int64_t e = 0; e < m; ++e) {
    const int64_t b = offsets[e], en = offsets[e + 1];
    if (en - b > n) { free(stamp); free(perm); return -2; }
    for (int64_t q = b; q < en; ++q) {
      int32_t v;
      int tries = 0;
      do {
        /* fall back to uniform after many collisions so the loop always ends */
        const int fresh = b == 0 || rng_below(&r, (uint64_t)n + (uint64_t)b) < (uint64_t)n;
        if (tries > 64) v = (int32_t)rng_below(&r, (uint64_t)n);
        else if (fresh && next_fresh < n && stamp[perm[next_fresh]] != e) v = perm[next_fresh++];
        else if (fresh || b == 0) v = (int32_t)rng_below(&r, (uint64_t)n);
        else v = pins[rng_below(&r, (uint64_t)b)];
        ++tries;
      } while (stamp[v] == e);
      stamp[v] = e;
      pins[q] = v;
    }
  }
  free(stamp);
  free(perm);
  return 0;
}

/* ---- scalars ---- */

void syn_uniform_ints(uint64_t seed, int64_t count, int32_t lo, int32_t hi, int32_t* out) {
  rng_t r;
  rng_seed(&r, seed);
  const uint64_t span = (uint64_t)((int64_t)hi - (int64_t)lo + 1);
  for (int64_t i = 0; i < count; ++i) out[i] = lo + (int32_t)rng_below(&r, span);
}

void syn_uniform_doubles(uint64_t seed, int64_t count, double* out) {
  rng_t r;
  rng_seed(&r, seed);
  for (int64_t i = 0; i < count; ++i) out[i] = rng_unif(&r);
}
