/*
 * Seeded synthetic-genome generator.
 *
 * Stands in for the real datasets of the paper's Table 2, which are not
 * available: it produces ASCII {A,C,G,T} sequences from seeded Markov sources
 * with planted repeats, shaped like the workloads the compressor is measured
 * on.  It holds none of the compressor's arithmetic; both the CUDA path's
 * tests/benchmarks and the CPU oracle draw their inputs from here.
 *
 * Random numbers: xoshiro256** (Blackman & Vigna, 2018) seeded through
 * splitmix64 (Steele, Lea & Flood, 2014), both from their published
 * definitions.  Plain C99, no platform intrinsics: the same seed gives the
 * same bytes on x86-64 and aarch64 as long as libm's exp/log/cos agree (they
 * only shape the Markov tables, which are then rounded to 32-bit thresholds).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct { uint64_t s[4]; } rng_t;

static uint64_t sm64(uint64_t *x) {
  uint64_t z = (*x += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

static void rng_seed(rng_t *r, uint64_t seed) {
  uint64_t x = seed;
  for (int i = 0; i < 4; ++i) r->s[i] = sm64(&x);
}

static inline uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static uint64_t rng_next(rng_t *r) {
  uint64_t *s = r->s;
  uint64_t res = rotl(s[1] * 5, 7) * 9;
  uint64_t t = s[1] << 17;
  s[2] ^= s[0];
  s[3] ^= s[1];
  s[1] ^= s[2];
  s[0] ^= s[3];
  s[2] ^= t;
  s[3] = rotl(s[3], 45);
  return res;
}

/* uniform double in [0,1) with 53 random bits */
static double rng_u01(rng_t *r) { return (double)(rng_next(r) >> 11) * (1.0 / 9007199254740992.0); }

/* uniform integer in [0, n) (n > 0), by 128-bit-free rejection */
static uint64_t rng_below(rng_t *r, uint64_t n) {
  uint64_t lim = UINT64_MAX - (UINT64_MAX % n);
  uint64_t x;
  do { x = rng_next(r); } while (x >= lim);
  return x % n;
}

static double rng_normal(rng_t *r) {
  /* Box-Muller; u1 in (0,1] */
  double u1 = 1.0 - rng_u01(r), u2 = rng_u01(r);
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

static const char ACGT[4] = {'A', 'C', 'G', 'T'};

static int code_of(uint8_t c) {
  switch (c) {
    case 'A': return 0;
    case 'C': return 1;
    case 'G': return 2;
    case 'T': return 3;
  }
  return 0;
}

/*
 * Markov transition table of order `order`: probs[ctx*4 + b], ctx the base-4
 * value of the previous `order` bases (oldest most significant).
 *   p(b | ctx) ∝ pi_b * exp(z_scale * Z),  Z ~ N(0,1) per (ctx, b),
 *   pi = ((1-gc)/2, gc/2, gc/2, (1-gc)/2);
 * if the previous base is C, p(G | ctx) is divided by cpg_factor (>= 1).
 */
void synth_markov_table(double *probs, int order, double gc, double cpg_factor, double z_scale,
                        uint64_t seed) {
  rng_t r;
  rng_seed(&r, seed);
  uint64_t nctx = 1ULL << (2 * order);
  double pi[4] = {(1 - gc) / 2, gc / 2, gc / 2, (1 - gc) / 2};
  for (uint64_t c = 0; c < nctx; ++c) {
    double w[4], sum = 0;
    for (int b = 0; b < 4; ++b) {
      w[b] = pi[b] * exp(z_scale * rng_normal(&r));
      if (order > 0 && (c & 3) == 1 && b == 2) w[b] /= cpg_factor;
      sum += w[b];
    }
    for (int b = 0; b < 4; ++b) probs[c * 4 + b] = w[b] / sum;
  }
}

/* p'(b|ctx) ∝ p(b|ctx) * (1 + amount*u), u ~ U[-1,1] (robustness workloads) */
void synth_perturb_table(double *probs, int order, double amount, uint64_t seed) {
  rng_t r;
  rng_seed(&r, seed);
  uint64_t nctx = 1ULL << (2 * order);
  for (uint64_t c = 0; c < nctx; ++c) {
    double sum = 0;
    for (int b = 0; b < 4; ++b) {
      probs[c * 4 + b] *= 1.0 + amount * (2.0 * rng_u01(&r) - 1.0);
      sum += probs[c * 4 + b];
    }
    for (int b = 0; b < 4; ++b) probs[c * 4 + b] /= sum;
  }
}

/* Sample n bases from a Markov table; the first `order` bases come from the stationary-free
 * uniform start (context 0 = "AA..A" is used until `order` bases exist). */
int synth_markov_sample(uint8_t *out, uint64_t n, int order, const double *probs, uint64_t seed) {
  rng_t r;
  rng_seed(&r, seed);
  uint64_t nctx = 1ULL << (2 * order);
  uint32_t *thr = (uint32_t *)malloc(sizeof(uint32_t) * nctx * 3);
  if (!thr) return -1;
  for (uint64_t c = 0; c < nctx; ++c) {
    double acc = 0;
    for (int b = 0; b < 3; ++b) {
      acc += probs[c * 4 + b];
      double t = acc * 4294967296.0;
      thr[c * 3 + b] = t >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)t;
    }
  }
  uint64_t mask = nctx - 1, ctx = 0;
  for (uint64_t i = 0; i < n; ++i) {
    uint32_t u = (uint32_t)(rng_next(&r) >> 32);
    const uint32_t *t = thr + ctx * 3;
    int b = u < t[0] ? 0 : (u < t[1] ? 1 : (u < t[2] ? 2 : 3));
    out[i] = (uint8_t)ACGT[b];
    ctx = order > 0 ? ((ctx << 2) | (uint64_t)b) & mask : 0;
  }
  free(thr);
  return 0;
}

static uint8_t mutate(rng_t *r, uint8_t c) {
  int b = code_of(c);
  int d = (b + 1 + (int)rng_below(r, 3)) & 3; /* uniformly one of the other three */
  return (uint8_t)ACGT[d];
}

/* Plant `count` copies of randomly chosen earlier segments of length `len` at random
 * positions (overwriting), each base of a copy replaced with probability mu. */
void synth_plant_repeats(uint8_t *buf, uint64_t n, int count, uint64_t len, double mu, uint64_t seed) {
  if (n < 2 * len + 1) return;
  rng_t r;
  rng_seed(&r, seed);
  for (int c = 0; c < count; ++c) {
    uint64_t src = rng_below(&r, n - len);
    uint64_t dst = rng_below(&r, n - len);
    for (uint64_t i = 0; i < len; ++i) {
      uint8_t b = buf[src + i];
      if (rng_u01(&r) < mu) b = mutate(&r, b);
      buf[dst + i] = b;
    }
  }
}

/* Interspersed repeat families (Alu-like): n_fam random consensus sequences of length
 * fam_len; mutated copies (rate mu) are written at random positions until `coverage`
 * of the bases are covered. */
int synth_plant_families(uint8_t *buf, uint64_t n, int n_fam, uint64_t fam_len, double coverage,
                         double mu, uint64_t seed, uint64_t place_seed) {
  if (n < fam_len + 1 || n_fam <= 0) return 0;
  rng_t r;
  rng_seed(&r, seed);
  uint8_t *cons = (uint8_t *)malloc((size_t)(n_fam * fam_len));
  if (!cons) return -1;
  for (uint64_t i = 0; i < (uint64_t)n_fam * fam_len; ++i) cons[i] = (uint8_t)ACGT[rng_below(&r, 4)];
  /* the copies' places and mutations: the same stream, or (place_seed != seed) their own, so that
   * another genome of the same "species" shares the family consensus sequences */
  if (place_seed != seed) rng_seed(&r, place_seed);
  uint64_t target = (uint64_t)(coverage * (double)n), done = 0;
  while (done < target) {
    const uint8_t *f = cons + rng_below(&r, (uint64_t)n_fam) * fam_len;
    uint64_t dst = rng_below(&r, n - fam_len);
    for (uint64_t i = 0; i < fam_len; ++i) {
      uint8_t b = f[i];
      if (rng_u01(&r) < mu) b = mutate(&r, b);
      buf[dst + i] = b;
    }
    done += fam_len;
  }
  free(cons);
  return 0;
}

/* Tandem repeats: a random unit of period in [pmin, pmax] repeated for a geometric run
 * length with mean `mean_run` bases, at random positions until `coverage` is covered. */
void synth_plant_tandem(uint8_t *buf, uint64_t n, double coverage, int pmin, int pmax, double mean_run,
                        uint64_t seed) {
  rng_t r;
  rng_seed(&r, seed);
  uint64_t target = (uint64_t)(coverage * (double)n), done = 0;
  uint8_t unit[64];
  if (pmax > 64) pmax = 64;
  while (done < target) {
    int p = pmin + (int)rng_below(&r, (uint64_t)(pmax - pmin + 1));
    for (int i = 0; i < p; ++i) unit[i] = (uint8_t)ACGT[rng_below(&r, 4)];
    /* geometric length with mean mean_run, at least one period */
    double u = 1.0 - rng_u01(&r);
    uint64_t run = (uint64_t)(-mean_run * log(u));
    if (run < (uint64_t)p) run = (uint64_t)p;
    if (run >= n) run = n - 1;
    uint64_t dst = rng_below(&r, n - run);
    for (uint64_t i = 0; i < run; ++i) buf[dst + i] = unit[i % (uint64_t)p];
    done += run;
  }
}

/* log-normal sequence lengths: ln L ~ N(mu, sigma), clipped to [lo, hi], then scaled so the
 * lengths sum exactly to `total` (the rounding remainder goes to the longest sequences).  When that
 * scaling takes a length above hi (the full-size batching workload: the 8 MB cap), the scale is
 * solved again with the clip inside it, L_i = clip(c x_i, lo, hi) with c such that the lengths sum
 * to `total` (bisection), and the rounding remainder goes one base at a time to the longest
 * sequences still below hi (or is taken from the longest above lo), so every length lies in
 * [lo, hi].  Draws whose single scaling stays at or below hi keep it unchanged. */
int synth_lognormal_lengths(uint64_t *lens, int count, double mu, double sigma, uint64_t lo, uint64_t hi,
                            uint64_t total, uint64_t seed) {
  rng_t r;
  rng_seed(&r, seed);
  double *x = (double *)malloc(sizeof(double) * (size_t)count);
  if (!x) return -1;
  double sum = 0;
  for (int i = 0; i < count; ++i) {
    double v = exp(mu + sigma * rng_normal(&r));
    if (v < (double)lo) v = (double)lo;
    if (v > (double)hi) v = (double)hi;
    x[i] = v;
    sum += v;
  }
  uint64_t acc = 0;
  for (int i = 0; i < count; ++i) {
    uint64_t v = (uint64_t)floor(x[i] * (double)total / sum);
    if (v < 1) v = 1;
    lens[i] = v;
    acc += v;
  }
  /* hand the remainder (or take the excess) one base at a time, longest first */
  while (acc != total) {
    int best = 0;
    for (int i = 1; i < count; ++i)
      if (lens[i] > lens[best]) best = i;
    if (acc < total) {
      uint64_t add = total - acc;
      lens[best] += add;
      acc += add;
    } else {
      uint64_t take = acc - total;
      if (take > lens[best] - 1) take = lens[best] - 1;
      lens[best] -= take;
      acc -= take;
    }
  }
  int over = 0;
  for (int i = 0; i < count; ++i) over |= lens[i] > hi;
  if (over && (double)count * (double)lo <= (double)total && (double)total <= (double)count * (double)hi) {
    double xmin = x[0];
    for (int i = 1; i < count; ++i)
      if (x[i] < xmin) xmin = x[i];
    double c_lo = 0.0, c_hi = (double)hi / xmin;  /* f(c_hi) = count * hi >= total */
    for (int it = 0; it < 200; ++it) {
      double c = 0.5 * (c_lo + c_hi), f = 0;
      for (int i = 0; i < count; ++i) {
        double v = c * x[i];
        f += v < (double)lo ? (double)lo : (v > (double)hi ? (double)hi : v);
      }
      if (f < (double)total)
        c_lo = c;
      else
        c_hi = c;
    }
    acc = 0;
    for (int i = 0; i < count; ++i) {
      double v = c_lo * x[i];
      v = v < (double)lo ? (double)lo : (v > (double)hi ? (double)hi : v);
      lens[i] = (uint64_t)floor(v);
      if (lens[i] < lo) lens[i] = lo;
      acc += lens[i];
    }
    while (acc != total) {
      int best = -1;
      for (int i = 0; i < count; ++i) {
        const int ok = acc < total ? lens[i] < hi : lens[i] > lo;
        if (ok && (best < 0 || lens[i] > lens[best])) best = i;
      }
      if (best < 0) break; /* cannot happen: count lo <= total <= count hi */
      if (acc < total) {
        lens[best] += 1;
        acc += 1;
      } else {
        lens[best] -= 1;
        acc -= 1;
      }
    }
  }
  free(x);
  return 0;
}
