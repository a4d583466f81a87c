/*
 * Seeded synthetic ballot generators.
 *
 * This file draws preference profiles and nothing else: it holds none of the
 * Schulze arithmetic (no tally, no widths, no winners). Both the CUDA path and
 * the CPU oracle are fed the buffers it writes.
 *
 * Ballot form: an [n, k] int32 row-major array; row v lists candidate ids
 * best first, all distinct, 0 <= id < m. k == m is a full ranking; with k < m
 * the absent candidates are tied below every listed one.
 *
 * Every voter draws from its own counter-based stream (splitmix64 seeded by
 * (seed, voter)), so the output does not depend on the thread count.
 * Floating point is restricted to +, *, / and comparisons of doubles, except
 * for the Zipf weights (pow), and the file is compiled with contraction off.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ RNG */

static inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

typedef struct {
  uint64_t s;
} rng_t;

static inline rng_t rng_for(uint64_t seed, uint64_t stream) {
  rng_t r;
  r.s = mix64(mix64(seed + 0x9E3779B97F4A7C15ULL) ^ (stream * 0xD1B54A32D192ED03ULL + 1));
  return r;
}

static inline uint64_t rng_next(rng_t* r) {
  r->s += 0x9E3779B97F4A7C15ULL;
  return mix64(r->s);
}

/* uniform double in [0, 1) with 53 random bits */
static inline double rng_u01(rng_t* r) { return (double)(rng_next(r) >> 11) * (1.0 / 9007199254740992.0); }

/* uniform integer in [0, bound), bound >= 1, by rejection (no modulo bias) */
static inline uint64_t rng_below(rng_t* r, uint64_t bound) {
  uint64_t lim = UINT64_MAX - (UINT64_MAX % bound);
  uint64_t x;
  do {
    x = rng_next(r);
  } while (x >= lim);
  return x % bound;
}

/* ------------------------------------------------------ thread fan-out */

typedef void (*voter_fn)(void* ctx, int64_t v0, int64_t v1);

typedef struct {
  voter_fn fn;
  void* ctx;
  int64_t v0, v1;
} span_t;

static void* span_main(void* a) {
  span_t* s = (span_t*)a;
  s->fn(s->ctx, s->v0, s->v1);
  return NULL;
}

static void run_voters(voter_fn fn, void* ctx, int64_t n, int nthreads) {
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  if (n < 4096 || nthreads == 1) {
    fn(ctx, 0, n);
    return;
  }
  pthread_t th[256];
  span_t sp[256];
  int64_t chunk = (n + nthreads - 1) / nthreads;
  int used = 0;
  for (int t = 0; t < nthreads; ++t) {
    int64_t a = (int64_t)t * chunk, b = a + chunk;
    if (a >= n) break;
    if (b > n) b = n;
    sp[t].fn = fn;
    sp[t].ctx = ctx;
    sp[t].v0 = a;
    sp[t].v1 = b;
    if (pthread_create(&th[t], NULL, span_main, &sp[t]) != 0) {
      fn(ctx, a, b); /* could not start a thread: do the span here */
      sp[t].fn = NULL;
    }
    used = t + 1;
  }
  for (int t = 0; t < used; ++t)
    if (sp[t].fn) pthread_join(th[t], NULL);
}

/* ----------------------------------------------------- permutations */

/* Uniform random permutation of 0..m-1 (Fisher-Yates). */
void gen_permutation(uint64_t seed, int32_t m, int32_t* out) {
  rng_t r = rng_for(seed, 0xFFFFFFFFFFFFULL);
  for (int32_t i = 0; i < m; ++i) out[i] = i;
  for (int32_t i = m - 1; i > 0; --i) {
    int32_t j = (int32_t)rng_below(&r, (uint64_t)i + 1);
    int32_t t = out[i];
    out[i] = out[j];
    out[j] = t;
  }
}

/* --------------------------------------------------- impartial culture */

typedef struct {
  uint64_t seed;
  int64_t n;
  int32_t m, k;
  int32_t* out;
} ic_ctx;

static void ic_span(void* c_, int64_t v0, int64_t v1) {
  ic_ctx* c = (ic_ctx*)c_;
  int32_t* perm = (int32_t*)malloc(sizeof(int32_t) * (size_t)c->m);
  for (int64_t v = v0; v < v1; ++v) {
    rng_t r = rng_for(c->seed, (uint64_t)v);
    for (int32_t i = 0; i < c->m; ++i) perm[i] = i;
    int32_t* row = c->out + v * c->k;
    /* partial Fisher-Yates: position q gets a uniform pick among the rest */
    for (int32_t q = 0; q < c->k; ++q) {
      int32_t j = q + (int32_t)rng_below(&r, (uint64_t)(c->m - q));
      int32_t t = perm[q];
      perm[q] = perm[j];
      perm[j] = t;
      row[q] = perm[q];
    }
  }
  free(perm);
}

/* Impartial culture: every ballot is a uniform random (top-k of a) linear order. */
int gen_impartial(uint64_t seed, int64_t n, int32_t m, int32_t k, int32_t* out, int nthreads) {
  if (n < 0 || m < 1 || k < 0 || k > m || (!out && n * k > 0)) return -1;
  ic_ctx c = {seed, n, m, k, out};
  run_voters(ic_span, &c, n, nthreads);
  return 0;
}

/* ------------------------------------------------------------- Mallows */
/*
 * P(ranking) proportional to phi^(Kendall tau distance to sigma0). Drawn top
 * down: with L candidates left, position q takes the j-th remaining candidate
 * in sigma0 order with probability proportional to phi^j, j = 0..L-1 (the
 * inversion-vector entries of a Mallows ranking are independent truncated
 * geometrics). Stopping after k positions gives the top-k marginal.
 * cum[t] = sum_{j<t} phi^j is built by repeated multiplication (no libm),
 * and j is found by binary search of u * cum[L].
 */

typedef struct {
  uint64_t seed;
  int64_t n;
  int32_t m, k;
  double phi;
  const int32_t* sigma0;
  const double* cum; /* [m + 1] */
  int32_t* out;
} mallows_ctx;

static int32_t trunc_geometric(rng_t* r, double phi, const double* cum, int32_t L) {
  if (phi >= 1.0) return (int32_t)rng_below(r, (uint64_t)L);
  double x = rng_u01(r) * cum[L];
  /* first t in [1, L] with cum[t] > x, j = t - 1 */
  int32_t lo = 1, hi = L;
  if (!(cum[L] > x)) return L - 1;
  while (lo < hi) {
    int32_t mid = lo + (hi - lo) / 2;
    if (cum[mid] > x)
      hi = mid;
    else
      lo = mid + 1;
  }
  return lo - 1;
}

static void mallows_span(void* c_, int64_t v0, int64_t v1) {
  mallows_ctx* c = (mallows_ctx*)c_;
  const int32_t m = c->m, k = c->k;
  int32_t* fen = NULL;    /* Fenwick tree over sigma0 slots (full/long ballots) */
  int32_t* taken = NULL;  /* sorted taken slots (short ballots) */
  int use_fenwick = k > 64;
  if (use_fenwick)
    fen = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m + 1));
  else
    taken = (int32_t*)malloc(sizeof(int32_t) * (size_t)(k + 1));
  int32_t logm = 1;
  while ((1 << logm) <= m) ++logm;
  for (int64_t v = v0; v < v1; ++v) {
    rng_t r = rng_for(c->seed, (uint64_t)v);
    int32_t* row = c->out + v * k;
    if (use_fenwick) {
      for (int32_t i = 1; i <= m; ++i) fen[i] = i & (-i); /* all slots free */
    }
    int32_t ntaken = 0;
    for (int32_t q = 0; q < k; ++q) {
      int32_t L = m - q;
      int32_t j = trunc_geometric(&r, c->phi, c->cum, L);
      int32_t slot;
      if (use_fenwick) {
        /* smallest slot whose prefix count of free slots is j + 1 */
        int32_t pos = 0, rem = j + 1;
        for (int32_t b = logm; b >= 0; --b) {
          int32_t nxt = pos + (1 << b);
          if (nxt <= m && fen[nxt] < rem) {
            pos = nxt;
            rem -= fen[nxt];
          }
        }
        slot = pos; /* 0-based slot = (pos + 1) - 1 */
        for (int32_t i = pos + 1; i <= m; i += i & (-i)) fen[i] -= 1;
      } else {
        /* j-th free slot: walk the sorted taken list */
        slot = j;
        int32_t t = 0;
        while (t < ntaken && taken[t] <= slot) {
          ++slot;
          ++t;
        }
        /* insert slot keeping taken sorted */
        int32_t ins = ntaken;
        while (ins > 0 && taken[ins - 1] > slot) {
          taken[ins] = taken[ins - 1];
          --ins;
        }
        taken[ins] = slot;
        ++ntaken;
      }
      row[q] = c->sigma0 ? c->sigma0[slot] : slot;
    }
  }
  free(fen);
  free(taken);
}

/* sigma0 == NULL means the identity reference order. */
int gen_mallows(uint64_t seed, int64_t n, int32_t m, int32_t k, double phi, const int32_t* sigma0, int32_t* out,
                int nthreads) {
  if (n < 0 || m < 1 || k < 0 || k > m || !(phi > 0.0) || phi > 1.0 || (!out && n * k > 0)) return -1;
  double* cum = (double*)malloc(sizeof(double) * (size_t)(m + 1));
  if (!cum) return -2;
  double pw = 1.0;
  cum[0] = 0.0;
  for (int32_t t = 1; t <= m; ++t) {
    cum[t] = cum[t - 1] + pw;
    pw = pw * phi;
  }
  mallows_ctx c = {seed, n, m, k, phi, sigma0, cum, out};
  run_voters(mallows_span, &c, n, nthreads);
  free(cum);
  return 0;
}

/* ------------------------------------------------ Plackett-Luce, Zipf */
/*
 * Item with popularity rank r (0-based) has weight (r + 1)^(-s); ids are
 * assigned to popularity ranks by `perm` (NULL = identity). A ballot draws k
 * distinct items sequentially, each with probability proportional to its
 * weight among the items not yet drawn: draw from a Vose alias table and
 * reject repeats.
 */

typedef struct {
  uint64_t seed;
  int64_t n;
  int32_t m, k;
  const double* prob;
  const int32_t* alias;
  const int32_t* perm;
  int32_t* out;
} pl_ctx;

static void pl_span(void* c_, int64_t v0, int64_t v1) {
  pl_ctx* c = (pl_ctx*)c_;
  const int32_t k = c->k;
  for (int64_t v = v0; v < v1; ++v) {
    rng_t r = rng_for(c->seed, (uint64_t)v);
    int32_t* row = c->out + v * k;
    for (int32_t q = 0; q < k; ++q) {
      int32_t item;
      for (;;) {
        int32_t b = (int32_t)rng_below(&r, (uint64_t)c->m);
        double u = rng_u01(&r);
        item = (u < c->prob[b]) ? b : c->alias[b];
        int dup = 0;
        for (int32_t t = 0; t < q; ++t)
          if (row[t] == item) {
            dup = 1;
            break;
          }
        if (!dup) break;
      }
      row[q] = item;
    }
    if (c->perm)
      for (int32_t q = 0; q < k; ++q) row[q] = c->perm[row[q]];
  }
}

int gen_plackett_luce_zipf(uint64_t seed, int64_t n, int32_t m, int32_t k, double s, const int32_t* perm,
                           int32_t* out, int nthreads) {
  if (n < 0 || m < 1 || k < 0 || k > m || (!out && n * k > 0)) return -1;
  /* rejection sampling stalls when almost every item is drawn; keep k modest */
  if (k > m / 2 + 1 && m > 2) return -1;
  double* w = (double*)malloc(sizeof(double) * (size_t)m);
  double* prob = (double*)malloc(sizeof(double) * (size_t)m);
  int32_t* alias = (int32_t*)malloc(sizeof(int32_t) * (size_t)m);
  int32_t* small = (int32_t*)malloc(sizeof(int32_t) * (size_t)m);
  int32_t* large = (int32_t*)malloc(sizeof(int32_t) * (size_t)m);
  if (!w || !prob || !alias || !small || !large) {
    free(w), free(prob), free(alias), free(small), free(large);
    return -2;
  }
  double tot = 0.0;
  for (int32_t r = 0; r < m; ++r) {
    w[r] = pow((double)(r + 1), -s);
    tot += w[r];
  }
  /* Vose's alias method */
  int32_t ns = 0, nl = 0;
  for (int32_t r = 0; r < m; ++r) {
    prob[r] = w[r] * (double)m / tot;
    if (prob[r] < 1.0)
      small[ns++] = r;
    else
      large[nl++] = r;
  }
  while (ns > 0 && nl > 0) {
    int32_t a = small[--ns], g = large[--nl];
    alias[a] = g;
    prob[g] = (prob[g] + prob[a]) - 1.0;
    if (prob[g] < 1.0)
      small[ns++] = g;
    else
      large[nl++] = g;
  }
  while (nl > 0) {
    int32_t g = large[--nl];
    prob[g] = 1.0;
    alias[g] = g;
  }
  while (ns > 0) {
    int32_t a = small[--ns];
    prob[a] = 1.0;
    alias[a] = a;
  }
  pl_ctx c = {seed, n, m, k, prob, alias, perm, out};
  run_voters(pl_span, &c, n, nthreads);
  free(w), free(prob), free(alias), free(small), free(large);
  return 0;
}

/* ------------------------------------------------------ many elections */

typedef struct {
  uint64_t seed;
  int32_t E;
  const int32_t *kind, *n, *m, *k;
  const double* phi;
  const int64_t* off;
  int32_t* out;
  volatile int32_t next;
  pthread_mutex_t lock;
} batch_ctx;

static void* batch_worker(void* a) {
  batch_ctx* b = (batch_ctx*)a;
  int32_t* sigma = NULL;
  int32_t cap = 0;
  for (;;) {
    pthread_mutex_lock(&b->lock);
    int32_t e = b->next++;
    pthread_mutex_unlock(&b->lock);
    if (e >= b->E) break;
    uint64_t es = b->seed * 1000003ULL + (uint64_t)e;
    int32_t* dst = b->out + b->off[e];
    if (b->kind[e] == 0) {
      if (b->m[e] > cap) {
        free(sigma);
        cap = b->m[e];
        sigma = (int32_t*)malloc(sizeof(int32_t) * (size_t)cap);
      }
      gen_permutation(es ^ 0x33, b->m[e], sigma);
      gen_mallows(es, b->n[e], b->m[e], b->k[e], b->phi[e], sigma, dst, 1);
    } else {
      gen_impartial(es, b->n[e], b->m[e], b->k[e], dst, 1);
    }
  }
  free(sigma);
  return NULL;
}

/* E elections in one buffer: election e's ballots at out + off[e]; kind 0 is
 * Mallows(phi[e]) around a seeded random reference, kind 1 impartial
 * culture. Same ballots as generating each election on its own with seed
 * seed * 1000003 + e; the elections are spread over threads. */
int gen_batch(uint64_t seed, int32_t E, const int32_t* kind, const int32_t* n, const int32_t* m, const int32_t* k,
              const double* phi, const int64_t* off, int32_t* out, int nthreads) {
  if (E < 0) return -1;
  for (int32_t e = 0; e < E; ++e)
    if (n[e] < 0 || m[e] < 1 || k[e] < 0 || k[e] > m[e] || (kind[e] == 0 && (!(phi[e] > 0.0) || phi[e] > 1.0)))
      return -1;
  batch_ctx b;
  b.seed = seed, b.E = E, b.kind = kind, b.n = n, b.m = m, b.k = k, b.phi = phi, b.off = off, b.out = out;
  b.next = 0;
  pthread_mutex_init(&b.lock, NULL);
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  pthread_t th[256];
  int started = 0;
  for (int t = 0; t < nthreads; ++t) {
    if (pthread_create(&th[t], NULL, batch_worker, &b) != 0) break;
    ++started;
  }
  if (started == 0) batch_worker(&b);
  for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
  pthread_mutex_destroy(&b.lock);
  return 0;
}
