/*
 * CPU oracle for the Schulze hot path.
 *
 * TEST INFRASTRUCTURE ONLY. This file is the plain, slow definition of what
 * the CUDA library computes; it is used by the tests, by the smoke check and
 * by the CPU-baseline leg of the benchmark, and by nothing in the product
 * path. It shares no code, header or table with the CUDA sources.
 *
 * Paper: Csar, Lackner, Pichler, "Computing the Schulze Method for
 * Large-Scale Preference Data Sets" (arXiv 2505.12976).
 *
 * Conventions (readings of the paper, all integer arithmetic):
 *  - ballots: int32 [n, k] row-major, row v lists candidate ids best first;
 *    candidates a ballot does not list are tied below every listed one;
 *  - d[i][j] = number of voters who strictly prefer i to j (Sect. 2.1,
 *    the counts behind the majority margin);
 *  - edge weights are winning votes: w[i][j] = d[i][j] if d[i][j] > d[j][i],
 *    else 0, and w[i][i] = 0 (the paper weights edges by the margin; the two
 *    agree on winners for full rankings);
 *  - p[i][j] = width of a widest path from i to j (Sect. 2.1), 0 when no path
 *    exists, and p[i][i] = 0;
 *  - i is a winner iff p[i][j] >= p[j][i] for every j (Sect. 2.1);
 *  - beaten_by[i] = #{j : p[j][i] > p[i][j]}; the ranking lists the ids
 *    sorted by (beaten_by, id).
 *
 * Parity pins for every function live in the CPU tests (the worked example of
 * Fig. 1, brute-force path enumeration, Dijkstra rows, tally identities and
 * the NL-hardness family of Sect. 3).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_EINVAL -1
#define ORACLE_ENOMEM -2
#define ORACLE_EDATA -4

/* Check every ballot row: ids in range and pairwise distinct. */
int oracle_validate(const int32_t* ranks, int64_t n, int32_t m, int32_t k) {
  if (n < 0 || m < 1 || k < 0 || k > m) return ORACLE_EINVAL;
  if (n > 0 && k > 0 && !ranks) return ORACLE_EINVAL;
  uint8_t* seen = (uint8_t*)calloc((size_t)m, 1);
  if (!seen) return ORACLE_ENOMEM;
  int rc = ORACLE_OK;
  for (int64_t v = 0; v < n && rc == ORACLE_OK; ++v) {
    const int32_t* row = ranks + v * k;
    for (int32_t q = 0; q < k; ++q) {
      int32_t c = row[q];
      if (c < 0 || c >= m || seen[c]) {
        rc = ORACLE_EDATA;
        break;
      }
      seen[c] = 1;
    }
    for (int32_t q = 0; q < k; ++q)
      if (row[q] >= 0 && row[q] < m) seen[row[q]] = 0;
  }
  free(seen);
  return rc;
}

/*
 * Pairwise tally (Sect. 2.1): d[i][j] = #{v : i is strictly preferred to j
 * by voter v}. Position of an unlisted candidate is k (tied below all listed
 * ones), so voter v prefers i to j iff pos_v(i) < pos_v(j). A candidate at
 * position k is preferred to nobody, so only listed i are visited.
 * O(n * k * m) work; d is int32 [m, m], overwritten.
 */
int oracle_tally(const int32_t* ranks, int64_t n, int32_t m, int32_t k, int32_t* d) {
  int rc = oracle_validate(ranks, n, m, k);
  if (rc) return rc;
  int64_t* acc = (int64_t*)calloc((size_t)m * (size_t)m, sizeof(int64_t));
  int32_t* pos = (int32_t*)malloc(sizeof(int32_t) * (size_t)m);
  if (!acc || !pos) {
    free(acc);
    free(pos);
    return ORACLE_ENOMEM;
  }
  for (int64_t v = 0; v < n; ++v) {
    const int32_t* row = ranks + v * k;
    for (int32_t c = 0; c < m; ++c) pos[c] = k;
    for (int32_t q = 0; q < k; ++q) pos[row[q]] = q;
    for (int32_t q = 0; q < k; ++q) {
      int32_t i = row[q];
      for (int32_t j = 0; j < m; ++j)
        if (j != i && pos[i] < pos[j]) acc[(int64_t)i * m + j] += 1;
    }
  }
  for (int64_t t = 0; t < (int64_t)m * m; ++t) d[t] = (int32_t)acc[t];
  free(acc);
  free(pos);
  return ORACLE_OK;
}

/*
 * Pairwise tally of weak-order ballots in position form (Sect. 2.1: a voter
 * may rank candidates equally): pos[v][c] is the position of c on ballot v,
 * smaller is better, equal positions are tied. d[i][j] = #{v : pos[v][i] <
 * pos[v][j]}; a tied pair counts for neither. Positions must lie in
 * [0, 65534] (else ORACLE_EDATA). O(n * m^2); d is int32 [m, m], overwritten.
 */
int oracle_tally_positions(const int32_t* pos, int64_t n, int32_t m, int32_t* d) {
  if (n < 0 || m < 1 || (n > 0 && !pos) || !d) return ORACLE_EINVAL;
  for (int64_t t = 0; t < n * (int64_t)m; ++t)
    if (pos[t] < 0 || pos[t] > 65534) return ORACLE_EDATA;
  int64_t* acc = (int64_t*)calloc((size_t)m * (size_t)m, sizeof(int64_t));
  if (!acc) return ORACLE_ENOMEM;
  for (int64_t v = 0; v < n; ++v) {
    const int32_t* row = pos + v * m;
    for (int32_t i = 0; i < m; ++i)
      for (int32_t j = 0; j < m; ++j)
        if (row[i] < row[j]) acc[(int64_t)i * m + j] += 1;
  }
  for (int64_t t = 0; t < (int64_t)m * m; ++t) d[t] = (int32_t)acc[t];
  free(acc);
  return ORACLE_OK;
}

/* One tally entry d[i][j], counted voter by voter (for sampled checks of
 * large profiles). Returns -1 on bad arguments. */
int64_t oracle_tally_entry(const int32_t* ranks, int64_t n, int32_t m, int32_t k, int32_t i, int32_t j) {
  if (n < 0 || m < 1 || k < 0 || k > m || i < 0 || i >= m || j < 0 || j >= m) return -1;
  if (i == j) return 0;
  int64_t cnt = 0;
  for (int64_t v = 0; v < n; ++v) {
    const int32_t* row = ranks + v * k;
    int32_t pi = k, pj = k;
    for (int32_t q = 0; q < k; ++q) {
      if (row[q] == i) pi = q;
      if (row[q] == j) pj = q;
    }
    if (pi < pj) cnt += 1;
  }
  return cnt;
}

/* Edge weights, winning votes: w[i][j] = d[i][j] if d[i][j] > d[j][i] else 0. */
void oracle_weights(const int32_t* d, int32_t m, int32_t* w) {
  for (int32_t i = 0; i < m; ++i)
    for (int32_t j = 0; j < m; ++j) {
      int32_t a = d[(int64_t)i * m + j], b = d[(int64_t)j * m + i];
      w[(int64_t)i * m + j] = (i != j && a > b) ? a : 0;
    }
}

/* Edge weights, margins (the paper's weighted tournament graph, Sect. 2.1):
 * w[i][j] = d[i][j] - d[j][i] if positive, else 0. */
void oracle_weights_margin(const int32_t* d, int32_t m, int32_t* w) {
  for (int32_t i = 0; i < m; ++i)
    for (int32_t j = 0; j < m; ++j) {
      int64_t mu = (int64_t)d[(int64_t)i * m + j] - (int64_t)d[(int64_t)j * m + i];
      w[(int64_t)i * m + j] = (i != j && mu > 0) ? (int32_t)mu : 0;
    }
}

static inline int32_t imin(int32_t a, int32_t b) { return a < b ? a : b; }
static inline int32_t imax(int32_t a, int32_t b) { return a > b ? a : b; }

/*
 * Widest paths, all pairs (the classical Floyd-Warshall algorithm in the
 * (max, min) semiring, Sect. 1 and Sect. 4): p starts as w and for every
 * intermediate k, p[i][j] = max(p[i][j], min(p[i][k], p[k][j])) over
 * i != k, j not in {i, k}. The diagonal stays 0. For a fixed k the rows are
 * independent, so they may be spread over threads.
 */
void oracle_closure(const int32_t* w, int32_t m, int32_t* p, int nthreads) {
  const int64_t mm = (int64_t)m * m;
  for (int64_t t = 0; t < mm; ++t) p[t] = w[t];
  for (int32_t i = 0; i < m; ++i) p[(int64_t)i * m + i] = 0;
  (void)nthreads;
  for (int32_t k = 0; k < m; ++k) {
    const int32_t* pk = p + (int64_t)k * m;
#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : 1)
    for (int32_t i = 0; i < m; ++i) {
      if (i == k) continue;
      int32_t* pi = p + (int64_t)i * m;
      const int32_t pik = pi[k];
      for (int32_t j = 0; j < m; ++j) {
        if (j == i || j == k) continue;
        pi[j] = imax(pi[j], imin(pik, pk[j]));
      }
    }
  }
}

/* Winners (Sect. 2.1): i wins iff nobody beats it, i.e. p[i][j] >= p[j][i]
 * for all j != i. win[i] in {0, 1}. */
void oracle_winners(const int32_t* p, int32_t m, int32_t* win) {
  for (int32_t i = 0; i < m; ++i) {
    int32_t ok = 1;
    for (int32_t j = 0; j < m; ++j)
      if (j != i && p[(int64_t)i * m + j] < p[(int64_t)j * m + i]) ok = 0;
    win[i] = ok;
  }
}

/* beaten_by[i] = #{j : p[j][i] > p[i][j]} (how many candidates beat i). */
void oracle_beaten_by(const int32_t* p, int32_t m, int32_t* bb) {
  for (int32_t i = 0; i < m; ++i) {
    int32_t c = 0;
    for (int32_t j = 0; j < m; ++j)
      if (j != i && p[(int64_t)j * m + i] > p[(int64_t)i * m + j]) ++c;
    bb[i] = c;
  }
}

/* Ranking: the ids sorted by (beaten_by, id), by insertion sort. */
void oracle_ranking(const int32_t* p, int32_t m, int32_t* order, int32_t* bb_out) {
  int32_t* bb = (int32_t*)malloc(sizeof(int32_t) * (size_t)m);
  oracle_beaten_by(p, m, bb);
  for (int32_t i = 0; i < m; ++i) {
    int32_t t = i;
    while (t > 0 && (bb[order[t - 1]] > bb[i] || (bb[order[t - 1]] == bb[i] && order[t - 1] > i))) {
      order[t] = order[t - 1];
      --t;
    }
    order[t] = i;
  }
  if (bb_out) memcpy(bb_out, bb, sizeof(int32_t) * (size_t)m);
  free(bb);
}

/*
 * Single-source widest paths by the max-min variant of dense Dijkstra:
 * out[v] = p(s, v) for v != s, out[s] = 0. This is the deterministic form of
 * the wide-path questions WP>= / WP> of Sect. 3 for one source. When
 * `transpose` is set it walks edges backwards and returns out[v] = p(v, s).
 */
void oracle_widest_one(const int32_t* w, int32_t m, int32_t s, int transpose, int32_t* out) {
  uint8_t* done = (uint8_t*)calloc((size_t)m, 1);
  int64_t* best = (int64_t*)malloc(sizeof(int64_t) * (size_t)m);
  for (int32_t v = 0; v < m; ++v) best[v] = -1; /* -1: not reached yet */
  best[s] = INT64_MAX;                          /* the empty path */
  for (int32_t it = 0; it < m; ++it) {
    int32_t u = -1;
    for (int32_t v = 0; v < m; ++v)
      if (!done[v] && best[v] >= 0 && (u < 0 || best[v] > best[u])) u = v;
    if (u < 0) break;
    done[u] = 1;
    for (int32_t v = 0; v < m; ++v) {
      if (done[v]) continue;
      int32_t e = transpose ? w[(int64_t)v * m + u] : w[(int64_t)u * m + v];
      if (e <= 0) continue; /* no edge */
      int64_t cand = best[u] < (int64_t)e ? best[u] : (int64_t)e;
      if (cand > best[v]) best[v] = cand;
    }
  }
  for (int32_t v = 0; v < m; ++v) out[v] = (v == s || best[v] < 0) ? 0 : (int32_t)best[v];
  free(done);
  free(best);
}

/*
 * Several rows (or, with `transpose`, columns) of the closure at once:
 * out[t * m + v] = p(src[t], v) (or p(v, src[t])), each computed by
 * oracle_widest_one; the sources are independent, so they are spread over
 * `nthreads` OpenMP threads. Used for exact checks of single candidates of
 * profiles too large for the full closure.
 */
void oracle_widest_many(const int32_t* w, int32_t m, const int32_t* src, int32_t count, int transpose,
                        int32_t* out, int nthreads) {
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
  for (int32_t t = 0; t < count; ++t) oracle_widest_one(w, m, src[t], transpose, out + (int64_t)t * m);
}

/*
 * Top-k ranking by iterated winner removal (Sect. 4, closing remark: run the
 * method again after removing the Schulze winners). Level t is the winner
 * set of the profile restricted to the candidates not placed in levels
 * 1 .. t-1; pairwise counts do not depend on the other candidates, so the
 * restricted profile's d is d on the remaining rows and columns. Levels are
 * assigned until at least k_top candidates are placed (or all are).
 * level[c] = t >= 1 for a placed candidate, 0 otherwise; *levels = number of
 * levels. margin != 0 uses margin weights instead of winning votes.
 */
int oracle_ranking_iterated(const int32_t* d, int32_t m, int32_t k_top, int margin, int32_t* level,
                            int32_t* levels) {
  if (m < 1 || !d || !level || !levels) return ORACLE_EINVAL;
  int32_t* idx = (int32_t*)malloc(sizeof(int32_t) * (size_t)m);
  int32_t* sd = (int32_t*)malloc(sizeof(int32_t) * (size_t)m * (size_t)m);
  int32_t* sw = (int32_t*)malloc(sizeof(int32_t) * (size_t)m * (size_t)m);
  int32_t* sp = (int32_t*)malloc(sizeof(int32_t) * (size_t)m * (size_t)m);
  int32_t* win = (int32_t*)malloc(sizeof(int32_t) * (size_t)m);
  if (!idx || !sd || !sw || !sp || !win) {
    free(idx), free(sd), free(sw), free(sp), free(win);
    return ORACLE_ENOMEM;
  }
  for (int32_t c = 0; c < m; ++c) level[c] = 0;
  int32_t placed = 0, t = 0;
  while (placed < m && placed < k_top) {
    int32_t r = 0;  /* the remaining candidates, in id order */
    for (int32_t c = 0; c < m; ++c)
      if (level[c] == 0) idx[r++] = c;
    for (int32_t a = 0; a < r; ++a)
      for (int32_t b = 0; b < r; ++b) sd[(int64_t)a * r + b] = d[(int64_t)idx[a] * m + idx[b]];
    if (margin)
      oracle_weights_margin(sd, r, sw);
    else
      oracle_weights(sd, r, sw);
    oracle_closure(sw, r, sp, 1);
    oracle_winners(sp, r, win);
    ++t;
    for (int32_t a = 0; a < r; ++a)
      if (win[a]) level[idx[a]] = t, ++placed;
  }
  *levels = t;
  free(idx), free(sd), free(sw), free(sp), free(win);
  return ORACLE_OK;
}

/*
 * Winners only, by the paper's vertex-centric algorithm (Sect. 4, Alg. 1-4),
 * simulated with synchronous rounds. w: edge weights [m, m] (w > 0 is an
 * edge). Ids are the candidate indices. Readings: a status, once decided,
 * does not change (every mark below only turns 'unknown' into 'loser' or
 * 'winner'); the optional zeroing of edges into dominated SCCs is left out
 * (the graph stays as it is). win[c] = 1 for the winners; *iterations = the
 * number of while-loop iterations, *rounds = propagation rounds in total.
 * Returns ORACLE_EDATA if an iteration decides nothing (never expected).
 */
#define PREGEL_INF 0x7fffffff
#define ST_UNKNOWN 0
#define ST_LOSER 1
#define ST_WINNER 2
int oracle_winners_pregel(const int32_t* w, int32_t m, int32_t* win, int32_t* iterations, int32_t* rounds) {
  if (m < 1 || !w || !win || !iterations || !rounds) return ORACLE_EINVAL;
  int32_t* st = (int32_t*)malloc(sizeof(int32_t) * (size_t)m);
  int32_t* s = (int32_t*)malloc(sizeof(int32_t) * (size_t)m * 8);
  if (!st || !s) {
    free(st), free(s);
    return ORACLE_ENOMEM;
  }
  int32_t *ws = s + m, *t = s + 2 * m, *wt = s + 3 * m;
  int32_t *ns = s + 4 * m, *nws = s + 5 * m, *nt = s + 6 * m, *nwt = s + 7 * m;
  int32_t* lose = (int32_t*)calloc((size_t)m + 1, sizeof(int32_t)); /* loser marks */
  int32_t* scc_lose = (int32_t*)calloc((size_t)m + 1, sizeof(int32_t)); /* SCC labels marked */
  /* Initialisation-of-vertices: heaviest incoming edge above the heaviest
   * outgoing one means some vertex beats c. */
  for (int32_t c = 0; c < m; ++c) {
    int32_t in = 0, out = 0;
    for (int32_t a = 0; a < m; ++a) {
      if (a == c) continue;
      in = imax(in, w[(int64_t)a * m + c]);
      out = imax(out, w[(int64_t)c * m + a]);
    }
    st[c] = in > out ? ST_LOSER : ST_UNKNOWN;
  }
  *iterations = 0, *rounds = 0;
  int rc = ORACLE_OK;
  for (;;) {
    int32_t unknown = 0;
    for (int32_t c = 0; c < m; ++c) unknown += st[c] == ST_UNKNOWN;
    if (!unknown) break;
    ++*iterations;
    /* Preprocessing (Alg. 2) */
    for (int32_t c = 0; c < m; ++c) {
      if (st[c] == ST_UNKNOWN)
        s[c] = t[c] = c, ws[c] = wt[c] = PREGEL_INF;
      else
        s[c] = t[c] = PREGEL_INF, ws[c] = wt[c] = 0;
    }
    /* Forward-Backward-Propagation (Alg. 3): a vertex keeps the smallest id
     * it receives and, for that id, the widest width; rounds until nothing
     * changes. Forward messages travel along edges (u, c), backward ones
     * against them. */
    for (;;) {
      int changed = 0;
      ++*rounds;
      for (int32_t c = 0; c < m; ++c) {
        int32_t bs = s[c], bw = ws[c], bt = t[c], bwt = wt[c];
        for (int32_t u = 0; u < m; ++u) {
          if (u == c) continue;
          const int32_t win_uc = w[(int64_t)u * m + c], w_cu = w[(int64_t)c * m + u];
          if (win_uc > 0 && s[u] != PREGEL_INF) {
            const int32_t cw = imin(ws[u], win_uc);
            if (s[u] < bs) bs = s[u], bw = cw;
            else if (s[u] == bs) bw = imax(bw, cw);
          }
          if (w_cu > 0 && t[u] != PREGEL_INF) {
            const int32_t cw = imin(wt[u], w_cu);
            if (t[u] < bt) bt = t[u], bwt = cw;
            else if (t[u] == bt) bwt = imax(bwt, cw);
          }
        }
        ns[c] = bs, nws[c] = bw, nt[c] = bt, nwt[c] = bwt;
        changed |= bs != s[c] || bw != ws[c] || bt != t[c] || bwt != wt[c];
      }
      for (int32_t c = 0; c < m; ++c) s[c] = ns[c], ws[c] = nws[c], t[c] = nt[c], wt[c] = nwt[c];
      if (!changed) break;
    }
    /* Postprocessing (Alg. 4): collect the loser marks of every vertex, then
     * apply them, then the winner rule. SCC labels are ids (or PREGEL_INF,
     * mapped to slot m). */
    memset(lose, 0, sizeof(int32_t) * ((size_t)m + 1));
    memset(scc_lose, 0, sizeof(int32_t) * ((size_t)m + 1));
    for (int32_t c = 0; c < m; ++c) {
      if (s[c] < t[c]) {
        lose[c] = 1;
      } else if (s[c] > t[c]) {
        lose[t[c]] = 1; /* t[c] is an id here: t < s <= PREGEL_INF */
      } else if (s[c] != PREGEL_INF) {
        if (ws[c] > wt[c]) lose[c] = 1;
        else if (ws[c] < wt[c]) lose[s[c]] = 1;
      }
      for (int32_t v = 0; v < m; ++v) {
        if (v == c || w[(int64_t)v * m + c] <= 0) continue;
        if (s[c] != s[v] || t[c] != t[v]) {
          if (s[c] == t[c])
            scc_lose[s[c] == PREGEL_INF ? m : s[c]] = 1;
          else
            lose[c] = 1;
        }
      }
    }
    int32_t decided = 0;
    for (int32_t c = 0; c < m; ++c) {
      if (st[c] != ST_UNKNOWN) continue;
      const int in_lost_scc = s[c] == t[c] && scc_lose[s[c] == PREGEL_INF ? m : s[c]];
      if (lose[c] || in_lost_scc) st[c] = ST_LOSER, ++decided;
    }
    for (int32_t c = 0; c < m; ++c)
      if (st[c] == ST_UNKNOWN && s[c] == c && t[c] == c) st[c] = ST_WINNER, ++decided;
    if (!decided) {
      rc = ORACLE_EDATA;
      break;
    }
  }
  for (int32_t c = 0; c < m; ++c) win[c] = st[c] == ST_WINNER;
  free(st), free(s), free(lose), free(scc_lose);
  return rc;
}
