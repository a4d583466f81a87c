"""Test-side constructions that pin the oracle to the paper and to mathematics.

Everything here is written independently of both the oracle and the CUDA
library: fixture parsing, McGarvey's construction (Sect. 3), the NL-hardness
reduction of Sect. 3, brute-force path enumeration, breadth-first search and
the Schwartz set (Sect. 2.1).
"""
from __future__ import annotations

import itertools
import os
from collections import deque

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _lines(name):
    with open(os.path.join(GOLDEN, name)) as f:
        for ln in f:
            ln = ln.strip()
            if ln and not ln.startswith("#"):
                yield ln.split()


def fig1():
    """Figure 1 of the paper: (names, margin matrix mu, width table p, winners)."""
    names, edges, rows, win = None, [], {}, []
    for tok in _lines("fig1_tournament.txt"):
        if tok[0] == "candidates":
            names = tok[1:]
        elif tok[0] == "edge":
            edges.append((tok[1], tok[2], int(tok[3])))
        elif tok[0] == "width":
            rows[tok[1]] = tok[2:]
        elif tok[0] == "winners":
            win = tok[1:]
    idx = {c: i for i, c in enumerate(names)}
    m = len(names)
    mu = np.zeros((m, m), dtype=np.int32)
    for u, v, wt in edges:
        mu[idx[u], idx[v]] = wt
    p = np.zeros((m, m), dtype=np.int32)
    for r, vals in rows.items():
        for j, t in enumerate(vals):
            p[idx[r], j] = 0 if t == "-" else int(t)
    return names, mu, p, sorted(idx[c] for c in win)


def topk_tie_counterexample():
    out = {"ballots": [], "d": [], "p": []}
    for tok in _lines("topk_tie_counterexample.txt"):
        key, vals = tok[0], [int(x) for x in tok[1:]]
        if key in ("ballot", "d", "p"):
            out["ballots" if key == "ballot" else key].append(vals)
        else:
            out[key] = vals[0] if key == "m" else vals
    out["ballots"] = np.array(out["ballots"], dtype=np.int32)
    out["d"] = np.array(out["d"], dtype=np.int32)
    out["p"] = np.array(out["p"], dtype=np.int32)
    return out


def mcgarvey_ballots(mu: np.ndarray) -> np.ndarray:
    """McGarvey's construction (cited in Sect. 3): for an asymmetric graph with
    even weights, mu(x,y)/2 pairs of linear orders (x, y, rest ascending) and
    (rest descending, x, y) realise exactly the margins mu."""
    m = mu.shape[0]
    out = []
    for x in range(m):
        for y in range(m):
            if mu[x, y] > 0:
                assert mu[x, y] % 2 == 0 and mu[y, x] == 0
                rest = [c for c in range(m) if c not in (x, y)]
                for _ in range(int(mu[x, y]) // 2):
                    out.append([x, y] + rest)
                    out.append(rest[::-1] + [x, y])
    return np.array(out, dtype=np.int32).reshape(-1, m)


def brute_force_widths(w: np.ndarray) -> np.ndarray:
    """p[i][j] = max over all simple paths i -> j of the minimum edge weight,
    0 if there is none (edges are the entries w > 0). Exponential; m <= 8."""
    m = w.shape[0]
    p = np.zeros((m, m), dtype=np.int64)
    adj = [[j for j in range(m) if j != i and w[i, j] > 0] for i in range(m)]

    def dfs(src, u, width, seen):
        for v in adj[u]:
            if v in seen:
                continue
            wd = min(width, int(w[u, v]))
            if wd > p[src, v]:
                p[src, v] = wd
            seen.add(v)
            dfs(src, v, wd, seen)
            seen.remove(v)

    for s in range(m):
        dfs(s, s, 1 << 62, {s})
    for i in range(m):
        p[i, i] = 0
    return p.astype(np.int32)


def reachable(adj: dict, a, b) -> bool:
    q, seen = deque([a]), {a}
    while q:
        u = q.popleft()
        if u == b:
            return True
        for v in adj.get(u, ()):
            if v not in seen:
                seen.add(v)
                q.append(v)
    return False


def nl_reduction(n_vertices: int, edges, a: int, b: int):
    """The weighted tournament graph of the NL-hardness proof (Sect. 3).

    Returns (mu, a_index, b_index). Steps: drop edges into a and out of b;
    replace one edge of every symmetric pair by a midpoint; for every vertex
    u != b (midpoints included, the r-vertices themselves excluded) add r_u
    with edges b -> r_u -> u; the edge r_a -> a weighs 2, every other edge 4.
    """
    E = {(u, v) for (u, v) in edges if u != v and v != a and u != b}
    verts = list(range(n_vertices))
    final = set()
    for (u, v) in sorted(E):
        if (v, u) in E and u < v:
            mid = len(verts)
            verts.append(mid)
            final.add((u, mid))
            final.add((mid, v))
        else:
            final.add((u, v))
    base = list(verts)
    r_of = {}
    for u in base:
        if u == b:
            continue
        r = len(verts)
        verts.append(r)
        r_of[u] = r
        final.add((b, r))
        final.add((r, u))
    m = len(verts)
    mu = np.zeros((m, m), dtype=np.int32)
    for (u, v) in final:
        mu[u, v] = 4
    mu[r_of[a], a] = 2
    return mu


def schwartz_set(d: np.ndarray) -> set:
    """Union of the SCCs of the dominance graph with no edge entering them
    from outside (Sect. 2.1). Tarjan-free: via reachability closure."""
    m = d.shape[0]
    dom = d > d.T
    reach = dom.copy()
    np.fill_diagonal(reach, True)
    for k in range(m):  # boolean transitive closure (Warshall)
        reach = reach | (reach[:, [k]] & reach[[k], :])
    out = set()
    for c in range(m):
        # c is in the Schwartz set iff every x that reaches c is reached back by c
        if all(reach[c, x] for x in range(m) if reach[x, c]):
            out.add(c)
    return out


def single_voter_matrix(ballot, m):
    """d for one ballot: 1 where i is listed above j or i listed and j not."""
    k = len(ballot)
    pos = {c: q for q, c in enumerate(ballot)}
    d = np.zeros((m, m), dtype=np.int32)
    for i in range(m):
        for j in range(m):
            if i != j and pos.get(i, k) < pos.get(j, k):
                d[i, j] = 1
    return d


def random_digraph(rs, nv, p_edge):
    return [(u, v) for u, v in itertools.permutations(range(nv), 2) if rs.random() < p_edge]
