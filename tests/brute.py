"""Brute-force reference for tiny inputs, written independently of the oracle's
index and search: naive suffix sorting by Python string comparison, and a
set-valued dynamic programme over the (read, target) alignment grid for every
substring T of the text.  Used only to pin the oracle.

The result definition it implements (the method's output as a plain statement):
a read W (codes 0..4, N=4) has a hit (strand, k, l) when some transcript aligns
all of W (forward strand) or its reverse complement (reverse strand) to a
substring T of X under the limits; the interval is that of reverse(T) in the
suffix array of reverse(X) (forward strand) or of T in that of X (reverse
strand).  Read index p counts from W's 5' end on both strands.
"""
from __future__ import annotations

from functools import lru_cache

import numpy as np

ALPHA = "ACGT"


def naive_sa(s: str) -> list[int]:
    """Suffix array of s + '$' with '$' smallest, by sorting the suffix strings."""
    t = s + "\x00"
    return sorted(range(len(t)), key=lambda i: t[i:])


def naive_interval(s: str, sa: list[int], p: str):
    """Closed SA interval of the rows whose suffix starts with p, or None."""
    t = s + "\x00"
    rows = [r for r, i in enumerate(sa) if t.startswith(p, i)]
    if not rows:
        return None
    assert rows == list(range(rows[0], rows[-1] + 1))
    return rows[0], rows[-1]


def _transcripts(Q, U, z, max_gapo, max_gape, seed_len, seed_z, e):
    """All reachable (n_mm, n_gapo, n_gape) at the end of aligning Q (processed in
    read order, p = read index) to U, under the limits.  Set-valued DP."""
    m, L = len(Q), len(U)
    e1 = max(e, 1)
    # state: (p, t) -> set of (last, n_mm, n_gapo, n_gape, seed)
    cur = {(0, 0): {(0, 0, 0, 0, 0)}}
    order = sorted(((p, t) for p in range(m + 1) for t in range(L + 1)))
    reach = {k: set(v) for k, v in cur.items()}
    for (p, t) in order:
        states = reach.get((p, t))
        if not states:
            continue
        for (last, mm, go, ge, sd) in list(states):
            in_seed = seed_len > 0 and p < seed_len
            # match / mismatch
            if p < m and t < L:
                is_mm = Q[p] == 4 or Q[p] != U[t]
                nm, ns = mm + is_mm, sd + (in_seed and is_mm)
                if nm + go + ge <= z and (not seed_len or ns <= seed_z):
                    reach.setdefault((p + 1, t + 1), set()).add((0, nm, go, ge, ns))
            # insertion of Q[p]
            if p < m and e <= p <= m - 1 - e:
                ngo, nge = (go, ge + 1) if last == 1 else (go + 1, ge)
                ns = sd + in_seed
                if ngo <= max_gapo and nge <= max_gape and mm + ngo + nge <= z and \
                        (not seed_len or ns <= seed_z):
                    reach.setdefault((p + 1, t), set()).add((1, mm, ngo, nge, ns))
            # deletion of U[t], placed before read index p
            if t < L and e1 <= p <= m - e1:
                ngo, nge = (go, ge + 1) if last == 2 else (go + 1, ge)
                ns = sd + in_seed
                if ngo <= max_gapo and nge <= max_gape and mm + ngo + nge <= z and \
                        (not seed_len or ns <= seed_z):
                    reach.setdefault((p, t + 1), set()).add((2, mm, ngo, nge, ns))
    return {(mm, go, ge) for (_l, mm, go, ge, _s) in reach.get((m, L), set())}


def brute_hits(X: str, W: list[int], *, z, max_gapo, max_gape, seed_len=0, seed_z=0, e=5,
               strata="FULL", hit_cap=255, score=(3, 11, 4), max_best=0):
    """Full result for one read by brute force.  Returns (hits, d_best, c0, c1, overflow)
    with hits as tuples (strand, k, l, n_diff, n_gapo, n_gape, n_mm, aligned_len) in
    the order (diffs, strand, k, l).  strata "SCORE" (hits ranked by the penalty
    M n_mm + O n_gapo + E n_gape, score = (M, O, E)) returns (hits, d_best, c0,
    c1, overflow, best_score, many_best) instead, hits in the order (score,
    strand, k, l): the best and second-best scores listed, the best only when
    more than max_best (> 0) places have the best score."""
    n = len(X)
    Xr = X[::-1]
    sa_x, sa_r = _sa_cached(X), _sa_cached(Xr)
    m = len(W)
    subs = set()
    for L in range(max(1, m - z), m + z + 1):
        for s in range(0, n - L + 1):
            subs.add(X[s:s + L])
    best = {}
    for strand in (0, 1):
        Q = list(W) if strand == 0 else [(3 - b) if b < 4 else 4 for b in W]
        for T in subs:
            U = [ALPHA.index(ch) for ch in (T if strand == 0 else T[::-1])]
            tr = _transcripts(Q, U, z, max_gapo, max_gape, seed_len, seed_z, e)
            if not tr:
                continue
            if strand == 0:
                iv = naive_interval(Xr, sa_r, T[::-1])
            else:
                iv = naive_interval(X, sa_x, T)
            assert iv is not None
            for (mm, go, ge) in tr:
                w = (mm + go + ge, go, ge, mm, len(T))
                if strata == "SCORE":
                    w = (score[0] * mm + score[1] * go + score[2] * ge,) + w
                key = (strand, iv[0], iv[1])
                if key not in best or w < best[key]:
                    best[key] = w
    if strata == "SCORE":
        if not best:
            return [], 255, 0, 0, False, 255, False
        s1 = min(w[0] for w in best.values())
        higher = [w[0] for w in best.values() if w[0] > s1]
        s2 = min(higher) if higher else None
        c0 = sum(l - k + 1 for (s, k, l), w in best.items() if w[0] == s1)
        c1 = sum(l - k + 1 for (s, k, l), w in best.items() if w[0] == s2)
        d_best = min(w[1] for w in best.values() if w[0] == s1)
        many = max_best > 0 and c0 > max_best
        kept = sorted((w[0], s, k, l, w) for (s, k, l), w in best.items()
                      if w[0] == s1 or (not many and w[0] == s2))
        hits = [(s, k, l, w[1], w[2], w[3], w[4], w[5]) for (_, s, k, l, w) in kept]
        return hits[:hit_cap], d_best, c0, c1, len(hits) > hit_cap, min(s1, 254), many
    if not best:
        return [], 255, 0, 0, False
    d_best = min(w[0] for w in best.values())
    keep_max = z if strata == "FULL" else min(z, d_best + 1)
    kept = [(w[0], s, k, l, w) for (s, k, l), w in best.items() if w[0] <= keep_max]
    kept.sort(key=lambda x: x[:4])
    c0 = sum(l - k + 1 for (d, s, k, l, w) in kept if d == d_best)
    c1 = sum(l - k + 1 for (d, s, k, l, w) in kept if d == d_best + 1)
    hits = [(s, k, l, w[0], w[1], w[2], w[3], w[4]) for (d, s, k, l, w) in kept]
    return hits[:hit_cap], d_best, c0, c1, len(hits) > hit_cap


@lru_cache(maxsize=64)
def _sa_cached(s: str):
    return naive_sa(s)


def positions(X: str, strand: int, T_len: int, k: int, l: int) -> list[int]:
    """Forward-strand start positions of a hit from the naive suffix arrays."""
    n = len(X)
    if strand == 1:
        sa = _sa_cached(X)
        return sorted(sa[r] for r in range(k, l + 1))
    sa = _sa_cached(X[::-1])
    return sorted(n - sa[r] - T_len for r in range(k, l + 1))


def codes_to_str(a) -> str:
    return "".join("ACGTN"[int(c)] for c in a)


def str_to_codes(s: str) -> np.ndarray:
    return np.array(["ACGTN".index(c) for c in s], dtype=np.uint8)
