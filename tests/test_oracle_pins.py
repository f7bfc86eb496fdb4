"""Pins for the CPU oracle against facts that do not come from the oracle itself:
a hand-worked example, naive suffix sorting, occurrence counting, Hamming scans,
a brute-force alignment DP over every substring, LF inversion and invariants."""
import os

import numpy as np
import pytest

import brute
from brute import codes_to_str, str_to_codes
import oracle
from synth import Rng, reference_iid, revcomp_codes, mix64

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_example.txt")


def _golden():
    d = {"sa": {}, "bwt": {}, "text": {}, "exact": [], "hits": []}
    for line in open(GOLDEN):
        if not line.strip() or line.startswith("#"):
            continue
        f = line.split()
        if f[0] in ("text", "bwt"):
            d[f[0]][f[1]] = f[2]
        elif f[0] == "sa":
            d["sa"][f[1]] = [int(x) for x in f[2:]]
        elif f[0] == "C":
            d["C"] = [int(x) for x in f[1:]]
        elif f[0] == "exact":
            d["exact"].append((f[1], f[2], int(f[3]), int(f[4])))
        elif f[0] == "read":
            d["read"] = f[1]
            d["limits"] = dict(zip(f[2::2], map(int, f[3::2])))
        elif f[0] == "hit":
            d["hits"].append(dict(zip(f[1::2], map(int, f[2::2]))))
        elif f[0] == "counts":
            d["counts"] = dict(zip(f[1::2], map(int, f[2::2])))
    return d


def test_hand_example():
    g = _golden()
    X = str_to_codes(g["text"]["X"])
    ix = oracle.OracleIndex(X)
    w = {"X": 0, "Xr": 1}
    for name, which in w.items():
        assert ix.sa(which).tolist() == g["sa"][name]
        assert "".join("ACGT$"[b] for b in ix.bwt(which)) == g["bwt"][name]
        assert ix.C(which).tolist() == g["C"]
    assert codes_to_str(ix.text(1)) == g["text"]["Xr"]
    for name, pat, k, l in g["exact"]:
        assert ix.exact(w[name], str_to_codes(pat)) == (k, l)
    W = str_to_codes(g["read"])
    L = g["limits"]
    res, hits, _ = ix.align(W, [0], [W.size], z_default=L["z"], max_gapo=L["gapo"],
                            max_gape=L["gape"], indel_end_skip=L["e"], strata=oracle.FULL,
                            hit_cap=8)
    nh = res[0]["n_hits"]
    assert nh == len(g["hits"])
    pos, npos = ix.positions(hits[0, :nh])
    for j, gh in enumerate(g["hits"]):
        h = hits[0, j]
        assert (h["strand"], h["k"], h["l"], h["n_diff"], h["aligned_len"]) == \
            (gh["strand"], gh["k"], gh["l"], gh["diff"], gh["len"])
        assert npos[j] == 1 and pos[j, 0] == gh["pos"]
    c = g["counts"]
    assert (res[0]["d_best"], res[0]["c0"], res[0]["c1"]) == (c["d_best"], c["c0"], c["c1"])


def _rand_text(n, seed, alphabet=4):
    r = Rng(seed, "pin-text")
    t = reference_iid(n, r)
    if alphabet < 4:
        t = t % alphabet
    return t


@pytest.mark.parametrize("bucket_k", [0, 3, 12])
@pytest.mark.parametrize("n,seed,alpha", [(1, 1, 4), (2, 2, 4), (57, 3, 4), (300, 4, 2),
                                          (1000, 5, 4), (777, 6, 1)])
def test_sa_bwt_against_naive_sort(n, seed, alpha, bucket_k):
    """Suffix arrays against Python's sort of the suffix strings, whatever the
    number of leading symbols the oracle's sort groups by first (suffixes shorter
    than the group key included)."""
    t = _rand_text(n, seed, alpha)
    ix = oracle.OracleIndex(t, threads=4, bucket_k=bucket_k)
    s = codes_to_str(t)
    assert ix.sa(0).tolist() == brute.naive_sa(s)
    assert ix.sa(1).tolist() == brute.naive_sa(s[::-1])
    # BWT definition and C, Occ against plain counting
    for which, y in ((0, t), (1, t[::-1])):
        sa = ix.sa(which)
        B = ix.bwt(which)
        exp = np.where(sa == 0, 4, y[(sa.astype(np.int64) - 1) % max(1, n)])
        assert np.array_equal(B, exp)
        assert ix.C(which).tolist() == [int((y < c).sum()) for c in range(4)]
        rows = np.random.default_rng(seed).integers(-1, n + 1, 40)
        for r in rows:
            for c in range(4):
                assert ix.occ(which, c, int(r)) == int((B[:r + 1] == c).sum())


@pytest.mark.parametrize("n,seed", [(500, 11), (5000, 12), (4096, 13)])
def test_lf_inverts_bwt(n, seed):
    """Walking LF from the primary row regenerates the text backwards (LF is the
    inverse of the BWT)."""
    t = _rand_text(n, seed)
    ix = oracle.OracleIndex(t)
    for which, y in ((0, t), (1, t[::-1])):
        B = ix.bwt(which)
        C = ix.C(which)
        r = 0  # row of the suffix "$": B[0] is the last text symbol
        out = []
        for _ in range(n):
            c = int(B[r])
            assert c < 4
            out.append(c)
            r = int(C[c]) + ix.occ(which, c, r - 1) + 1
        assert r == ix.primary(which) or n == 0
        assert np.array_equal(np.array(out[::-1], np.uint8), y)


@pytest.mark.parametrize("seed", [21, 22])
def test_exact_interval_is_naive_scan(seed):
    t = _rand_text(800, seed)
    ix = oracle.OracleIndex(t)
    s = codes_to_str(t)
    sa = brute.naive_sa(s)
    rng = np.random.default_rng(seed)
    for _ in range(200):
        L = int(rng.integers(1, 9))
        if rng.random() < 0.6:
            p0 = int(rng.integers(0, len(s) - L))
            p = s[p0:p0 + L]
        else:
            p = "".join(rng.choice(list("ACGT"), L))
        got = ix.exact(0, str_to_codes(p))
        exp = brute.naive_interval(s, sa, p)
        assert got == exp
        cnt = sum(1 for i in range(len(s) - L + 1) if s.startswith(p, i))
        assert (0 if got is None else got[1] - got[0] + 1) == cnt


def _reads_from(t, n_reads, m, seed, n_mut=1, with_n=False):
    rng = np.random.default_rng(seed)
    reads = []
    for _ in range(n_reads):
        p = int(rng.integers(0, t.size - m - 3))
        w = t[p:p + m].copy()
        if rng.random() < 0.5:
            w = revcomp_codes(w)
        for _ in range(int(rng.integers(0, n_mut + 1))):
            op = rng.integers(0, 3)
            j = int(rng.integers(0, m))
            if op == 0:
                w[j] = (w[j] + 1 + rng.integers(0, 3)) % 4
            elif op == 1 and 2 < j < m - 3:
                w = np.concatenate([w[:j], [rng.integers(0, 4)], w[j:-1]]).astype(np.uint8)
            elif op == 2 and 2 < j < m - 3:
                w = np.concatenate([w[:j], w[j + 1:], [t[(p + m) % t.size]]]).astype(np.uint8)
        if with_n and rng.random() < 0.3:
            w[int(rng.integers(0, m))] = 4
        reads.append(w.astype(np.uint8))
    return reads


def _batch(reads):
    lens = np.array([r.size for r in reads], np.uint16)
    offs = np.zeros(len(reads), np.uint64)
    offs[1:] = np.cumsum(lens[:-1].astype(np.uint64))
    return np.concatenate(reads) if reads else np.zeros(0, np.uint8), offs, lens


def test_z0_is_exact_matching():
    """With z = 0 the hit set is exact matching: width = number of occurrences."""
    t = _rand_text(3000, 31)
    s = codes_to_str(t)
    ix = oracle.OracleIndex(t)
    reads = _reads_from(t, 60, 12, 32, n_mut=0)
    codes, offs, lens = _batch(reads)
    res, hits, _ = ix.align(codes, offs, lens, z_default=0, max_gapo=0, max_gape=0,
                            strata=oracle.FULL, hit_cap=4)
    for i, w in enumerate(reads):
        ws = codes_to_str(w)
        rc = codes_to_str(revcomp_codes(w))
        cf = sum(1 for p in range(len(s)) if s.startswith(ws, p))
        cr = sum(1 for p in range(len(s)) if s.startswith(rc, p))
        got = {int(h["strand"]): int(h["l"] - h["k"] + 1) for h in hits[i, :res[i]["n_hits"]]}
        assert got.get(0, 0) == cf and got.get(1, 0) == cr
        assert res[i]["c0"] == cf + cr


@pytest.mark.parametrize("z", [1, 2, 3])
def test_mismatch_only_is_hamming_scan(z):
    """With no gaps the hits are the windows within Hamming distance z (N always
    mismatches): compare widths per distance with a numpy scan over all windows."""
    t = _rand_text(2500, 40 + z, alphabet=4)
    ix = oracle.OracleIndex(t)
    m = 10
    reads = _reads_from(t, 40, m, 41 + z, n_mut=z, with_n=True)
    reads = [r[:m] if r.size >= m else np.pad(r, (0, m - r.size)) for r in reads]
    codes, offs, lens = _batch(reads)
    res, hits, _ = ix.align(codes, offs, lens, z_default=z, max_gapo=0, max_gape=0,
                            strata=oracle.FULL, hit_cap=255)
    win = np.lib.stride_tricks.sliding_window_view(t, m)
    for i, w in enumerate(reads):
        exp = {}
        for strand, q in ((0, w), (1, revcomp_codes(w))):
            d = ((win != q[None, :]) | (q[None, :] == 4)).sum(axis=1)
            for dd in range(z + 1):
                c = int((d == dd).sum())
                if c:
                    exp[(strand, dd)] = c
        got = {}
        for h in hits[i, :res[i]["n_hits"]]:
            key = (int(h["strand"]), int(h["n_diff"]))
            got[key] = got.get(key, 0) + int(h["l"] - h["k"] + 1)
        assert got == exp


CASES = [
    # (n, m, limits, n_reads, seed)
    (120, 10, dict(z=2, max_gapo=1, max_gape=1, seed_len=0, seed_z=0, e=2), 6, 50),
    (150, 12, dict(z=2, max_gapo=1, max_gape=2, seed_len=0, seed_z=0, e=3), 6, 51),
    (90, 9, dict(z=3, max_gapo=2, max_gape=1, seed_len=0, seed_z=0, e=1), 4, 52),
    (100, 11, dict(z=2, max_gapo=1, max_gape=1, seed_len=5, seed_z=1, e=2), 6, 53),
    (80, 8, dict(z=2, max_gapo=1, max_gape=1, seed_len=0, seed_z=0, e=0), 5, 54),
    (60, 7, dict(z=3, max_gapo=1, max_gape=2, seed_len=3, seed_z=0, e=1), 4, 55),
]


@pytest.mark.parametrize("n,m,lim,n_reads,seed", CASES)
@pytest.mark.parametrize("strata", ["FULL", "BEST1"])
def test_against_brute_force(n, m, lim, n_reads, seed, strata):
    """The oracle's hit set, witnesses, c0/c1 and order equal the brute-force DP
    over every substring of the text (FULL and BEST1)."""
    t = _rand_text(n, seed, alphabet=4 if seed % 2 else 2)
    X = codes_to_str(t)
    ix = oracle.OracleIndex(t)
    reads = _reads_from(t, n_reads, m, seed + 100, n_mut=2, with_n=True)
    codes, offs, lens = _batch(reads)
    res, hits, _ = ix.align(codes, offs, lens, z_default=lim["z"], max_gapo=lim["max_gapo"],
                            max_gape=lim["max_gape"], seed_len=lim["seed_len"],
                            seed_z=lim["seed_z"], indel_end_skip=lim["e"], hit_cap=255,
                            strata=oracle.FULL if strata == "FULL" else oracle.BEST1)
    for i, w in enumerate(reads):
        exp, d_best, c0, c1, _ = brute.brute_hits(X, list(w), z=lim["z"], max_gapo=lim["max_gapo"],
                                                  max_gape=lim["max_gape"], seed_len=lim["seed_len"],
                                                  seed_z=lim["seed_z"], e=lim["e"], strata=strata)
        got = [(int(h["strand"]), int(h["k"]), int(h["l"]), int(h["n_diff"]), int(h["n_gapo"]),
                int(h["n_gape"]), int(h["n_mm"]), int(h["aligned_len"]))
               for h in hits[i, :res[i]["n_hits"]]]
        assert got == exp, (codes_to_str(w), lim)
        assert int(res[i]["d_best"]) == d_best
        assert (int(res[i]["c0"]), int(res[i]["c1"])) == (c0, c1)


SCORE_CASES = [
    (300, 16, dict(z=3, max_gapo=1, max_gape=1, seed_len=0, seed_z=0, e=2), 14, 51, (3, 11, 4), 0),
    (250, 14, dict(z=3, max_gapo=2, max_gape=2, seed_len=0, seed_z=0, e=1), 14, 52, (1, 2, 1), 0),
    (200, 12, dict(z=2, max_gapo=1, max_gape=1, seed_len=6, seed_z=1, e=1), 12, 56, (3, 11, 4), 1),
    (120, 10, dict(z=2, max_gapo=1, max_gape=1, seed_len=0, seed_z=0, e=1), 12, 54, (2, 3, 1), 2),
]


@pytest.mark.parametrize("case", range(len(SCORE_CASES)))
def test_score_mode_against_brute_force(case):
    """Score-ordered mode: hits with their least witness by penalty score, the
    best and second-best score strata, c0 / c1, the best score, d_best and the
    cap on equally best places, against the brute-force DP over every substring
    (two-letter texts give many near-equal places, so the cap is exercised)."""
    n, m, lim, n_reads, seed, score, max_best = SCORE_CASES[case]
    t = _rand_text(n, seed, alphabet=4 if seed % 2 else 2)
    X = codes_to_str(t)
    ix = oracle.OracleIndex(t)
    reads = _reads_from(t, n_reads, m, seed + 100, n_mut=2, with_n=True)
    codes, offs, lens = _batch(reads)
    res, hits, _ = ix.align(codes, offs, lens, z_default=lim["z"], max_gapo=lim["max_gapo"],
                            max_gape=lim["max_gape"], seed_len=lim["seed_len"], seed_z=lim["seed_z"],
                            indel_end_skip=lim["e"], hit_cap=255, strata=oracle.SCORE, score=score,
                            max_best=max_best)
    many_seen = 0
    for i, w in enumerate(reads):
        exp, d_best, c0, c1, _, s1, many = brute.brute_hits(
            X, list(w), z=lim["z"], max_gapo=lim["max_gapo"], max_gape=lim["max_gape"],
            seed_len=lim["seed_len"], seed_z=lim["seed_z"], e=lim["e"], strata="SCORE", score=score,
            max_best=max_best)
        got = [(int(h["strand"]), int(h["k"]), int(h["l"]), int(h["n_diff"]), int(h["n_gapo"]),
                int(h["n_gape"]), int(h["n_mm"]), int(h["aligned_len"]))
               for h in hits[i, :res[i]["n_hits"]]]
        assert got == exp, (codes_to_str(w), lim, score)
        assert (int(res[i]["d_best"]), int(res[i]["c0"]), int(res[i]["c1"])) == (d_best, c0, c1)
        assert int(res[i]["pad"]) == s1  # 255 without a hit
        assert bool(res[i]["flags"] & oracle.FLAG_MANY_BEST) == many
        many_seen += many
    if max_best:
        assert many_seen > 0


def test_positions_match_brute_force():
    t = _rand_text(400, 61)
    X = codes_to_str(t)
    ix = oracle.OracleIndex(t)
    reads = _reads_from(t, 10, 9, 62, n_mut=1)
    codes, offs, lens = _batch(reads)
    res, hits, _ = ix.align(codes, offs, lens, z_default=2, max_gapo=1, max_gape=1,
                            indel_end_skip=2, hit_cap=64, strata=oracle.FULL)
    for i in range(len(reads)):
        hs = hits[i, :res[i]["n_hits"]]
        pos, npos = ix.positions(hs, 16)
        for j, h in enumerate(hs):
            exp = brute.positions(X, int(h["strand"]), int(h["aligned_len"]), int(h["k"]), int(h["l"]))
            if len(exp) <= 16:
                assert npos[j] == len(exp) and pos[j, :npos[j]].tolist() == exp
                # and the target text at each position aligns with the read's length
                for p in exp:
                    assert 0 <= p <= len(X) - int(h["aligned_len"])
            else:
                assert npos[j] == 0


def test_d_array_properties_and_safety():
    """D[m] = 0, D non-increasing in i, D[0] <= the best difference count on that
    strand, and searching with D disabled gives the same results."""
    t = _rand_text(20000, 71)
    ix = oracle.OracleIndex(t)
    reads = _reads_from(t, 80, 30, 72, n_mut=3, with_n=True)
    codes, offs, lens = _batch(reads)
    kw = dict(z_default=3, max_gapo=1, max_gape=2, indel_end_skip=5, hit_cap=255,
              strata=oracle.FULL)
    r1, h1, l1 = ix.align(codes, offs, lens, use_d=True, **kw)
    r0, h0, l0 = ix.align(codes, offs, lens, use_d=False, **kw)
    assert np.array_equal(r1, r0) and np.array_equal(h1, h0)
    assert (l1 <= l0).all() and l1.sum() < l0.sum()
    for i, w in enumerate(reads):
        for strand in (0, 1):
            D = ix.dscan(strand, w)
            assert D[-1] == 0 and (np.diff(D) <= 0).all()
            ds = [int(h["n_diff"]) for h in h1[i, :r1[i]["n_hits"]] if h["strand"] == strand]
            if ds:
                assert D[0] <= min(ds)


def test_best1_is_full_filtered():
    t = _rand_text(20000, 81)
    ix = oracle.OracleIndex(t)
    reads = _reads_from(t, 60, 24, 82, n_mut=3, with_n=True)
    codes, offs, lens = _batch(reads)
    kw = dict(z_default=3, max_gapo=1, max_gape=2, indel_end_skip=4, hit_cap=255)
    rf, hf, _ = ix.align(codes, offs, lens, strata=oracle.FULL, **kw)
    rb, hb, _ = ix.align(codes, offs, lens, strata=oracle.BEST1, **kw)
    for i in range(len(reads)):
        full = hf[i, :rf[i]["n_hits"]]
        d = rf[i]["d_best"]
        keep = full[full["n_diff"] <= min(3, int(d) + 1)] if rf[i]["n_hits"] else full
        assert np.array_equal(hb[i, :rb[i]["n_hits"]], keep)
        assert (rb[i]["c0"], rb[i]["c1"], rb[i]["d_best"]) == (rf[i]["c0"], rf[i]["c1"], d)


def test_order_duplication_invariance_and_cap():
    t = _rand_text(30000, 91)
    ix = oracle.OracleIndex(t)
    reads = _reads_from(t, 50, 20, 92, n_mut=2, with_n=True)
    codes, offs, lens = _batch(reads)
    kw = dict(z_default=2, max_gapo=1, max_gape=2, indel_end_skip=5, hit_cap=255)
    r, h, _ = ix.align(codes, offs, lens, **kw)
    perm = np.random.default_rng(93).permutation(len(reads))
    dup = list(perm) + list(perm[:10])
    c2, o2, l2 = _batch([reads[j] for j in dup])
    rr, hh, _ = ix.align(c2, o2, l2, threads=3, **kw)
    assert np.array_equal(rr, r[dup]) and np.array_equal(hh, h[dup])
    # a hit cap truncates the ordered list, sets the overflow flag, keeps c0/c1
    rc, hc, _ = ix.align(codes, offs, lens, **dict(kw, hit_cap=1))
    for i in range(len(reads)):
        nh = int(r[i]["n_hits"])
        assert rc[i]["n_hits"] == min(1, nh)
        assert bool(rc[i]["flags"] & oracle.FLAG_HIT_OVERFLOW) == (nh > 1)
        assert (rc[i]["c0"], rc[i]["c1"]) == (r[i]["c0"], r[i]["c1"])
        if nh:
            assert hc[i, 0] == h[i, 0]


def test_edge_reads():
    t = _rand_text(5000, 101)
    ix = oracle.OracleIndex(t)
    long = np.zeros(256, np.uint8)
    reads = [np.zeros(0, np.uint8), t[100:101].copy(), np.full(12, 4, np.uint8), long,
             t[200:455].copy()]
    codes, offs, lens = _batch(reads)
    z = np.array([2, 0, 2, 2, 8], np.uint8)
    r, h, _ = ix.align(codes, offs, lens, z=z, hit_cap=4)
    assert r[0]["n_hits"] == 0 and r[0]["d_best"] == 255 and r[0]["flags"] == 0
    assert r[1]["n_hits"] >= 1 and r[1]["d_best"] == 0  # single base: exact
    assert r[2]["n_hits"] == 0  # 12 N with z=2: every N mismatches
    assert r[3]["flags"] & oracle.FLAG_READ_TOO_LONG and r[3]["n_hits"] == 0
    assert r[4]["flags"] & oracle.FLAG_BAD_LIMIT and r[4]["n_hits"] == 0


def test_n_in_reference_replaced_by_splitmix():
    """Each N of the text is indexed as mix64(n_seed ^ pos) & 3."""
    t = _rand_text(3000, 111)
    t[100:150] = 4
    t[2999] = 4
    ix = oracle.OracleIndex(t, n_seed=12345)
    exp = t.copy()
    pos = np.nonzero(t == 4)[0].astype(np.uint64)
    exp[t == 4] = (mix64(np.uint64(12345) ^ pos) & np.uint64(3)).astype(np.uint8)
    assert np.array_equal(ix.text(0), exp)
    assert np.array_equal(ix.text(1), exp[::-1])


def _splitmix_vectors():
    out = []
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "splitmix64.txt")):
        f = line.split()
        if f and f[0] == "seed":
            out.append((int(f[1]), [int(x) for x in f[2:]]))
    return out


def test_mix64_matches_published_splitmix64():
    """The oracle's and the input generator's mix64 give SplitMix64's published
    outputs: output i of a generator seeded with s is mix64(s + i * golden)."""
    G = 0x9E3779B97F4A7C15
    vecs = _splitmix_vectors()
    assert len(vecs) == 2
    for seed, outs in vecs:
        for i, v in enumerate(outs):
            st = (seed + i * G) & 0xFFFFFFFFFFFFFFFF
            assert oracle.mix64(st) == v
            assert mix64(st) == v
        arr = mix64(np.array([(seed + i * G) & 0xFFFFFFFFFFFFFFFF for i in range(len(outs))], np.uint64))
        assert arr.tolist() == outs


EDIT_LIMITS = [
    dict(z=2, max_gapo=1, max_gape=1, seed_len=0, seed_z=0, e=1),
    dict(z=2, max_gapo=2, max_gape=1, seed_len=0, seed_z=0, e=2),
    dict(z=2, max_gapo=1, max_gape=1, seed_len=4, seed_z=0, e=1),
    dict(z=1, max_gapo=1, max_gape=0, seed_len=0, seed_z=0, e=0),
]


def _every_edit(w):
    """The read itself and every single edit of it: a substitution to each other
    base, an N, an insertion of each base before every position, a deletion of
    every base."""
    out = [w.copy()]
    m = w.size
    for p in range(m):
        for b in range(5):
            if b != w[p]:
                v = w.copy()
                v[p] = b
                out.append(v)
        out.append(np.delete(w, p))
    for p in range(m + 1):
        for b in range(4):
            out.append(np.insert(w, p, b).astype(np.uint8))
    return out


@pytest.mark.parametrize("li", range(len(EDIT_LIMITS)))
def test_every_position_every_edit(li):
    """Brute force on a tiny text: for a read cut from the text and every single
    edit of it at every position, the oracle equals the brute-force DP."""
    lim = EDIT_LIMITS[li]
    t = _rand_text(70, 200 + li, alphabet=4)
    X = codes_to_str(t)
    ix = oracle.OracleIndex(t)
    w0 = t[20:28].copy()
    reads = _every_edit(w0)
    codes, offs, lens = _batch(reads)
    res, hits, _ = ix.align(codes, offs, lens, z_default=lim["z"], max_gapo=lim["max_gapo"],
                            max_gape=lim["max_gape"], seed_len=lim["seed_len"],
                            seed_z=lim["seed_z"], indel_end_skip=lim["e"], hit_cap=255,
                            strata=oracle.FULL)
    for i, w in enumerate(reads):
        exp, d_best, c0, c1, _ = brute.brute_hits(X, list(w), z=lim["z"], max_gapo=lim["max_gapo"],
                                                  max_gape=lim["max_gape"], seed_len=lim["seed_len"],
                                                  seed_z=lim["seed_z"], e=lim["e"], strata="FULL")
        got = [(int(h["strand"]), int(h["k"]), int(h["l"]), int(h["n_diff"]), int(h["n_gapo"]),
                int(h["n_gape"]), int(h["n_mm"]), int(h["aligned_len"]))
               for h in hits[i, :res[i]["n_hits"]]]
        assert got == exp, (codes_to_str(w), lim)
        assert (int(res[i]["c0"]), int(res[i]["c1"]), int(res[i]["d_best"])) == (c0, c1, d_best)


def test_homopolymer_gap_witness():
    """A read with four C's against a text with two: the two extra C's can be
    inserted adjacent (1 gap open + 1 extension) or apart (2 gap opens), both 2
    differences; the minimal witness is the single gap, as the brute force says."""
    t = _rand_text(70, 200)
    t2 = np.concatenate([t[:40], np.array([0, 1, 1, 2, 3, 2], np.uint8), t[40:]])
    hp = np.array([0, 1, 1, 1, 1, 2, 3, 2], np.uint8)
    ix2 = oracle.OracleIndex(t2)
    r2, h2, _ = ix2.align(hp, [0], [hp.size], z_default=2, max_gapo=2, max_gape=1,
                          indel_end_skip=1, hit_cap=255, strata=oracle.FULL)
    exp, *_ = brute.brute_hits(codes_to_str(t2), list(hp), z=2, max_gapo=2, max_gape=1, e=1,
                               strata="FULL")
    got = [(int(h["strand"]), int(h["k"]), int(h["l"]), int(h["n_diff"]), int(h["n_gapo"]),
            int(h["n_gape"]), int(h["n_mm"]), int(h["aligned_len"])) for h in h2[0, :r2[0]["n_hits"]]]
    assert got == exp
    assert any(g[3] == 2 and g[4] == 1 and g[5] == 1 and g[6] == 0 for g in got)


@pytest.mark.parametrize("seed_z", [0, 1])
def test_every_pair_of_edits_in_seed(seed_z):
    """A deletion (or insertion) and a substitution at every pair of positions,
    with a seed limit: two seed differences exceed seed_z = 1.  Oracle equals the
    brute-force DP."""
    lim = dict(z=3, max_gapo=1, max_gape=1, seed_len=5, seed_z=seed_z, e=1)
    t = _rand_text(80, 300 + seed_z, alphabet=4)
    X = codes_to_str(t)
    ix = oracle.OracleIndex(t)
    w0 = t[30:39].copy()
    reads = []
    for p1 in range(1, w0.size - 1):
        for kind in ("del", "ins"):
            v = np.delete(w0, p1) if kind == "del" else np.insert(w0, p1, (w0[p1] + 1) % 4)
            for p2 in range(0, v.size, 2):
                u = v.copy()
                u[p2] = (u[p2] + 2) % 4
                reads.append(u.astype(np.uint8))
    codes, offs, lens = _batch(reads)
    res, hits, _ = ix.align(codes, offs, lens, z_default=lim["z"], max_gapo=lim["max_gapo"],
                            max_gape=lim["max_gape"], seed_len=lim["seed_len"],
                            seed_z=lim["seed_z"], indel_end_skip=lim["e"], hit_cap=255,
                            strata=oracle.FULL)
    for i, w in enumerate(reads):
        exp, d_best, c0, c1, _ = brute.brute_hits(X, list(w), z=lim["z"], max_gapo=lim["max_gapo"],
                                                  max_gape=lim["max_gape"], seed_len=lim["seed_len"],
                                                  seed_z=lim["seed_z"], e=lim["e"], strata="FULL")
        got = [(int(h["strand"]), int(h["k"]), int(h["l"]), int(h["n_diff"]), int(h["n_gapo"]),
                int(h["n_gape"]), int(h["n_mm"]), int(h["aligned_len"]))
               for h in hits[i, :res[i]["n_hits"]]]
        assert got == exp, (codes_to_str(w), lim)
