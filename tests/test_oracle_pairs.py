"""Pins for the oracle's pairing of mates (the pairing stage after the search):
a hand-worked example (tests/golden/pairing_example.txt) and facts the read
generator fixes (fragment length ~ Normal(500, 50), mates on opposite strands,
chimeric mates from unrelated loci)."""
import os

import numpy as np

import oracle
from synth import Reads, Rng, reference_iid, revcomp_codes, workload

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "pairing_example.txt")
LIM = dict(z_default=0, max_gapo=0, max_gape=0, seed_len=0, seed_z=0, indel_end_skip=5)


def _golden():
    pairs, window = [], None
    for line in open(GOLDEN):
        f = line.split()
        if not f or f[0].startswith("#"):
            continue
        if f[0] == "window":
            window = dict(zip(f[1::2], map(int, f[2::2])))
        elif f[0] == "pair":
            pairs.append(dict(m1=(f[1], int(f[2])), m2=(f[3], int(f[4])), flags=int(f[5]), insert=int(f[6]),
                              n_proper=int(f[7]), pos=f[8:10], strand=f[10:12]))
    return pairs, window


def _hand_text():
    t = reference_iid(3000, Rng(2024, "pair-hand"))
    t[2000:2030] = t[1000:1030]
    t[2600:2630] = t[2550:2580]
    return t


def _mate(t, kind, a):
    if kind == "f":
        return t[a:a + 30]
    if kind == "r":
        return revcomp_codes(t[a - 30:a])
    return reference_iid(30, Rng(7, "pair-x"))


def test_pairing_hand_example():
    pairs, window = _golden()
    t = _hand_text()
    seqs = []
    for p in pairs:
        seqs += [_mate(t, *p["m1"]), _mate(t, *p["m2"])]
    lens = np.array([s.size for s in seqs], np.uint16)
    offs = np.zeros(lens.size, np.uint64)
    offs[1:] = np.cumsum(lens[:-1].astype(np.uint64))
    ox = oracle.OracleIndex(t)
    res, hits, _ = ox.align(np.concatenate(seqs), offs, lens, hit_cap=8, **LIM)
    out, st = ox.pair_resolve(res, hits, max_place=16)
    assert st == window
    for i, p in enumerate(pairs):
        o = out[i]
        assert int(o["flags"]) == p["flags"], (i, int(o["flags"]))
        assert int(o["n_proper"]) == p["n_proper"], i
        assert int(o["insert"]) == p["insert"], i
        if p["pos"][0] == "-":
            assert o["pos"].tolist() == [2 ** 64 - 1] * 2 and o["strand"].tolist() == [255, 255]
        else:
            assert o["pos"].tolist() == [int(x) for x in p["pos"]], i
            assert o["strand"].tolist() == [int(x) for x in p["strand"]], i


def test_pairing_recovers_the_generated_fragments():
    """2 x 100 bp pairs from Normal(500, 50) fragments: the median insert of the
    unique pairs is the fragment mean within 10, the quartile spread that of a
    normal with sd 50; uniquely placed mates pair at their true origins; mates
    from unrelated loci (chimeric pairs) are discordant."""
    w = workload("human_pairs", ref_len=2_000_000, n_reads=3000, seed=12)
    ox = oracle.OracleIndex(w.text)
    lim = w.params
    res, hits, _ = ox.align(w.reads.codes, w.reads.offsets, w.reads.lens, z_default=lim["z"],
                            max_gapo=lim["max_gapo"], max_gape=lim["max_gape"],
                            indel_end_skip=lim["indel_end_skip"], hit_cap=16)
    out, st = ox.pair_resolve(res, hits, max_place=16)
    assert st["n_unique"] > 2000
    assert abs(st["q2"] - 500) <= 10
    assert 50 <= st["q3"] - st["q1"] <= 85          # 1.349 sd = 67 for sd 50
    assert st["lo"] < 400 and st["hi"] > 600
    tp = w.reads.true_pos.astype(np.int64).reshape(-1, 2)
    far = np.abs(tp[:, 0] - tp[:, 1]) > 5000        # mate 2 from an unrelated locus
    uniq = (out["flags"] & oracle.PAIR_UNIQUE) != 0
    proper = (out["flags"] & oracle.PAIR_PROPER) != 0
    near = np.abs(out["pos"].astype(np.int64) - tp).max(axis=1) <= lim["z"]
    assert (proper & near)[uniq & ~far].mean() > 0.98
    both = (out["flags"] & (oracle.PAIR_PLACED1 | oracle.PAIR_PLACED2)) == (oracle.PAIR_PLACED1 | oracle.PAIR_PLACED2)
    assert ((out["flags"] & oracle.PAIR_DISCORDANT) != 0)[far & both].all()
    assert (out["flags"][~(both)] & oracle.PAIR_DISCORDANT == 0).all()
