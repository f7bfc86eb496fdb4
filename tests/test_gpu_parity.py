"""GPU parity: the CUDA search and SA walk against the oracle, bit-exact, through
the C ABI (the Python binding passes device pointers to libaln_gb300.so)."""
import numpy as np
import pytest

import oracle
import paper_1505_07855_gb300 as aln
from parity_util import compare, oracle_align
from synth import Rng, Reads, reference_iid, simulate_reads, workload, z_for_length

pytestmark = pytest.mark.gpu

MODES = [aln.MODE_PLAIN, aln.MODE_PERSISTENT]
BENCH_KMER = 10  # prefix-trie depth the benchmark uses


@pytest.fixture(scope="module")
def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


class Pair:
    """Product index on the device and the oracle's own index of the same text.
    ``kmers`` lists prefix-trie depths; ``al`` uses the first, ``als[k]`` any."""

    def __init__(self, text, kmer_k=0, n_seed=0, kmers=None):
        self.text = text
        self.ox = oracle.OracleIndex(text, n_seed=n_seed)
        self.als = {}
        for k in (kmers or [kmer_k]):
            hix = aln.Index.build(text, n_seed=n_seed, kmer_k=k)
            self.als[k] = aln.Aligner(hix.to_device(0))
        self.al = self.als[(kmers or [kmer_k])[0]]


@pytest.fixture(scope="module")
def tiny36(cuda):
    w = workload("tiny36")
    return w, Pair(w.text, kmers=[0, 10])


def _run(pair, reads, lim, hit_cap=32, strata=aln.STRATA_BEST1, mode=aln.MODE_PLAIN, z=None, zmax=None,
         kmer=None):
    p = aln.Params.from_limits(lim, hit_cap=hit_cap, strata=strata, mode=mode)
    if zmax is not None:
        p.z = zmax
    al = pair.al if kmer is None else pair.als[kmer]
    return al.align(reads.codes, reads.offsets, reads.lens, p, z=z)


@pytest.mark.parametrize("mode,kmer", [(aln.MODE_PLAIN, 0), (aln.MODE_PERSISTENT, 0),
                                       (aln.MODE_PERSISTENT, 10)])
@pytest.mark.parametrize("strata", [aln.STRATA_BEST1, aln.STRATA_FULL])
def test_tiny36_full_parity(tiny36, mode, kmer, strata):
    """1 Mbp i.i.d. text, 10 000 x 36 bp reads, z=2: every read bit-exact (plain
    form; persistent form without and with a depth-10 prefix-trie table)."""
    w, pair = tiny36
    rg, hg = _run(pair, w.reads, w.params, strata=strata, mode=mode, kmer=kmer)
    ro, ho, _ = oracle_align(pair.ox, w.reads, w.params, 32, strata)
    assert compare(rg, hg, ro, ho, what="tiny36") == 10_000
    assert (rg["n_hits"] > 0).mean() > 0.95


def test_hand_example(cuda):
    enc = {c: i for i, c in enumerate("ACGT")}
    X = np.array([enc[c] for c in "ACGTTACGAT"], np.uint8)
    pair = Pair(X)
    W = np.array([enc[c] for c in "ACGA"], np.uint8)
    reads = Reads(W, np.zeros(1, np.uint64), np.array([4], np.uint16), np.array([1], np.uint8),
                  np.zeros(1, np.int64), np.zeros(1, np.uint8))
    lim = dict(z=1, max_gapo=0, max_gape=0, seed_len=0, seed_z=0, indel_end_skip=5)
    rg, hg = _run(pair, reads, lim, hit_cap=8, strata=aln.STRATA_FULL)
    assert rg[0]["n_hits"] == 3 and (rg[0]["d_best"], rg[0]["c0"], rg[0]["c1"]) == (0, 1, 2)
    assert [(int(h["strand"]), int(h["k"]), int(h["l"])) for h in hg[0, :3]] == [(0, 2, 2), (0, 9, 9), (1, 2, 2)]
    pos, npos = pair.al.positions(hg[0, :3], 16)
    assert npos.tolist() == [1, 1, 1] and pos[:, 0].tolist() == [5, 0, 0]


LIMITS = [
    dict(z=1, max_gapo=0, max_gape=0, seed_len=0, seed_z=0, indel_end_skip=5),
    dict(z=2, max_gapo=1, max_gape=2, seed_len=0, seed_z=0, indel_end_skip=5),
    dict(z=3, max_gapo=2, max_gape=1, seed_len=0, seed_z=0, indel_end_skip=0),
    dict(z=3, max_gapo=1, max_gape=3, seed_len=12, seed_z=1, indel_end_skip=3),
    dict(z=4, max_gapo=1, max_gape=6, seed_len=32, seed_z=2, indel_end_skip=5),
    dict(z=5, max_gapo=1, max_gape=2, seed_len=0, seed_z=0, indel_end_skip=5),
    dict(z=7, max_gapo=2, max_gape=3, seed_len=8, seed_z=3, indel_end_skip=1),
]


@pytest.mark.parametrize("li", range(len(LIMITS)))
@pytest.mark.parametrize("strata", [aln.STRATA_BEST1, aln.STRATA_FULL])
def test_limits_parity(cuda, li, strata):
    """Small texts (several Occ blocks, ragged tails), reads with errors and N,
    across gap / seed / end-window / z settings and both strata."""
    lim = LIMITS[li]
    rng = Rng(1000 + li, "lim")
    text = reference_iid(20_000 + 37 * li, rng.sub("t"))
    kmers = [0, 3 + li, 12]
    pair = Pair(text, kmers=kmers)
    m = [20, 36, 50, 36, 60, 76, 40][li]
    reads = simulate_reads(text, 600, m, rng.sub("r"), sub_rate=(0.02, 0.04), indel_rate=0.005,
                           indel_lens=(1, 2), n_frac=0.1, z=lim["z"])
    ro, ho, _ = oracle_align(pair.ox, reads, lim, 40, strata)
    for mode, k in [(aln.MODE_PLAIN, 0)] + [(aln.MODE_PERSISTENT, k) for k in kmers]:
        rg, hg = _run(pair, reads, lim, hit_cap=40, strata=strata, mode=mode, kmer=k)
        compare(rg, hg, ro, ho, what=f"limits {li} mode {mode} kmer {k}")


def test_mixed_lengths_per_read_z(cuda):
    """Reads of 36..250 bp mixed in one batch with z = min(6, ceil(0.04 len)),
    repeats and N runs in the text (the mixed-length recipe at small scale)."""
    w = workload("human_mixed", ref_len=3_000_000, n_reads=3000, seed=3)
    pair = Pair(w.text, n_seed=7, kmers=[0, 11])
    lim = w.params
    ro, ho, _ = oracle_align(pair.ox, w.reads, lim, 32, oracle.BEST1, z=w.reads.z)
    for mode, k in [(aln.MODE_PLAIN, 0), (aln.MODE_PERSISTENT, 0), (aln.MODE_PERSISTENT, 11)]:
        rg, hg = _run(pair, w.reads, lim, hit_cap=32, mode=mode, z=w.reads.z, zmax=6, kmer=k)
        compare(rg, hg, ro, ho, what=f"mixed mode {mode} kmer {k}")
    # schedule knobs are result-neutral: heavy reads helped at once or only at the
    # end, every shared-memory stack depth, few resident blocks
    for help_after, smem, bps, win, heavy in [(1, 4, 0, 0, 0), (0xFFFFFFFF, 12, 0, 1, 1), (64, 8, 1, 0, 64),
                                              (0, 12, 2, 1, 0xFFFFFFFF)]:
        p = aln.Params.from_limits(lim, hit_cap=32, mode=aln.MODE_PERSISTENT, z=6, help_after=help_after,
                                   smem_stack=smem, blocks_per_sm=bps, l2_window=win, heavy_after=heavy)
        rg, hg = pair.als[11].align(w.reads.codes, w.reads.offsets, w.reads.lens, p, z=w.reads.z)
        compare(rg, hg, ro, ho, what=f"mixed help_after {help_after} smem {smem} blocks {bps} l2 window {win} "
                                     f"heavy_after {heavy}")


@pytest.mark.parametrize("li", [1, 4, 6])
@pytest.mark.parametrize("strata", [aln.STRATA_BEST1, aln.STRATA_FULL])
def test_heavy_phase_parity(cuda, li, strata):
    """The heavy phase (reads handed to a search by every lane of the GPU) gives
    the oracle's results: with heavy_after = 1 almost every read of the batch is
    handed over (2048 per call; the rest stay with their warps), across gap,
    seed and z settings and both strata."""
    lim = LIMITS[li]
    rng = Rng(3000 + li, "heavy")
    text = reference_iid(30_000, rng.sub("t"))
    pair = Pair(text, kmers=[0, 6])
    m = [20, 36, 50, 36, 60, 76, 40][li]
    reads = simulate_reads(text, 2500, m, rng.sub("r"), sub_rate=(0.02, 0.04), indel_rate=0.005,
                           indel_lens=(1, 2), n_frac=0.1, z=lim["z"])
    ro, ho, _ = oracle_align(pair.ox, reads, lim, 40, strata)
    for k in (0, 6):
        p = aln.Params.from_limits(lim, hit_cap=40, strata=strata, mode=aln.MODE_PERSISTENT, heavy_after=1)
        rg, hg = pair.als[k].align(reads.codes, reads.offsets, reads.lens, p)
        compare(rg, hg, ro, ho, what=f"heavy limits {li} kmer {k}")


def _positions_parity(pair, rg, hg, what):
    """sa_to_pos of every written hit against the oracle's full suffix arrays."""
    cap = hg.shape[1]
    hits = hg[np.arange(cap)[None, :] < rg["n_hits"][:, None]]
    pos, npos = pair.al.positions(hits, 16)
    ohits = np.zeros(hits.size, oracle.HIT_DTYPE)
    for f in ("k", "l", "aligned_len", "strand"):
        ohits[f] = hits[f]
    opos, onpos = pair.ox.positions(ohits, 16)
    wide = (hits["l"].astype(np.int64) - hits["k"] + 1) > 16
    assert (npos[wide] == aln.POS_TOO_WIDE).all(), what
    assert np.array_equal(npos[~wide], onpos[~wide]), what
    for i in np.nonzero(~wide)[0]:
        assert np.array_equal(pos[i, :npos[i]], opos[i, :npos[i]]), f"{what}: hit {i}"
    return int((~wide).sum())


def test_pairs_recipe_parity(cuda):
    """The paired-end recipe (2 x 100 bp, fragment ~ Normal(500, 50), mates on
    opposite strands, 0.1 % chimeric pairs, repeats and N runs) at 3 Mbp: both
    mates of every pair in one batch, every read bit-exact in the plain and the
    persistent form, and the SA positions of every hit equal to the oracle's."""
    w = workload("human_pairs", ref_len=3_000_000, n_reads=3000, seed=4)
    assert w.reads.n == 6000 and (w.reads.true_strand[0::2] != w.reads.true_strand[1::2]).mean() > 0.99
    pair = Pair(w.text, kmers=[0, BENCH_KMER])
    ro, ho, _ = oracle_align(pair.ox, w.reads, w.params, 32, oracle.BEST1)
    for mode, k in [(aln.MODE_PLAIN, 0), (aln.MODE_PERSISTENT, 0), (aln.MODE_PERSISTENT, BENCH_KMER)]:
        rg, hg = _run(pair, w.reads, w.params, mode=mode, kmer=k)
        compare(rg, hg, ro, ho, what=f"pairs mode {mode} kmer {k}")
    assert (rg["n_hits"] > 0).mean() > 0.95
    assert _positions_parity(pair, rg, hg, "pairs positions") > 5000


@pytest.mark.parametrize("li,score,max_best", [(1, (3, 11, 4), 0), (4, (3, 11, 4), 2), (6, (1, 2, 1), 0),
                                               (2, (2, 3, 1), 1)])
def test_score_mode_parity(cuda, li, score, max_best):
    """Score-ordered mode (hits ranked by mismatch / gap-open / gap-extension
    penalties, best and second-best score strata, cap on equally best places)
    against the oracle, in the persistent search and in the heavy phase, on
    texts with and without repeats."""
    lim = LIMITS[li]
    rng = Rng(4000 + li, "score")
    text = reference_iid(20_000, rng.sub("t"))
    text[5000:5400] = text[1000:1400]  # a repeat, so that best places tie
    text[9000:9400] = text[1000:1400]
    pair = Pair(text, kmers=[0, 7])
    m = [20, 36, 50, 36, 60, 76, 40][li]
    reads = simulate_reads(text, 1500, m, rng.sub("r"), sub_rate=(0.02, 0.04), indel_rate=0.005,
                           indel_lens=(1, 2), n_frac=0.05, z=lim["z"])
    ro, ho, _ = oracle_align(pair.ox, reads, lim, 40, oracle.SCORE, score=score, max_best=max_best)
    for k, heavy in ((0, 0), (7, 0), (7, 1)):
        p = aln.Params.from_limits(lim, hit_cap=40, strata=aln.STRATA_SCORE, mode=aln.MODE_PERSISTENT,
                                   score_mm=score[0], score_gapo=score[1], score_gape=score[2],
                                   max_best=max_best, heavy_after=heavy)
        rg, hg = pair.als[k].align(reads.codes, reads.offsets, reads.lens, p)
        compare(rg, hg, ro, ho, what=f"score limits {li} kmer {k} heavy_after {heavy}")
    if max_best:
        assert (rg["flags"] & aln.FLAG_MANY_BEST).any()
    with pytest.raises(aln.AlnError):  # the plain form has no score-ordered mode
        pair.al.align(reads.codes, reads.offsets, reads.lens,
                      aln.Params.from_limits(lim, strata=aln.STRATA_SCORE, mode=aln.MODE_PLAIN))


def test_pairing_parity(cuda):
    """The pairing stage on the GPU (compaction, SA walk, aln_pair_resolve) against
    the oracle's pairing of its own search results: every field of every pair and
    the insert-size window, on the paired-end recipe at 3 Mbp (N runs, repeats,
    chimeric pairs) with two placement caps."""
    w = workload("human_pairs", ref_len=3_000_000, n_reads=5000, seed=8)
    pair = Pair(w.text, kmers=[BENCH_KMER])
    al = pair.al
    cap = 32
    p = aln.Params.from_limits(w.params, hit_cap=cap, mode=aln.MODE_PERSISTENT)
    d = al.upload(w.reads.codes, w.reads.offsets, w.reads.lens)
    res, hits = al.outputs(d["n"], cap)
    al.search_device(d, p, res, hits)
    ro, ho, _ = oracle_align(pair.ox, w.reads, w.params, cap, oracle.BEST1)
    rg = res.cpu().numpy().view(aln.RES_DTYPE)[:d["n"]]
    hg = hits.cpu().numpy().view(aln.HIT_DTYPE)[:d["n"] * cap].reshape(d["n"], cap)
    compare(rg, hg, ro, ho, what="pairing input")
    for max_place in (16, 4):
        gp, gst = al.pair(res, d["n"], cap, hits, 16, max_place)
        op, ost = pair.ox.pair_resolve(ro, ho, max_place)
        assert gst == ost, (gst, ost)
        for f in ("pos", "insert", "n_proper", "strand", "flags"):
            bad = np.nonzero((gp[f] != op[f]).reshape(gp.size, -1).any(axis=1))[0]
            assert bad.size == 0, f"max_place {max_place}: {f} differs at pair {bad[0]}: {gp[bad[0]]} vs {op[bad[0]]}"
        assert ((gp["flags"] & aln.PAIR_PROPER) != 0).mean() > 0.9
    assert gst["n_unique"] > 3000 and abs(gst["q2"] - 500) <= 10


def test_chr100_scaled_parity(cuda):
    """The 100 bp Markov + repeat-family recipe at 4 Mbp, every read."""
    w = workload("chr100", ref_len=4_000_000, n_reads=4000, seed=1)
    pair = Pair(w.text, kmers=[0, 12])
    ro, ho, _ = oracle_align(pair.ox, w.reads, w.params, 32, oracle.BEST1)
    for mode, k in [(aln.MODE_PLAIN, 0), (aln.MODE_PERSISTENT, 0), (aln.MODE_PERSISTENT, 12)]:
        rg, hg = _run(pair, w.reads, w.params, mode=mode, kmer=k)
        compare(rg, hg, ro, ho, what=f"chr100-4M mode {mode} kmer {k}")


def test_edge_cases(cuda):
    text = reference_iid(5000, Rng(7, "edge"))
    pair = Pair(text, kmers=[0, 8])
    parts = [np.zeros(0, np.uint8), text[10:11], np.full(12, 4, np.uint8), np.zeros(256, np.uint8),
             text[100:355], text[4000:4036], text[4964:5000], text[0:36]]
    lens = np.array([p.size for p in parts], np.uint16)
    offs = np.zeros(lens.size, np.uint64)
    offs[1:] = np.cumsum(lens[:-1].astype(np.uint64))
    z = np.array([2, 0, 2, 2, 6, 7, 2, 2], np.uint8)
    reads = Reads(np.concatenate(parts), offs, lens, z, np.zeros(lens.size, np.int64),
                  np.zeros(lens.size, np.uint8))
    lim = dict(z=7, max_gapo=1, max_gape=2, seed_len=0, seed_z=0, indel_end_skip=5)
    for cap, mode, k in [(1, aln.MODE_PLAIN, 0), (4, aln.MODE_PLAIN, 0), (1, aln.MODE_PERSISTENT, 8),
                         (4, aln.MODE_PERSISTENT, 8), (4, aln.MODE_PERSISTENT, 0)]:
        rg, hg = _run(pair, reads, lim, hit_cap=cap, z=z, zmax=6, mode=mode, kmer=k)
        ro, ho, _ = oracle_align(pair.ox, reads, lim, cap, oracle.BEST1, z=z)
        # z=7 > params.z=6 is flagged by the GPU (declared bound), not by the oracle
        assert rg[5]["flags"] & aln.FLAG_BAD_LIMIT and rg[5]["n_hits"] == 0
        keep = np.array([i for i in range(lens.size) if i != 5])
        compare(rg[keep], hg[keep], ro[keep], ho[keep], idx=keep, what=f"edge cap {cap} mode {mode} k {k}")
        assert rg[3]["flags"] & aln.FLAG_READ_TOO_LONG
        assert rg[0]["n_hits"] == 0 and rg[0]["d_best"] == 255


def test_unaligned_offsets_and_order(cuda, tiny36):
    """Reads shuffled and duplicated (36 bp reads packed back to back start at
    base offsets that are not word aligned): each read's result is unchanged."""
    w, pair = tiny36
    sub = w.reads.subset(np.arange(500))
    rng = np.random.default_rng(3)
    perm = np.concatenate([rng.permutation(500), rng.integers(0, 500, 100)])
    shuffled = sub.subset(perm)
    p = aln.Params.from_limits(w.params, hit_cap=32)
    r1, h1 = pair.al.align(sub.codes, sub.offsets, sub.lens, p)
    r2, h2 = pair.al.align(shuffled.codes, shuffled.offsets, shuffled.lens, p)
    assert np.array_equal(r2, r1[perm])
    valid = np.arange(32)[None, :] < r2["n_hits"][:, None]
    for f in ("k", "l", "aligned_len", "strand", "n_diff", "n_mm", "n_gapo", "n_gape"):
        assert np.array_equal(np.where(valid, h2[f], 0), np.where(valid, h1[perm][f], 0))


def test_sa_to_pos_parity(cuda, tiny36):
    w, pair = tiny36
    rg, hg = _run(pair, w.reads.subset(np.arange(3000)), w.params, strata=aln.STRATA_FULL)
    hits = np.concatenate([hg[i, :rg[i]["n_hits"]] for i in range(rg.size)])
    pos, npos = pair.al.positions(hits, 16)
    ohits = np.zeros(hits.size, oracle.HIT_DTYPE)
    for f in ("k", "l", "aligned_len", "strand"):
        ohits[f] = hits[f]
    opos, onpos = pair.ox.positions(ohits, 16)
    width = hits["l"].astype(np.int64) - hits["k"] + 1
    wide = width > 16
    assert (npos[wide] == aln.POS_TOO_WIDE).all()
    assert np.array_equal(npos[~wide], onpos[~wide])
    for i in np.nonzero(~wide)[0]:
        assert np.array_equal(pos[i, :npos[i]], opos[i, :npos[i]])
    # every position is where the target starts: the forward read's true origin
    # is among the positions of its best forward hit for error-free reads
    assert (~wide).sum() > 2000


def test_chr100_full_size_sampled(cuda):
    """Full size (100 Mbp text, 1 M x 100 bp reads, z=4, seed 32/2) in the launch
    configurations the benchmark times: every read searched on the GPU, a seeded
    sample of 3000 reads (plus every read with more than one hit) recomputed by
    the oracle one by one and compared bit-exact; plain == persistent on all."""
    w = workload("chr100")
    pair = Pair(w.text, kmers=[0, BENCH_KMER])
    p = aln.Params.from_limits(w.params, hit_cap=32)
    rp, hp = pair.als[0].align(w.reads.codes, w.reads.offsets, w.reads.lens, p)
    p.mode = aln.MODE_PERSISTENT
    rq, hq = pair.als[BENCH_KMER].align(w.reads.codes, w.reads.offsets, w.reads.lens, p)
    assert np.array_equal(rp, rq)
    valid = np.arange(32)[None, :] < rp["n_hits"][:, None]
    for f in ("k", "l", "aligned_len", "strand", "n_diff", "n_mm", "n_gapo", "n_gape"):
        assert np.array_equal(np.where(valid, hp[f], 0), np.where(valid, hq[f], 0))
    rng = np.random.default_rng(2024)
    sample = np.unique(np.concatenate([rng.choice(w.reads.n, 3000, replace=False),
                                       np.nonzero(rp["n_hits"] > 1)[0][:2000]]))
    sub = w.reads.subset(sample)
    ro, ho, _ = oracle_align(pair.ox, sub, w.params, 32, oracle.BEST1)
    compare(rp[sample], hp[sample], ro, ho, idx=sample, what="chr100 full")


def test_autotune_and_graph_replay(cuda, tiny36):
    """The autotuner picks a feasible blocks-per-SM value whose results equal the
    default's; a search captured in a CUDA graph and replayed twice (with the
    input buffers refilled in between) gives the direct results."""
    w, pair = tiny36
    al = pair.al
    torch = cuda
    p = aln.Params.from_limits(w.params, hit_cap=16, mode=aln.MODE_PERSISTENT)
    d = al.upload(w.reads.codes, w.reads.offsets, w.reads.lens)
    res, hits = al.outputs(d["n"], 16)
    tuned, ms = al.autotune(d, p, res, hits)
    assert 1 <= tuned.blocks_per_sm <= 16 and ms > 0 and tuned.smem_stack in aln.SMEM_STACK_CHOICES
    assert (tuned.help_after, tuned.heavy_after) == (p.help_after, p.heavy_after)  # not tuned
    again, ms2 = al.autotune(d, p, res, hits)  # cached per index, sample and limits
    assert (again.blocks_per_sm, again.smem_stack, ms2) == (tuned.blocks_per_sm, tuned.smem_stack, ms)
    ref = al.align(w.reads.codes, w.reads.offsets, w.reads.lens, p)
    got = al.align(w.reads.codes, w.reads.offsets, w.reads.lens, tuned)
    assert np.array_equal(ref[0], got[0])
    ro, ho, _ = oracle_align(pair.ox, w.reads, w.params, 16, oracle.BEST1)
    compare(got[0], got[1], ro, ho, what="autotuned")
    g = al.capture(d, p, res, hits)
    assert g.aln_scratch.numel() == aln.scratch_bytes(d["n"])
    for _ in range(2):
        res.fill_(0)
        hits.fill_(0)
        d2 = al.upload(w.reads.codes, w.reads.offsets, w.reads.lens)
        for key in ("bases", "nmask", "offsets", "lens"):
            d[key].copy_(d2[key])
        g.replay()
        torch.cuda.synchronize()
        r = res.cpu().numpy().view(aln.RES_DTYPE)[:d["n"]]
        h = hits.cpu().numpy().view(aln.HIT_DTYPE)[:d["n"] * 16].reshape(d["n"], 16)
        compare(r, h, ro, ho, what="graph replay")
        assert al.last_status() == 0
