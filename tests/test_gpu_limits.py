"""Bounds that the C ABI promises, exercised on the GPU without a fault: the
persistent loop's trip bound (params.loop_limit) stops the search with a status
bit and flags, never a hang; sa_to_pos refuses records that are not hits of the
index before it reads anything of the index; the work-queue counters of
captured searches are reserved, so two graphs replay side by side."""
import numpy as np
import pytest

import oracle
import paper_1505_07855_gb300 as aln
from parity_util import HIT_FIELDS, compare, oracle_align
from synth import workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    w = workload("tiny36", ref_len=300_000, n_reads=3000, seed=21)
    ox = oracle.OracleIndex(w.text)
    al = aln.Aligner(aln.Index.build(w.text, kmer_k=8).to_device(0))
    ro, ho, _ = oracle_align(ox, w.reads, w.params, 16, oracle.BEST1)
    return torch, w, ox, al, ro, ho


def test_loop_limit_stops_with_status_and_flags(setup):
    """A tiny trip bound: the status word carries ALN_STATUS_LOOP_LIMIT, every
    read has a written result, the unfinished ones are flagged
    ALN_FLAG_LOOP_LIMIT with no hits, and the finished ones equal the oracle."""
    torch, w, ox, al, ro, ho = setup
    n = w.reads.n
    d = al.upload(w.reads.codes, w.reads.offsets, w.reads.lens)
    res, hits = al.outputs(n, 16)
    for limit in (1, 40):
        res.fill_(0xFF)  # flags 0xFF cannot be written by the search
        p = aln.Params.from_limits(w.params, hit_cap=16, mode=aln.MODE_PERSISTENT, loop_limit=limit)
        al.search_device(d, p, res, hits)
        torch.cuda.synchronize()
        assert al.last_status() & aln.STATUS_LOOP_LIMIT
        with pytest.raises(aln.AlnError) as e:
            al.check_status()
        assert e.value.status == aln.ALN_ELIMIT
        r = res.cpu().numpy().view(aln.RES_DTYPE)[:n]
        h = hits.cpu().numpy().view(aln.HIT_DTYPE)[:n * 16].reshape(n, 16)
        assert (r["flags"] != 0xFF).all(), "a read was left without a result"
        cut = (r["flags"] & aln.FLAG_LOOP_LIMIT) != 0
        assert cut.any()
        assert (r["n_hits"][cut] == 0).all() and (r["d_best"][cut] == 255).all()
        done = np.nonzero(~cut)[0]
        if done.size:
            compare(r[done], h[done], ro[done], ho[done], idx=done, what=f"finished under limit {limit}")
    # the default bound is never reached, and the status word is cleared per call
    p = aln.Params.from_limits(w.params, hit_cap=16, mode=aln.MODE_PERSISTENT)
    r, h = al.align(w.reads.codes, w.reads.offsets, w.reads.lens, p)
    assert al.last_status() == 0
    compare(r, h, ro, ho, what="default bound")


def test_sa_to_pos_rejects_records_that_are_not_hits(setup):
    """Rows past the text, an inverted interval and a strand above 1 get
    ALN_POS_BAD_HIT; the real hits around them keep their positions."""
    torch, w, ox, al, ro, ho = setup
    n = w.text.size
    first = ho[ro["n_hits"] > 0][:, 0][:50]
    good = np.zeros(first.size, aln.HIT_DTYPE)
    for f in ("k", "l", "aligned_len", "strand", "n_diff", "n_mm", "n_gapo", "n_gape"):
        good[f] = first[f]
    bad = np.zeros(5, aln.HIT_DTYPE)
    bad["k"] = [n + 1, 0xFFFFFFF0, 5, 3, 0xFFFFFFFF]
    bad["l"] = [n + 1, 0xFFFFFFFF, 4, 3, 0xFFFFFFFF]
    bad["strand"] = [0, 1, 0, 2, 1]
    bad["aligned_len"] = 36
    hits = np.concatenate([good[:25], bad, good[25:]])
    hits_o = np.zeros(hits.size, oracle.HIT_DTYPE)
    for f in ("k", "l", "aligned_len", "strand"):
        hits_o[f] = hits[f]
    pos, npos = al.positions(hits, 16)
    isbad = np.zeros(hits.size, bool)
    isbad[25:30] = True
    assert (npos[isbad] == aln.POS_BAD_HIT).all()
    opos, onpos = ox.positions(hits_o[~isbad], 16)
    gp, gn = pos[~isbad], npos[~isbad]
    wide = (hits[~isbad]["l"].astype(np.int64) - hits[~isbad]["k"] + 1) > 16
    assert (gn[wide] == aln.POS_TOO_WIDE).all()
    assert np.array_equal(gn[~wide], onpos[~wide])
    for i in np.nonzero(~wide)[0]:
        assert np.array_equal(gp[i, :gn[i]], opos[i, :gn[i]])


def test_two_captured_searches_replay_side_by_side(setup):
    """Each captured search owns its queue counter: two graphs over two halves
    of the batch, replayed on two streams at once, both equal the oracle."""
    torch, w, ox, al, ro, ho = setup
    p = aln.Params.from_limits(w.params, hit_cap=16, mode=aln.MODE_PERSISTENT)
    halves = [np.arange(0, 1500), np.arange(1500, 3000)]
    graphs, outs = [], []
    for idx in halves:
        sub = w.reads.subset(idx)
        d = al.upload(sub.codes, sub.offsets, sub.lens)
        res, hits = al.outputs(d["n"], 16)
        graphs.append((al.capture(d, p, res, hits), d))
        outs.append((res, hits))
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    torch.cuda.synchronize()
    for (g, _), st in zip(graphs, streams):
        with torch.cuda.stream(st):
            g.replay()
    torch.cuda.synchronize()
    for idx, (res, hits) in zip(halves, outs):
        m = idx.size
        r = res.cpu().numpy().view(aln.RES_DTYPE)[:m]
        h = hits.cpu().numpy().view(aln.HIT_DTYPE)[:m * 16].reshape(m, 16)
        compare(r, h, ro[idx], ho[idx], idx=idx, what="side-by-side replay")
    assert HIT_FIELDS


def test_compact_hits_equals_host_compaction(setup):
    """aln_compact_hits: per-read offsets and the written hits back to back, equal
    to compacting the per-read slots on the host; with a dense array too small
    the total is still reported and only the hits that fit are written."""
    torch, w, ox, al, ro, ho = setup
    n, cap = w.reads.n, 16
    p = aln.Params.from_limits(w.params, hit_cap=cap, mode=aln.MODE_PERSISTENT)
    d = al.upload(w.reads.codes, w.reads.offsets, w.reads.lens)
    res, hits = al.outputs(n, cap)
    al.search_device(d, p, res, hits)
    r = res.cpu().numpy().view(aln.RES_DTYPE)[:n]
    h = hits.cpu().numpy().view(aln.HIT_DTYPE)[:n * cap].reshape(n, cap)
    exp = h[np.arange(cap)[None, :] < r["n_hits"][:, None]]
    exp_off = np.concatenate([[0], np.cumsum(r["n_hits"].astype(np.int64))])
    scratch = al.compact_scratch(n)
    for room in (exp.size + 7, exp.size // 2):
        offsets = torch.zeros(n + 1, dtype=torch.int32, device=al.dev)
        dense = torch.full((max(1, room) * aln.HIT_DTYPE.itemsize,), 0xEE, dtype=torch.uint8, device=al.dev)
        al.compact(res, hits, n, cap, offsets, dense, scratch)
        torch.cuda.synchronize()
        off = offsets.cpu().numpy().view(np.uint32)
        dd = dense.cpu().numpy().view(aln.HIT_DTYPE)
        assert np.array_equal(off.astype(np.int64), exp_off)
        k = min(room, exp.size)
        assert dd[:k].tobytes() == exp[:k].tobytes()
        if room > exp.size:
            assert (dense.cpu().numpy()[exp.size * 16:] == 0xEE).all()
