"""Serving loop (continuous batching): results through the server equal a direct
aln_search bit-exact, each request's result is the same alone and in a mix of
concurrent requests (split across batches and overlapping on the device), and
latency statistics are reported."""
import threading

import numpy as np
import pytest

import paper_1505_07855_gb300 as aln
from synth import Rng, simulate_reads, workload, z_for_length

pytestmark = pytest.mark.gpu

FIELDS = ("k", "l", "aligned_len", "strand", "n_diff", "n_mm", "n_gapo", "n_gape")


@pytest.fixture(scope="module")
def setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    w = workload("human_mixed", ref_len=4_000_000, n_reads=1, seed=9)
    dix = aln.Index.build(w.text, kmer_k=10).to_device(0)
    return w, dix


def _requests(w, n_req, seed):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_req):
        n = int(np.exp(rng.uniform(0, np.log(3000))))  # log-uniform sizes
        r = simulate_reads(w.text, n, (50, 76, 100, 150, 250), Rng(seed * 1000 + i, "req"),
                           sub_rate=(0.01, 0.01), indel_rate=0.0005, n_frac=0.02, z_of_len=z_for_length,
                           nmask=w.nmask)
        out.append(r)
    return out


def _same(a, b, cap):
    ra, ha = a
    rb, hb = b
    assert np.array_equal(ra, rb)
    valid = np.arange(cap)[None, :] < ra["n_hits"][:, None]
    for f in FIELDS:
        assert np.array_equal(np.where(valid, ha[f], 0), np.where(valid, hb[f], 0)), f


@pytest.mark.parametrize("heavy_after", [0, 1])
def test_server_matches_direct_and_alone_equals_mixed(setup, heavy_after):
    """heavy_after 0: the server runs no heavy phase; 1: every batch's tail reads
    go to the heavy phase, while other slots' batches are in flight."""
    w, dix = setup
    params = aln.Params.from_limits(w.params, hit_cap=8, mode=aln.MODE_PERSISTENT, z=6, heavy_after=heavy_after)
    reqs = _requests(w, 24, 3)
    al = aln.Aligner(dix)
    direct = [al.align(r.codes, r.offsets, r.lens, params, z=r.z) for r in reqs]
    # small batches so that requests are split and several batches are in flight
    srv = aln.Server(dix, params, n_slots=3, max_batch_reads=1500, coalesce_us=100)
    try:
        alone = []
        for r in reqs:  # one at a time
            rid = srv.submit(r.codes, r.offsets, r.lens, r.z)
            res, hits, lat = srv.poll(rid, r.n)
            alone.append((res, hits))
            assert lat >= 0
        ids = [None] * len(reqs)

        def submit_all(idx):
            for i in idx:
                ids[i] = srv.submit(reqs[i].codes, reqs[i].offsets, reqs[i].lens, reqs[i].z)
        th = [threading.Thread(target=submit_all, args=(list(range(k, len(reqs), 3)),)) for k in range(3)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        mixed = [srv.poll(ids[i], reqs[i].n)[:2] for i in range(len(reqs))]
        st = srv.stats()
    finally:
        srv.close()
    for d, a, m in zip(direct, alone, mixed):
        _same(d, a, 8)
        _same(d, m, 8)
    assert st["requests_done"] == 2 * len(reqs)
    assert st["reads_done"] == 2 * sum(r.n for r in reqs)
    assert st["batches"] > len(reqs)  # large requests were split
    assert 0 <= st["p50_ms"] <= st["p95_ms"] <= st["p99_ms"]


def test_server_empty_and_poll_timeout(setup):
    w, dix = setup
    params = aln.Params.from_limits(w.params, hit_cap=4, z=6)
    srv = aln.Server(dix, params, n_slots=1, max_batch_reads=1000)
    try:
        rid = srv.submit(np.zeros(0, np.uint8), np.zeros(0, np.uint64), np.zeros(0, np.uint16))
        res, hits, lat = srv.poll(rid, 0)
        assert res.size == 0
        with pytest.raises(aln.AlnError):
            srv.poll(rid, 0)  # forgotten after the first successful poll
    finally:
        srv.close()
