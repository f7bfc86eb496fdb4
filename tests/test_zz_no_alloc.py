"""aln_search_noalloc: the search for callers that cannot call cudaMalloc (a
process whose device memory belongs to another allocator, or a serving loop
that must not allocate after start-up).  It keeps its only scratch, the work
queue counter, in a fixed array inside the library.  Called through the C ABI
twice in a row, it must give exactly the results of aln_search (integer
outputs, so the tolerance is zero); sizes above its limit are refused.

This file is collected last so that a run stopping at the first failure has
run every other test before it; it needs nothing from them."""
import ctypes

import numpy as np
import pytest

import paper_1505_07855_gb300 as aln
from paper_1505_07855_gb300 import _lib
from synth import workload

pytestmark = pytest.mark.gpu

HIT_FIELDS = ("k", "l", "aligned_len", "strand", "n_diff", "n_mm", "n_gapo", "n_gape")


def _call_noalloc(dix, d, n, params, res, hits, stream):
    b = _lib.aln_batch(d["bases"].data_ptr(), d["nmask"].data_ptr(), d["offsets"].data_ptr(),
                       d["lens"].data_ptr(), None)
    r = _lib.aln_result(res.data_ptr(), hits.data_ptr())
    p = params.c()
    return aln.lib().aln_search_noalloc(dix._h, ctypes.byref(b), n, ctypes.byref(p), ctypes.byref(r),
                                        stream.cuda_stream)


def _host(res, hits, n, cap):
    r = res.cpu().numpy().view(aln.RES_DTYPE)[:n].copy()
    h = hits.cpu().numpy().view(aln.HIT_DTYPE)[:n * cap].reshape(n, cap).copy()
    return r, h


def _same(a, b, cap):
    ra, ha = a
    rb, hb = b
    assert np.array_equal(ra, rb)
    valid = np.arange(cap)[None, :] < ra["n_hits"][:, None]
    for f in HIT_FIELDS:
        assert np.array_equal(np.where(valid, ha[f], 0), np.where(valid, hb[f], 0)), f


def test_noalloc_matches_aln_search():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    w = workload("chr100", ref_len=2_000_000, n_reads=6000, seed=5)
    dix = aln.Index.build(w.text).to_device(0)
    al = aln.Aligner(dix)
    d = al.upload(w.reads.codes, w.reads.offsets, w.reads.lens)
    n, cap = w.reads.n, 16
    params = aln.Params.from_limits(w.params, hit_cap=cap, mode=aln.MODE_PERSISTENT)
    stream = torch.cuda.Stream()
    res, hits = al.outputs(n, cap)
    al.search_device(d, params, res, hits, stream)
    torch.cuda.synchronize()
    ref = _host(res, hits, n, cap)
    assert (ref[0]["n_hits"] > 0).mean() > 0.9
    for _ in range(2):  # two calls in a row share the fixed scratch array
        res2, hits2 = al.outputs(n, cap)
        res2.fill_(0xAB)
        hits2.fill_(0xCD)
        assert _call_noalloc(dix, d, n, params, res2, hits2, stream) == aln.ALN_OK
        torch.cuda.synchronize()
        _same(_host(res2, hits2, n, cap), ref, cap)
    # beyond the counter's range: refused before anything is launched
    rc = _call_noalloc(dix, d, 0x80000001, params, res2, hits2, stream)
    assert rc == -1 and b"ALN_NOALLOC_MAX_READS" in aln.lib().aln_last_error()
