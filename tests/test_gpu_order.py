"""The persistent search visits reads in an order computed on the GPU (by the
lower bound D(0) from its D pre-pass); a read's result must not depend on that
order or on its neighbours.  Searching a permuted batch must give, read for
read, the results of the original batch (integer outputs: exact), on a mix of
lengths, per-read limits and N bases, and those results must equal the plain
form's (one thread per read, no pre-pass)."""
import numpy as np
import pytest

import paper_1505_07855_gb300 as aln
from synth import workload

pytestmark = pytest.mark.gpu

HIT_FIELDS = ("k", "l", "aligned_len", "strand", "n_diff", "n_mm", "n_gapo", "n_gape")


def _same(a, b, cap):
    ra, ha = a
    rb, hb = b
    assert np.array_equal(ra, rb)
    valid = np.arange(cap)[None, :] < ra["n_hits"][:, None]
    for f in HIT_FIELDS:
        assert np.array_equal(np.where(valid, ha[f], 0), np.where(valid, hb[f], 0)), f


def test_results_do_not_depend_on_read_order():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    w = workload("human_mixed", ref_len=3_000_000, n_reads=8000, seed=9)
    al = aln.Aligner(aln.Index.build(w.text, kmer_k=8).to_device(0))
    cap = 16
    p = aln.Params.from_limits(w.params, hit_cap=cap, mode=aln.MODE_PERSISTENT, z=6)
    base = al.align(w.reads.codes, w.reads.offsets, w.reads.lens, p, z=w.reads.z)
    assert len(np.unique(base[0]["d_best"])) > 2  # several lower bounds in the batch
    perm = np.random.default_rng(4).permutation(w.reads.n)
    sub = w.reads.subset(perm)
    got = al.align(sub.codes, sub.offsets, sub.lens, p, z=sub.z)
    _same((base[0][perm], base[1][perm]), got, cap)
    p.mode = aln.MODE_PLAIN
    _same(base, al.align(w.reads.codes, w.reads.offsets, w.reads.lens, p, z=w.reads.z), cap)
