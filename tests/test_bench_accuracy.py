"""The bench's placement report (best stratum against the simulated origin),
driven by the oracle's hits and positions on a small workload: error-bounded
reads of a repeat-free i.i.d. text place at their origin, and a truth shifted
beyond the tolerance places none.  Both bench arms describe the same workload."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import bench  # noqa: E402
import oracle  # noqa: E402
from synth import workload  # noqa: E402


def _report(w, cap=32):
    lim = w.params
    ox = oracle.OracleIndex(w.text, threads=4)
    r, h, _ = ox.align(w.reads.codes, w.reads.offsets, w.reads.lens, w.reads.z, z_default=lim["z"],
                       max_gapo=lim["max_gapo"], max_gape=lim["max_gape"], seed_len=lim["seed_len"],
                       seed_z=lim["seed_z"], indel_end_skip=lim["indel_end_skip"], hit_cap=cap, threads=4)
    h = h.reshape(-1, cap)
    valid = np.arange(cap)[None, :] < r["n_hits"][:, None]
    opos, onpos = ox.positions(h[valid], 16)
    pos = torch.from_numpy(np.ascontiguousarray(opos.astype(np.uint64)).view(np.int64).reshape(-1))
    npos = torch.from_numpy(np.ascontiguousarray(onpos.astype(np.uint32)).view(np.int32))
    return bench.accuracy_report(w, (r, h), pos, npos, cap, valid)


def test_reads_place_at_origin():
    w = workload("tiny36", ref_len=200_000, n_reads=800, seed=11)
    rep = _report(w)
    assert rep["mapped"] > 0.9
    assert rep["best_covers_origin"] > 0.9 * rep["mapped"]
    assert rep["unique_best_correct"] > 0.95


def test_shifted_truth_places_none():
    w = workload("tiny36", ref_len=200_000, n_reads=400, seed=12)
    w.reads.true_pos = w.reads.true_pos + 1000
    assert _report(w)["best_covers_origin"] == 0.0


def test_both_bench_arms_name_the_same_workload():
    w = workload("chr100", ref_len=300_000, n_reads=50, seed=1)
    gpu = bench.workload_config("chr100", w, w.reads.n, 1)
    ref = bench.workload_config("chr100", w, 20, 1, mode="oracle (CPU)")
    same = ("workload", "ref_bp", "read_len", "z", "seed", "strata", "parallelism")
    assert {k: gpu[k] for k in same} == {k: ref[k] for k in same}
    assert gpu["read_len"] == 100 and gpu["z"] == 4 and gpu["seed"] == [32, 2]
