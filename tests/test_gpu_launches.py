"""The kernels one search call launches, counted by the CUDA profiler, equal the
count bench.py reports as gpu_launches (search_launches): the plain form one;
the persistent form the D pre-pass, the two visit-order kernels and the search,
and unless the heavy phase is off its start kernel and one pass and one decide
kernel per deepening pass."""
import pytest

import paper_1505_07855_gb300 as aln
from synth import workload

pytestmark = pytest.mark.gpu


def _kernels(torch, fn):
    from torch.profiler import ProfilerActivity, profile
    torch.cuda.synchronize()
    with profile(activities=[ProfilerActivity.CUDA]) as prof:
        fn()
        torch.cuda.synchronize()
    names = [ev.name for ev in prof.events() if ev.device_type == torch.autograd.DeviceType.CUDA]
    return [n for n in names if "aln_" in n]


def test_launch_count_matches_the_bench(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import bench
    w = workload("tiny36", ref_len=100_000, n_reads=3000, seed=21)
    al = aln.Aligner(aln.Index.build(w.text).to_device(0))
    d = al.upload(w.reads.codes, w.reads.offsets, w.reads.lens)
    res, hits = al.outputs(d["n"], 8)
    cases = [(aln.MODE_PLAIN, 0), (aln.MODE_PERSISTENT, 0), (aln.MODE_PERSISTENT, 0xFFFFFFFF),
             (aln.MODE_PERSISTENT, 1)]
    p0 = aln.Params.from_limits(w.params, hit_cap=8, mode=aln.MODE_PLAIN)
    for _ in range(3):  # the profiler's first sessions in a process can miss kernels
        if _kernels(torch, lambda: al.search_device(d, p0, res, hits)):
            break
    for mode, heavy in cases:
        p = aln.Params.from_limits(w.params, hit_cap=8, mode=mode, heavy_after=heavy)
        al.search_device(d, p, res, hits)  # warm-up (pool, lazy module load)
        got = _kernels(torch, lambda: al.search_device(d, p, res, hits))
        assert len(got) == bench.search_launches(aln, p), (mode, heavy, got)
        if mode == aln.MODE_PERSISTENT and heavy != 0xFFFFFFFF:
            assert sum("aln_heavy_pass_kernel" in n for n in got) == aln.HEAVY_PASSES
