"""Host logic of the benchmark (no GPU): the launch count it claims per search,
the roofline's choice of denominator and its traffic figure, and the range
partition of reads over replicas."""
import numpy as np
import pytest

import bench
import paper_1505_07855_gb300 as aln


def test_search_launches():
    never = 0xFFFFFFFF
    plain = aln.Params(mode=aln.MODE_PLAIN)
    assert bench.search_launches(aln, plain) == 1
    assert bench.search_launches(aln, aln.Params(mode=aln.MODE_PERSISTENT)) == 4 + 1 + 2 * aln.HEAVY_PASSES
    assert bench.search_launches(aln, aln.Params(mode=aln.MODE_PERSISTENT, heavy_after=never)) == 4
    # without scratch (a captured search that brought none): the search kernel alone
    assert bench.search_launches(aln, aln.Params(mode=aln.MODE_PERSISTENT), scratch=False) == 1


PROBES = {"l2": {"gbs": 16000.0, "buffer_bytes": 64 << 20}, "hbm": {"gbs": 2600.0, "buffer_bytes": 4 << 30}}


def test_roofline_bound_follows_the_index_size():
    small = bench.roofline(1000.0, 1_000_000, 50.0, PROBES, 89_000_000, "chr100")
    big = bench.roofline(1000.0, 1_000_000, 50.0, PROBES, 2_089_000_000, "human_pairs")
    assert small["bound"] == "l2" and small["peak"] == 16000.0
    assert big["bound"] == "hbm" and big["peak"] == 2600.0
    achieved = 1000.0 * bench.BYTES_PER_LOOKUP * 1_000_000 / 0.050 / 1e9
    for r in (small, big):
        assert r["achieved"] == pytest.approx(achieved)
        assert r["frac"] == pytest.approx(achieved / r["peak"])
        assert r["unit"] == "GB/s"


def test_roofline_traffic_only_for_the_captured_sources(monkeypatch):
    cap = {"src_sha256_16": bench._src_hash(), "dram_bytes_per_read": 1000}
    monkeypatch.setitem(bench.TRAFFIC_CAPTURE, "chr100", cap)
    r = bench.roofline(10.0, 5000, 1.0, PROBES, 1, "chr100")
    assert r["traffic"] == 1000 * 5000
    monkeypatch.setitem(bench.TRAFFIC_CAPTURE, "chr100", dict(cap, src_sha256_16="0" * 16))
    assert bench.roofline(10.0, 5000, 1.0, PROBES, 1, "chr100")["traffic"] is None
    assert bench.roofline(10.0, 5000, 1.0, PROBES, 1, "tiny36")["traffic"] is None


@pytest.mark.parametrize("n,ws", [(0, 1), (1, 2), (7, 3), (1_000_000, 8), (1001, 4)])
def test_partition_range_covers_the_batch_once(n, ws):
    ranges = [bench.partition_range(n, r, ws) for r in range(ws)]
    assert ranges[0][0] == 0 and ranges[-1][1] == n
    assert all(ranges[i][1] == ranges[i + 1][0] for i in range(ws - 1))
    sizes = np.array([hi - lo for lo, hi in ranges])
    assert sizes.min() >= 0 and sizes.max() - sizes.min() <= 1


def test_gpus_n_relaunches_under_torchrun_and_rank0_alone_prints():
    """`bench.py --gpus 2` starts itself again under torch.distributed.run with two
    ranks; in the reference arm rank 0 alone runs the oracle and prints the one
    JSON line (the other rank exits 0 without work)."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = {k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK", "MASTER_ADDR",
                                                            "MASTER_PORT")}
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--gpus", "2",
                          "--workload", "tiny36", "--steps", "1", "--warmup", "0", "--ref-sample", "200"],
                         cwd=root, env=env, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out.stdout
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["config"]["workload"] == "tiny36"
