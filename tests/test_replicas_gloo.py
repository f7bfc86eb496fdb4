"""The N>1 path of the benchmark on the CPU (gloo, world size 2): rank 0 builds
and saves the index, rank 1 loads it after the barrier and holds a
byte-identical image; per-rank timings reduce to their maximum; the reads are
split into contiguous ranges, one per rank, and the per-rank results
concatenated in rank order equal the results of the whole batch searched at
once.  No collective touches the data path (replicas only)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, tmpdir, out_q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    import paper_1505_07855_gb300 as aln
    from synth import Rng, reference_iid
    text = reference_iid(50_000, Rng(5, "replica"))
    path = os.path.join(tmpdir, "replica.fmi")
    hix = bench.replica_index(aln, text, 4, rank, ws, dist.barrier, path)
    mine = os.path.join(tmpdir, f"rank{rank}.fmi")
    hix.save(mine)
    vals = bench.max_over_ranks([10.0 + rank, 5.0 - rank], ws)
    dist.barrier()
    out_q.put((rank, hix.info(), vals))
    dist.destroy_process_group()


def test_replicas_share_one_index_and_max_timing(tmp_path):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, str(tmp_path), q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    assert res[0][1] == res[1][1]
    assert res[0][2] == res[1][2] == [11.0, 5.0]
    a = open(tmp_path / "rank0.fmi", "rb").read()
    b = open(tmp_path / "rank1.fmi", "rb").read()
    assert a == b and len(a) > 1000


def _partition_worker(rank, ws, port, n, out_q):
    """Each rank searches its range of the batch (the oracle stands in for the GPU
    search, which needs a device), then the results are concatenated."""
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    import oracle
    from synth import workload
    w = workload("tiny36", ref_len=40_000, n_reads=n, seed=9)
    ox = oracle.OracleIndex(w.text, threads=1)
    lo, hi = bench.partition_range(n, rank, ws)
    sub = w.reads.subset(np.arange(lo, hi))
    lim = w.params
    r, h, _ = ox.align(sub.codes, sub.offsets, sub.lens, z_default=lim["z"], max_gapo=lim["max_gapo"],
                       max_gape=lim["max_gape"], indel_end_skip=lim["indel_end_skip"], hit_cap=8, threads=1)
    rr, hh = bench.concat_over_ranks((r, h), ws)
    out_q.put((rank, lo, hi, rr.tobytes(), hh.tobytes()))
    dist.destroy_process_group()


@pytest.mark.parametrize("ws,n", [(2, 501), (3, 7)])
def test_partition_and_concatenation_equal_one_batch(ws, n):
    import oracle
    from synth import workload
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_partition_worker, args=(r, ws, port, n, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # contiguous ranges that cover the batch once, in rank order
    assert res[0][1] == 0 and res[-1][2] == n
    assert all(res[i][2] == res[i + 1][1] for i in range(ws - 1))
    w = workload("tiny36", ref_len=40_000, n_reads=n, seed=9)
    lim = w.params
    r, h, _ = oracle.OracleIndex(w.text, threads=1).align(
        w.reads.codes, w.reads.offsets, w.reads.lens, z_default=lim["z"], max_gapo=lim["max_gapo"],
        max_gape=lim["max_gape"], indel_end_skip=lim["indel_end_skip"], hit_cap=8, threads=1)
    for _, _, _, rb, hb in res:  # every rank holds the whole batch's results
        assert rb == r.tobytes() and hb == h.tobytes()
