"""The N>1 path of the benchmark on the CPU (gloo, world size 2): rank 0 builds
and saves the index, rank 1 loads it after the barrier and holds a
byte-identical image; per-rank timings reduce to their maximum.  No collective
touches the data path (replicas only)."""
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
