#!/usr/bin/env python
"""Benchmark of the GB300 BWA-aln inexact FM-index search.

Workload (default): 100 Mbp order-3 Markov reference (41 % GC, 5 % copies of 50
repeat families), 1 M single-end 100 bp reads (substitutions 0.5 % -> 2 %,
0.02 % indels of 1-3 bp), z=4, seed 32 with <= 2 seed differences, gap opens
<= 1, gap extensions <= 6, no indel within 5 bp of an end; BEST1 strata.

A step is one aln_search over the whole 1 M-read batch (both strands, D scans,
backtracking search, hit reduction).  The headline is the persistent (batched)
form; the plain one-launch-per-batch form is timed beside it.  L2 is flushed
(a 512 MiB write) before every timed step.  Then (unless `--human 0`) the
3.1 Gbp text: its index built on the GPU, a 1 M-read paired batch and a 1 M-read
mixed-length batch (autotuned, replayed from a CUDA graph), each persistent
against plain and checked against the oracle on a seeded 1 % plus every flagged
read, and serving on the resident text.  `--impl reference` times the CPU
oracle on bounded samples of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "reads/s bit-exact vs oracle (batched vs plain, 1 GB300); % HBM roofline; p99 ms"
BYTES_PER_LOOKUP = 64
# DRAM bytes (read + write) of aln_persistent_kernel per read from one ncu capture
# of each workload (a few hundred thousand reads, scaled per read; the profile
# summaries under profiles/ give the command).  Used only while the kernel
# sources hash to the value they had at capture time.
KERNEL_SOURCES = ("aln_device.cuh", "aln_search.cuh", "aln_flat.cuh", "aln_kernels.cu")
TRAFFIC_CAPTURE = {  # workload -> capture; the profile summaries give the commands
    # 300 000 of the 1 M reads: 6.778 GB read + 0.254 GB written in one launch
    "chr100": {"src_sha256_16": "b5a44875db83a4ce", "dram_bytes_per_read": 23441},
    # the first 200 000 reads of the 1 M-read paired batch: 143.55 GB + 1.06 GB
    "human_pairs": {"src_sha256_16": "b5a44875db83a4ce", "dram_bytes_per_read": 723067},
}
L2_BYTES = 126 << 20  # GB300 L2 (cudaDevAttrL2CacheSize reports 126 MiB)


HEAVY_BEGIN = b"// ---------------------------------------------------------------- heavy phase\n"
HEAVY_END = b"// ---------------------------------------------------------------- end of the heavy phase\n"


def _src_hash() -> str:
    """Hash of the sources the search kernel is compiled from: the heavy phase's
    own kernels (a separate launch, between its two section lines in
    aln_kernels.cu) are left out, since the captured traffic is the search
    kernel's alone."""
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(f.encode())
        with open(os.path.join(ROOT, "paper_1505_07855_gb300", "csrc", f), "rb") as fh:
            src = fh.read()
        a, b = src.find(HEAVY_BEGIN), src.find(HEAVY_END)
        if a >= 0 and b > a:
            src = src[:a] + src[b + len(HEAVY_END):]
        h.update(src)
    return h.hexdigest()[:16]


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """Samples nvidia-smi clocks and throttle reasons while running."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def replica_index(aln, text, kmer_k, rank, ws, barrier, path, device=None):
    """Replicas: rank 0 builds the index (on its GPU when device is given) and
    saves it, the other ranks load the image after the barrier (no collective
    touches the data path)."""
    if ws > 1:
        if rank == 0:
            aln.Index.build(text, kmer_k=kmer_k, device=device).save(path)
        barrier()
        return aln.Index.load(path)
    return aln.Index.build(text, kmer_k=kmer_k, device=device)


def partition_range(n, rank, ws):
    """Reads [lo, hi) of rank `rank` out of ws replicas: contiguous ranges of
    near-equal size in read order (every GPU holds the whole index)."""
    return n * rank // ws, n * (rank + 1) // ws


def concat_over_ranks(parts, ws):
    """Per-rank result arrays (a tuple of numpy arrays over the rank's reads),
    concatenated in rank order on every rank: the results of the whole batch in
    read order.  No collective touches the timed search; this runs after it."""
    if ws <= 1:
        return parts
    import torch.distributed as dist
    objs = [None] * ws
    dist.all_gather_object(objs, parts)
    return tuple(np.concatenate([o[i] for o in objs]) for i in range(len(parts)))


def max_over_ranks(values, ws, device=None):
    """Element-wise maximum of per-rank timings (the whole job is as slow as its
    slowest replica)."""
    if ws <= 1:
        return list(values)
    import torch
    import torch.distributed as dist
    t = torch.tensor(values, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t]


def oracle_sample(w, n_sample, threads, seed=7):
    """Oracle index of the text and its results on a seeded sample of reads."""
    import oracle
    t0 = time.time()
    ox = oracle.OracleIndex(w.text, threads=threads)
    t_index = time.time() - t0
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(w.reads.n, min(n_sample, w.reads.n), replace=False))
    sub = w.reads.subset(idx)
    lim = w.params
    t0 = time.time()
    ro, ho, look = ox.align(sub.codes, sub.offsets, sub.lens, sub.z, z_default=lim["z"],
                            max_gapo=lim["max_gapo"], max_gape=lim["max_gape"],
                            seed_len=lim["seed_len"], seed_z=lim["seed_z"],
                            indel_end_skip=lim["indel_end_skip"], hit_cap=32, threads=threads)
    t_align = time.time() - t0
    return ox, idx, ro, ho, look, t_index, t_align


def serving_phase(aln, dix, w, lam, seconds, seed=5, text_note="the 100 Mbp bench text stands in for the 3.1 Gbp one",
                  slots=3, batch_reads=1 << 19):
    """Poisson request stream on the resident index: request sizes log-uniform on
    [1, 100000] reads, lengths uniform over 50..250 bp, z = min(6, ceil(0.04 len)),
    errors as the tiny36 recipe; reads are cut from a pre-simulated pool."""
    import threading
    from synth import Rng, simulate_reads, z_for_length
    pool_n = 400_000
    pool = simulate_reads(w.text, pool_n, np.arange(50, 251), Rng(seed, "serve-pool"), sub_rate=(0.01, 0.01),
                          indel_rate=0.0005, indel_lens=(1,), n_frac=0.02, z_of_len=z_for_length,
                          nmask=w.nmask)
    rng = np.random.default_rng(seed)
    params = aln.Params(z=6, max_gapo=w.params["max_gapo"], max_gape=w.params["max_gape"],
                        seed_len=0, seed_z=0, indel_end_skip=5, hit_cap=8, mode=aln.MODE_PERSISTENT)
    srv = aln.Server(dix, params, n_slots=slots, max_batch_reads=batch_reads, coalesce_us=500)
    done, lock = [], threading.Lock()
    pending = []
    stop = threading.Event()
    offered = [0]

    def poller():
        while not stop.is_set() or pending:
            with lock:
                items = list(pending)
            for it in items:
                r = srv.poll(it[0], it[1], wait_ms=1)
                if r is not None:
                    with lock:
                        pending.remove(it)
                        done.append(r[2])
            if not items:
                stop.wait(0.001)

    th = threading.Thread(target=poller, daemon=True)
    th.start()
    t0 = time.time()
    t_next = t0
    while True:
        t_next += rng.exponential(1.0 / lam)
        if t_next - t0 > seconds:
            break
        delay = t_next - time.time()
        if delay > 0:
            time.sleep(delay)
        n = int(np.exp(rng.uniform(0, np.log(100_000))))
        a = int(rng.integers(0, pool_n - n))
        lens = pool.lens[a:a + n]
        offs = pool.offsets[a:a + n] - pool.offsets[a]
        codes = pool.codes[int(pool.offsets[a]):int(pool.offsets[a + n - 1]) + int(lens[-1])]
        rid = srv.submit(codes, offs, lens, pool.z[a:a + n])
        offered[0] += n
        with lock:
            pending.append((rid, n))
    stop.set()
    th.join(timeout=300)
    elapsed = time.time() - t0
    st = srv.stats()
    srv.close()
    lat = np.array(done)
    return {"lambda_req_per_s": lam, "seconds": seconds, "requests": int(lat.size),
            "reads_per_s": st["reads_done"] / elapsed, "offered_reads_per_s": offered[0] / seconds,
            "p50_ms": float(np.percentile(lat, 50)) if lat.size else None,
            "p95_ms": float(np.percentile(lat, 95)) if lat.size else None,
            "p99_ms": float(np.percentile(lat, 99)) if lat.size else None,
            "batches": st["batches"], "slots": st["n_slots"], "max_batch_reads": batch_reads, "text": text_note}


def _levenshtein(a, b):
    """Edit distance with an N (4) in the read matching nothing."""
    prev = np.arange(b.size + 1)
    for i in range(1, a.size + 1):
        cur = np.empty_like(prev)
        cur[0] = i
        sub = prev[:-1] + ((b != a[i - 1]) | (a[i - 1] == 4))
        cur[1:] = np.minimum(sub, prev[1:] + 1)
        for j in range(1, b.size + 1):  # insertion chain along the row
            if cur[j - 1] + 1 < cur[j]:
                cur[j] = cur[j - 1] + 1
        prev = cur
    return int(prev[-1])


def property_checks(w, outp, pos, npos, hit_cap, n_hits, valid, n_sample=400, seed=3):
    """Checks that hold at any size (used where the oracle's index is too large
    to build): every sampled hit's target, at each reported position, lies
    within the hit's difference count of the read (edit distance, the text's N
    replaced as the index replaced it), and the simulated origin of each
    sampled read is among its hits' positions (recall)."""
    from synth import mix64, revcomp_codes
    rg, hg = outp
    rng = np.random.default_rng(seed)
    sel = np.sort(rng.choice(rg.size, min(n_sample, rg.size), replace=False))
    pos_h = pos.cpu().numpy().view(np.uint64)[:n_hits * 16].reshape(-1, 16)
    np_h = npos.cpu().numpy().view(np.uint32)[:n_hits]
    row_of = np.full(valid.size, -1, np.int64)
    iv = np.nonzero(valid.reshape(-1))[0]
    row_of[iv] = np.arange(iv.size)
    text = w.text
    sound = checked = found = eligible = 0
    for r in sel:
        read = w.reads.read(int(r))
        hit_pos = set()
        for j in range(int(rg[r]["n_hits"])):
            h = hg[r, j]
            row = row_of[r * hit_cap + j]
            if np_h[row] > 16:
                continue
            q = read if h["strand"] == 0 else revcomp_codes(read)
            for p in pos_h[row, :np_h[row]]:
                p = int(p)
                hit_pos.add((p, int(h["strand"])))
                T = text[p:p + int(h["aligned_len"])].copy()
                nm = T == 4
                if nm.any():
                    T[nm] = (mix64(np.uint64(0) ^ (np.nonzero(nm)[0] + p).astype(np.uint64)) & np.uint64(3)).astype(np.uint8)
                checked += 1
                sound += _levenshtein(q, T) <= int(h["n_diff"])
        eligible += 1
        found += (int(w.reads.true_pos[r]), int(w.reads.true_strand[r])) in hit_pos
    return {"kind": "properties (oracle index not built at this size)", "sampled_reads": int(sel.size),
            "hits_checked": checked, "hits_sound": sound, "all_sound": sound == checked,
            "origin_recall": found / max(1, eligible)}


def gather_probe_phase(aln, torch, dev, stream, buf_bytes=4 << 30, n_gathers=1 << 27, best_of=10, warmup=3):
    """Random 64-byte block-read rate over a buffer (best of best_of launches,
    CUDA events on the launching stream).  4 GiB: far larger than L2, the HBM
    random-block rate; 64 MiB: held by L2, the L2 random-sector rate."""
    buf = torch.empty(buf_bytes, dtype=torch.uint8, device=dev)
    sink = torch.zeros(1, dtype=torch.int32, device=dev)
    ms = []
    with torch.cuda.stream(stream):
        buf.fill_(0x5A)
        for it in range(warmup + best_of):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            aln.gather_probe(buf, n_gathers, it, sink, stream)
            e1.record(stream)
            e1.synchronize()
            if it >= warmup:
                ms.append(e0.elapsed_time(e1))
    del buf
    best = min(ms)
    return {"gbs": n_gathers * 64 / (best / 1000) / 1e9, "unit": "GB/s", "buffer_bytes": buf_bytes,
            "gathers_per_launch": n_gathers, "bytes_per_gather": 64, "best_of": best_of, "ms": best}


def accuracy_report(w, outp, pos, npos, hit_cap, valid):
    """Placement against the simulated origin: a read counts as placed correctly
    when a hit of its best stratum (n_diff == d_best) on the read's true strand
    has a position within z bases of the true start.  Hits wider than 16 rows
    have no positions; reads whose best stratum is all such hits are
    'unresolved' (repeats)."""
    rg, hg = outp
    n = rg.size
    rows = np.nonzero(valid)[0]
    hv = hg[valid]
    nh = hv.size
    widths = npos.cpu().numpy().view(np.uint32)[:nh].astype(np.int64)
    p = pos.cpu().numpy().view(np.uint64)[:nh * 16].reshape(-1, 16).astype(np.int64) if nh else np.zeros((0, 16), np.int64)
    tp = w.reads.true_pos.astype(np.int64)
    ts = w.reads.true_strand.astype(np.int64)
    z = w.reads.z.astype(np.int64) if np.any(w.reads.z) else np.full(n, int(w.params["z"]), np.int64)
    best = hv["n_diff"].astype(np.int64) == rg["d_best"][rows].astype(np.int64)
    resolved = widths <= 16
    near = (np.arange(16)[None, :] < np.where(resolved, widths, 0)[:, None]) & \
           (np.abs(p - tp[rows][:, None]) <= z[rows][:, None])
    hit_ok = best & (hv["strand"].astype(np.int64) == ts[rows]) & near.any(axis=1)
    ok = np.bincount(rows, weights=hit_ok, minlength=n) > 0
    best_resolved = np.bincount(rows, weights=best & resolved, minlength=n) > 0
    mapped = rg["n_hits"] > 0
    unique = mapped & (rg["c0"] == 1)
    out = {"reads": int(n), "mapped": float(mapped.mean()), "best_covers_origin": float(ok.mean()),
           "unresolved_repeats": float((mapped & ~best_resolved).mean()),
           "unique_best": float(unique.mean()),
           "unique_best_correct": float(ok[unique].mean()) if unique.any() else None,
           "tolerance": "z bases"}
    lens = w.reads.lens.astype(np.int64)
    if np.unique(lens).size > 1:
        out["best_covers_origin_by_len"] = {int(m): float(ok[lens == m].mean()) for m in np.unique(lens)}
    return out


def roofline(lookups_per_read, n, ms, probes, index_bytes, workload_name):
    """Achieved algorithmic bytes/s of the search (64 B per Occ lookup of the
    oracle's canonical count, the D scans included) against the random 64-byte
    gather rate of the memory that serves the index: L2 when the searched index
    (Occ blocks + prefix-trie tables of both texts) fits in L2, else HBM; the
    fraction of the streaming copy peak is reported beside it."""
    copy_peak, src = _peaks()
    bytes_per_read = lookups_per_read * BYTES_PER_LOOKUP
    achieved = bytes_per_read * n / (ms / 1000) / 1e9
    in_l2 = index_bytes <= L2_BYTES
    bound = "l2" if in_l2 else "hbm"
    probe = probes.get(bound)
    peak = probe["gbs"] if probe else copy_peak
    traffic = None
    cap = TRAFFIC_CAPTURE.get(workload_name)
    if cap and _src_hash() == cap["src_sha256_16"]:
        traffic = cap["dram_bytes_per_read"] * n
    return {"bound": bound, "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic,
            "peak_source": (f"aln_gather_probe, random 64-byte reads over a {probe['buffer_bytes'] >> 20} MiB "
                            f"buffer ({'L2-resident' if in_l2 else 'HBM'}), measured in this run") if probe
                           else f"streaming copy peak ({src})",
            "index_bytes": int(index_bytes), "copy_peak": copy_peak, "copy_peak_source": src,
            "frac_of_copy_peak": achieved / copy_peak, "bytes_per_read": bytes_per_read,
            "occ_lookups_per_s": lookups_per_read * n / (ms / 1000)}


def workload_config(name, w, n_per_step, ws, mode="persistent"):
    """The JSON line's config: the workload by name and sizes, the limits."""
    lim = w.params
    mixed = name == "human_mixed"
    return {"workload": name, "ref_bp": int(w.text.size), "reads_per_step": int(n_per_step),
            "read_len": "36-250 mixed" if mixed else int(w.reads.lens[0]) if w.reads.n else 0,
            "z": "min(6, ceil(0.04 len))" if mixed else lim["z"], "seed": [lim["seed_len"], lim["seed_z"]],
            "strata": "BEST1", "mode": mode,
            "l2": "flushed (512 MiB write) before every step" if mode == "persistent" else "n/a (CPU)",
            "parallelism": f"replicas{ws}" if ws > 1 else "single"}


def search_launches(aln, params, scratch=True):
    """Kernels one search launches (the same list whether launched directly or
    replayed from a graph): the plain form one; the persistent form the search,
    with scratch the D pre-pass and the two visit-order kernels before it, and
    unless the heavy phase is off its start kernel and one pass and one decide
    kernel per deepening pass after it."""
    if params.mode == aln.MODE_PLAIN:
        return 1
    n = 1
    if scratch:
        n += 3
        if params.heavy_after != 0xFFFFFFFF:
            n += 1 + 2 * aln.HEAVY_PASSES
    return n


def time_search(al, d, params, res, hits, stream, flush, steps, warmup, torch, graph=None):
    """Mean device time (ms, CUDA events on the launching stream) of `steps`
    searches after `warmup` untimed ones, L2 flushed before each."""
    ms = []
    with torch.cuda.stream(stream):
        for it in range(warmup + steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            if graph is not None:
                graph.replay()
            else:
                al.search_device(d, params, res, hits, stream)
            e1.record(stream)
            e1.synchronize()
            if it >= warmup:
                ms.append(e0.elapsed_time(e1))
    al.check_status()
    return float(np.mean(ms)), ms


def _host_results(aln, res, hits, n, cap):
    return (res.cpu().numpy().view(aln.RES_DTYPE)[:n].copy(),
            hits.cpu().numpy().view(aln.HIT_DTYPE)[:n * cap].reshape(n, cap).copy())


def _flag_counts(aln, r):
    fl = r["flags"]
    return {"incomplete": int(((fl & aln.FLAG_INCOMPLETE) != 0).sum()),
            "work_limit": int(((fl & aln.FLAG_WORK_LIMIT) != 0).sum()),
            "cand_overflow": int(((fl & aln.FLAG_CAND_OVERFLOW) != 0).sum()),
            "hit_overflow": int(((fl & aln.FLAG_HIT_OVERFLOW) != 0).sum()),
            "no_hit": int((r["n_hits"] == 0).sum())}


HIT_FIELDS = ("k", "l", "aligned_len", "strand", "n_diff", "n_mm", "n_gapo", "n_gape")


def compare_fields(rg, hg, ro, ho, rows):
    """Every result field and every written hit field of GPU vs oracle; returns
    (equal, description of the first difference or None)."""
    for f in ("c0", "c1", "n_hits", "d_best", "flags"):
        bad = np.nonzero(rg[f] != ro[f])[0]
        if bad.size:
            i = bad[0]
            return False, f"read {int(rows[i])}: {f} gpu {int(rg[f][i])} oracle {int(ro[f][i])}"
    cap = hg.shape[1]
    valid = np.arange(cap)[None, :] < rg["n_hits"][:, None]
    for f in HIT_FIELDS:
        bad = np.argwhere(np.where(valid, hg[f], 0) != np.where(valid, ho[f], 0))
        if bad.size:
            i, j = bad[0]
            return False, f"read {int(rows[i])} hit {int(j)}: {f} gpu {int(hg[f][i, j])} oracle {int(ho[f][i, j])}"
    return True, None


def oracle_check(ox, w, rg, hg, sel, hit_cap, threads):
    """The oracle on the reads `sel` (every field of every read, bit-exact) and the
    canonical Occ-lookup count per read."""
    import oracle
    sub = w.reads.subset(sel)
    lim = w.params
    per_read_z = bool(np.any(sub.z != sub.z[0])) if sub.n else False
    t0 = time.time()
    ro, ho, look = ox.align(sub.codes, sub.offsets, sub.lens, sub.z if per_read_z else None, z_default=lim["z"],
                            max_gapo=lim["max_gapo"], max_gape=lim["max_gape"], seed_len=lim["seed_len"],
                            seed_z=lim["seed_z"], indel_end_skip=lim["indel_end_skip"], hit_cap=hit_cap,
                            strata=oracle.BEST1, threads=threads)
    dt = time.time() - t0
    ok, first_diff = compare_fields(rg[sel], hg[sel], ro, ho, sel)
    return {"kind": "oracle", "reads": int(sel.size), "bit_exact": bool(ok), "first_difference": first_diff,
            "oracle_s": dt, "oracle_threads": threads}, look


def human_phase(args, aln, torch, dev, stream, flush):
    """The 3.1 Gbp human-scale text (45 % repeats, 1 % N runs): the paired-end
    batch (2 x 100 bp, z=4) and the mixed-length batch (36-250 bp, z by length,
    autotuned, replayed through a captured CUDA graph), persistent vs plain; the
    oracle index is built on the host cores while the GPU runs, then checks a
    seeded 1 % of each batch plus every read with a flag, bit-exact; SA positions
    of the paired batch; placement vs the simulated origins; serving at
    lambda = 50 requests/s on the resident index."""
    import threading
    import oracle
    from synth.workloads import human_workloads
    out = {}
    n_reads = args.human_reads
    t0 = time.time()
    mixed, pairs = human_workloads(args.human_ref or None, n_mixed=n_reads, n_pairs=n_reads // 2)
    out["gen_s"] = time.time() - t0
    out["ref_bp"] = int(mixed.text.size)
    threads = max(1, oracle.default_threads() - 1)  # one core stays with the thread that drives the GPU
    box = {}

    def build_oracle():
        t = time.time()
        try:
            box["ox"] = oracle.OracleIndex(mixed.text, threads=threads)
        except MemoryError as e:
            box["err"] = str(e)
        box["s"] = time.time() - t

    th = threading.Thread(target=build_oracle, daemon=True)
    if not args.no_oracle:
        th.start()
    torch.cuda.empty_cache()
    t0 = time.time()
    hix = aln.Index.build(mixed.text, kmer_k=args.kmer_k, device=dev.index, stream=stream)
    out["index_build"] = {"where": "gpu (fm_index_build_gpu)", "s": time.time() - t0}
    dix = hix.to_device(dev.index)
    info = dix.info()
    index_bytes = 2 * (info["occ_bytes"] + info["kmer_bytes"])
    del hix
    al = aln.Aligner(dix)
    hit_cap = 32
    blocks = {}
    for w, name in ((pairs, "pairs"), (mixed, "mixed")):
        n = w.reads.n
        per_read_z = name == "mixed"
        d = al.upload(w.reads.codes, w.reads.offsets, w.reads.lens, w.reads.z if per_read_z else None)
        res, hits = al.outputs(n, hit_cap)
        zkw = {"z": 6} if per_read_z else {}
        pp = aln.Params.from_limits(w.params, hit_cap=hit_cap, mode=aln.MODE_PERSISTENT, l2_window=args.l2_window,
                                    **zkw)
        pl = aln.Params.from_limits(w.params, hit_cap=hit_cap, mode=aln.MODE_PLAIN, **zkw)
        b = {"reads_per_step": n, "steps": args.human_steps, "warmup": args.human_warmup}
        graph = None
        if per_read_z:  # the mixed batch: autotuned schedule, graph replay
            ns = min(n, 100_000)
            dsub = dict(d)
            dsub["n"] = ns
            t = time.time()
            pp, tuned_ms = al.autotune(dsub, pp, res, hits, stream)
            b["autotune"] = {"blocks_per_sm": pp.blocks_per_sm, "smem_stack": pp.smem_stack,
                             "sample_reads": ns, "sample_ms": tuned_ms,
                             "s": time.time() - t}
            with torch.cuda.stream(stream):
                graph = al.capture(d, pp, res, hits)
            b["graph_replay"] = True
        ms_p, _ = time_search(al, d, pp, res, hits, stream, flush, args.human_steps, args.human_warmup, torch, graph)
        rq, hq = _host_results(aln, res, hits, n, hit_cap)
        ms_l, _ = time_search(al, d, pl, res, hits, stream, flush, args.human_steps, args.human_warmup, torch)
        rp, hp = _host_results(aln, res, hits, n, hit_cap)
        inc = ((rp["flags"] | rq["flags"]) & aln.FLAG_INCOMPLETE) != 0
        vm = np.arange(hit_cap)[None, :] < rq["n_hits"][:, None]
        same = bool(np.array_equal(rp[~inc], rq[~inc]) and all(
            np.array_equal(np.where(vm, hp[f], 0)[~inc], np.where(vm, hq[f], 0)[~inc])
            for f in ("k", "l", "aligned_len", "strand", "n_diff", "n_mm", "n_gapo", "n_gape")))
        b["persistent"] = {"value": n / (ms_p / 1000), "ms_per_step": ms_p}
        b["plain"] = {"value": n / (ms_l / 1000), "ms_per_step": ms_l,
                      "bit_identical_to_persistent_on_complete_reads": same}
        b["persistent_over_plain"] = ms_l / ms_p
        b["flags"] = _flag_counts(aln, rq)
        b["gpu_launches_per_step"] = {"persistent": search_launches(aln, pp), "plain": search_launches(aln, pl)}
        b["_out"] = (w, rq, hq, ms_p)
        blocks[name] = b
        del d, res, hits, graph
        torch.cuda.empty_cache()
    # SA positions of every hit of the paired batch
    w, rq, hq, _ = blocks["pairs"]["_out"]
    valid = np.arange(hit_cap)[None, :] < rq["n_hits"][:, None]
    hits_all = hq[valid]
    dh = torch.from_numpy(hits_all.view(np.uint8).copy()).to(dev)
    pos = torch.empty(max(1, hits_all.size * 16), dtype=torch.int64, device=dev)
    npos = torch.empty(max(1, hits_all.size), dtype=torch.int32, device=dev)
    sa_ms = []
    with torch.cuda.stream(stream):
        for it in range(args.human_warmup + args.human_steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            dix.sa_to_pos(dh, hits_all.size, 16, pos, npos, stream)
            e1.record(stream)
            e1.synchronize()
            if it >= args.human_warmup:
                sa_ms.append(e0.elapsed_time(e1))
    np_h = npos.cpu().numpy().view(np.uint32)[:hits_all.size]
    pos_h = pos.cpu().numpy().view(np.uint64)[:hits_all.size * 16].reshape(-1, 16)
    n_pos = int(np_h[np_h <= 16].sum())
    blocks["pairs"]["sa_to_pos"] = {"hits": int(hits_all.size), "positions": n_pos, "ms": float(np.mean(sa_ms)),
                                    "positions_per_s": n_pos / (np.mean(sa_ms) / 1000)}
    blocks["pairs"]["accuracy"] = accuracy_report(w, (rq, hq), pos, npos, hit_cap, valid)
    # serving on the resident index while the oracle index may still be building
    if args.human_serve_seconds > 0:
        out["serving"] = serving_phase(aln, dix, mixed, args.human_serve_lambda, args.human_serve_seconds,
                                       text_note="the 3.1 Gbp text, resident", slots=args.serve_slots,
                                       batch_reads=args.serve_batch_reads)
    # oracle parity: a seeded 1 % of each batch plus every read with a flag
    if not args.no_oracle:
        th.join()
        out["oracle_index_s"] = box.get("s")
        ox = box.get("ox")
        if ox is None:
            out["oracle_error"] = box.get("err", "oracle index not built")
        for name, b in blocks.items():
            w, rq, hq, ms_p = b["_out"]
            if ox is None:
                continue
            rng = np.random.default_rng(17)
            n = w.reads.n
            flagged = np.nonzero(rq["flags"] != 0)[0]
            sel = np.unique(np.concatenate([rng.choice(n, max(1, n // 100), replace=False), flagged]))
            par, look = oracle_check(ox, w, rq, hq, sel, hit_cap, oracle.default_threads())
            par["sample"] = f"seeded 1 % of the {n}-read batch plus every flagged read ({flagged.size})"
            par["rows_above_2_31"] = int((hq[sel][np.arange(hit_cap)[None, :] < rq[sel]["n_hits"][:, None]]["l"]
                                          >= 2 ** 31).sum())
            b["parity"] = par
            b["roofline"] = roofline(float(look.mean()), n, ms_p, args._probes, index_bytes, "human_" + name)
            if name == "pairs":
                sh = hq[sel][np.arange(hit_cap)[None, :] < rq[sel]["n_hits"][:, None]]
                oh = np.zeros(sh.size, oracle.HIT_DTYPE)
                for f in ("k", "l", "aligned_len", "strand"):
                    oh[f] = sh[f]
                opos, onpos = ox.positions(oh, 16)
                gpos, gnpos = al.positions(sh, 16)
                wide = (sh["l"].astype(np.int64) - sh["k"] + 1) > 16
                okp = bool((gnpos[wide] == aln.POS_TOO_WIDE).all() and np.array_equal(gnpos[~wide], onpos[~wide])
                           and all(np.array_equal(gpos[i, :gnpos[i]], opos[i, :gnpos[i]])
                                   for i in np.nonzero(~wide)[0]))
                par["positions_bit_exact"] = okp
                par["positions_hits_checked"] = int(sh.size)
        del ox
        box.clear()
    for b in blocks.values():
        b.pop("_out", None)
    out.update(blocks)
    del al, dix
    torch.cuda.empty_cache()
    return out


def run_reference(args):
    """CPU oracle arm: each step aligns a bounded seeded sample on all host cores."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import oracle
    from synth import workload
    w = workload(args.workload)
    threads = oracle.default_threads()
    ox = oracle.OracleIndex(w.text, threads=threads)
    lim = w.params
    rng = np.random.default_rng(11)
    per_step = args.ref_sample

    def step(i):
        idx = np.sort(rng.choice(w.reads.n, per_step, replace=False))
        sub = w.reads.subset(idx)
        ox.align(sub.codes, sub.offsets, sub.lens, sub.z, z_default=lim["z"], max_gapo=lim["max_gapo"],
                 max_gape=lim["max_gape"], seed_len=lim["seed_len"], seed_z=lim["seed_z"],
                 indel_end_skip=lim["indel_end_skip"], hit_cap=32, threads=threads)
    for i in range(args.warmup):
        step(i)
    t0 = time.time()
    for i in range(args.steps):
        step(i)
    dt = time.time() - t0
    v = per_step * args.steps / dt
    sample = f"{per_step} seeded reads per step of the {w.reads.n}-read batch"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "reads/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * dt / args.steps,
        "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic", "config": workload_config(args.workload, w, per_step, 1, mode="oracle (CPU)"),
        "cpu_baseline": {"value": v, "unit": "reads/s", "cores": threads, "kind": "oracle", "sample": sample,
                         "where": "rank 0's host cores; no GPU is used"},
        "e2e": {"value": v, "unit": "reads/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_gpu(args):
    import torch
    import paper_1505_07855_gb300 as aln
    from synth import workload

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    t_all = time.time()
    big = args.workload in ("human_mixed", "human_pairs")
    n_req = args.reads or (1_000_000 if big else None)
    if args.workload == "human_pairs" and n_req:
        n_req //= 2  # pairs: two reads each, both mates in one batch
    t_gen = time.time()
    w = workload(args.workload, ref_len=args.ref_len or None, n_reads=n_req)
    t_gen = time.time() - t_gen
    if args.reads and w.reads.n > args.reads:
        w.reads = w.reads.subset(np.arange(args.reads))
    lim = w.params
    n = w.reads.n  # reads of the whole job
    per_read_z = args.workload == "human_mixed"
    # replicas: every GPU holds the whole index and searches its own range of reads
    lo, hi = partition_range(n, rank, ws)
    rl = w.reads.subset(np.arange(lo, hi)) if ws > 1 else w.reads
    n_local = rl.n
    build_dev = local if args.index_build == "gpu" else None
    # index: rank 0 builds and saves, the other replicas load the image
    t0 = time.time()
    if ws > 1:
        hix = replica_index(aln, w.text, args.kmer_k, rank, ws, torch.distributed.barrier,
                            f"/tmp/aln_bench_{args.workload}.fmi", device=build_dev)
    elif args.index_cache and os.path.exists(args.index_cache):
        hix = aln.Index.load(args.index_cache)
    else:
        hix = aln.Index.build(w.text, kmer_k=args.kmer_k, device=build_dev)
        if args.index_cache:
            hix.save(args.index_cache)
    t_build = time.time() - t0
    dix = hix.to_device(local)
    del hix
    al = aln.Aligner(dix)
    stream = torch.cuda.Stream(device=dev)
    bases, nmask, offs = aln.pack_reads(rl.codes, rl.offsets, rl.lens)
    lens = np.ascontiguousarray(rl.lens)
    d = {"bases": torch.from_numpy(bases.view(np.int32)).to(dev),
         "nmask": torch.from_numpy(nmask.view(np.int32)).to(dev),
         "offsets": torch.from_numpy(offs.view(np.int64)).to(dev),
         "lens": torch.from_numpy(lens.view(np.int16)).to(dev),
         "z": torch.from_numpy(np.ascontiguousarray(rl.z)).to(dev) if per_read_z else None, "n": n_local}
    hit_cap = 32
    res, hits = al.outputs(n_local, hit_cap)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    modes = {"persistent": aln.MODE_PERSISTENT, "plain": aln.MODE_PLAIN}
    params = {k: aln.Params.from_limits(lim, hit_cap=hit_cap, mode=m, blocks_per_sm=args.blocks_per_sm,
                                        work_limit=args.work_limit, l2_window=args.l2_window if k == "persistent" else 0,
                                        **({"z": 6} if per_read_z else {}))
              for k, m in modes.items()}

    tuned_ms = None
    if args.autotune:
        ns = min(n_local, 100_000)
        dsub = dict(d)
        dsub["n"] = ns
        params["persistent"], tuned_ms = al.autotune(dsub, params["persistent"], res, hits, stream)
    graph = None
    if args.graph:
        with torch.cuda.stream(stream):
            graph = al.capture(d, params["persistent"], res, hits)

    def step(mode):
        if graph is not None and mode == "persistent":
            graph.replay()
        else:
            al.search_device(d, params[mode], res, hits, stream)

    with torch.cuda.stream(stream):
        for mode in modes:
            for _ in range(args.warmup):
                flush.zero_()
                step(mode)
    torch.cuda.synchronize(dev)
    times = {}
    out = {}
    if ws > 1:
        torch.distributed.barrier()
    with Clocks(local) as clk:
        for mode in modes:
            evs = []
            torch.cuda.synchronize(dev)
            with torch.cuda.stream(stream):
                for _ in range(args.steps):
                    flush.zero_()
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    step(mode)
                    e1.record(stream)
                    evs.append((e0, e1))
            torch.cuda.synchronize(dev)
            ms = [a.elapsed_time(b) for a, b in evs]
            times[mode] = ms
            out[mode] = (res.cpu().numpy().view(aln.RES_DTYPE)[:n_local].copy(),
                         hits.cpu().numpy().view(aln.HIT_DTYPE)[:n_local * hit_cap].reshape(n_local, hit_cap).copy())
    clocks = clk.summary()
    al.check_status()
    ms_head = float(np.mean(times["persistent"]))
    ms_plain = float(np.mean(times["plain"]))
    ms_head, ms_plain = max_over_ranks([ms_head, ms_plain], ws, dev)
    for mode in modes:  # the whole batch's results, in read order, on every rank
        out[mode] = concat_over_ranks(out[mode], ws)
    rp, hp = out["plain"]
    rq, hq = out["persistent"]
    inc = ((rp["flags"] | rq["flags"]) & aln.FLAG_INCOMPLETE) != 0
    okr = ~inc
    vmask = np.arange(hit_cap)[None, :] < rq["n_hits"][:, None]
    same = bool(np.array_equal(rp[okr], rq[okr]) and all(
        np.array_equal(np.where(vmask, hp[f], 0)[okr], np.where(vmask, hq[f], 0)[okr])
        for f in ("k", "l", "aligned_len", "strand", "n_diff", "n_mm", "n_gapo", "n_gape")))
    fl = rq["flags"]
    flag_counts = {"incomplete": int(((fl & aln.FLAG_INCOMPLETE) != 0).sum()),
                   "work_limit": int(((fl & aln.FLAG_WORK_LIMIT) != 0).sum()),
                   "cand_overflow": int(((fl & aln.FLAG_CAND_OVERFLOW) != 0).sum()),
                   "stack_overflow": int(((fl & aln.FLAG_STACK_OVERFLOW) != 0).sum()),
                   "hit_overflow": int(((fl & aln.FLAG_HIT_OVERFLOW) != 0).sum()),
                   "no_hit": int((rq["n_hits"] == 0).sum())}

    # end to end through the public API with host buffers (pinned), copies timed:
    # inputs in, the search, aln_compact_hits, then the per-read results, the hit
    # offsets and exactly the hits written come back (the hit count is read first)
    h_bases = torch.from_numpy(bases.view(np.int32)).pin_memory()
    h_nmask = torch.from_numpy(nmask.view(np.int32)).pin_memory()
    h_offs = torch.from_numpy(offs.view(np.int64)).pin_memory()
    h_lens = torch.from_numpy(lens.view(np.int16)).pin_memory()
    h_res = torch.empty(res.numel(), dtype=torch.uint8).pin_memory()
    hit_off = torch.empty(n_local + 1, dtype=torch.int32, device=dev)
    dense = torch.empty(hits.numel(), dtype=torch.uint8, device=dev)
    cscratch = al.compact_scratch(n_local)
    h_off = torch.empty(n_local + 1, dtype=torch.int32).pin_memory()
    h_dense = torch.empty(hits.numel(), dtype=torch.uint8).pin_memory()
    h2d = sum(x.numel() * x.element_size() for x in (h_bases, h_nmask, h_offs, h_lens))
    e2e_ms, d2h_list = [], []
    with torch.cuda.stream(stream):
        for it in range(args.warmup + args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            d["bases"].copy_(h_bases, non_blocking=True)
            d["nmask"].copy_(h_nmask, non_blocking=True)
            d["offsets"].copy_(h_offs, non_blocking=True)
            d["lens"].copy_(h_lens, non_blocking=True)
            step("persistent")
            al.compact(res, hits, n_local, hit_cap, hit_off, dense, cscratch, stream)
            h_res.copy_(res, non_blocking=True)
            h_off.copy_(hit_off, non_blocking=True)
            stream.synchronize()
            total = int(h_off[n_local])
            nb = total * aln.HIT_DTYPE.itemsize
            h_dense[:nb].copy_(dense[:nb], non_blocking=True)
            e1.record(stream)
            e1.synchronize()
            if it >= args.warmup:
                e2e_ms.append(e0.elapsed_time(e1))
                d2h_list.append(h_res.numel() + h_off.numel() * 4 + nb)
    d2h = int(np.mean(d2h_list))
    # the compacted hits are the search's hits
    rq_l, hq_l = (res.cpu().numpy().view(aln.RES_DTYPE)[:n_local],
                  hits.cpu().numpy().view(aln.HIT_DTYPE)[:n_local * hit_cap].reshape(n_local, hit_cap))
    e2e_same = h_dense.numpy()[:total * 16].tobytes() == \
        hq_l[np.arange(hit_cap)[None, :] < rq_l["n_hits"][:, None]].tobytes()
    e2e_ms = max_over_ranks([float(np.mean(e2e_ms))], ws, dev)[0]
    e2e_v = n / (e2e_ms / 1000)

    line = {
        "metric": METRIC, "value": n / (ms_head / 1000), "unit": "reads/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_head, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": workload_config(args.workload, w, n, ws),
        "plain": {"value": n / (ms_plain / 1000), "ms_per_step": ms_plain,
                  "bit_identical_to_persistent_on_complete_reads": same},
        "flags": flag_counts,
        "schedule": {"blocks_per_sm": params["persistent"].blocks_per_sm or "max",
                     "smem_stack": params["persistent"].smem_stack or 8,
                     "help_after": params["persistent"].help_after or "once the read queue is empty",
                     "heavy_after": params["persistent"].heavy_after or aln.HEAVY_AFTER_DEFAULT,
                     "l2_window": args.l2_window,
                     "autotune_ms": tuned_ms, "graph_replay": bool(graph is not None),
                     "reads_per_rank": [partition_range(n, r, ws)[1] - partition_range(n, r, ws)[0]
                                        for r in range(ws)]},
        # timed regions: the persistent steps and the plain steps (search_launches)
        "gpu_launches": args.steps * (search_launches(aln, params["persistent"])
                                      + search_launches(aln, params["plain"])),
        "e2e": {"value": e2e_v, "unit": "reads/s", "h2d_bytes_per_step": int(h2d) * ws,
                "d2h_bytes_per_step": int(d2h) * ws, "hits_compacted": "aln_compact_hits",
                "compacted_hits_equal_search_hits": bool(e2e_same)},
        "clocks": clocks,
        "build_s": t_build, "gen_s": t_gen,
    }
    if rank != 0:  # the other replicas are done once their timings and results are in
        torch.distributed.destroy_process_group()
        return
    probes = {}
    if args.gather_probe:
        probes["hbm"] = gather_probe_phase(aln, torch, dev, stream)
        probes["l2"] = gather_probe_phase(aln, torch, dev, stream, buf_bytes=64 << 20)
        line["gather_probe"] = probes
    info = dix.info()
    index_bytes = 2 * (info["occ_bytes"] + info["kmer_bytes"])
    use_oracle = rank == 0 and not args.no_oracle and w.text.size <= args.oracle_max_bp
    if use_oracle:
        import oracle
        threads = oracle.default_threads()
        # size the sample to ~15 s of oracle search on all host cores
        ox, idx, ro, ho, look, t_index, t_align = oracle_sample(w, 300, threads)
        rate = len(idx) / max(t_align, 1e-6)
        target = int(min(max(1000, rate * args.cpu_seconds), 50_000))
        rng = np.random.default_rng(7)
        sel = np.sort(rng.choice(n, min(target, n), replace=False))
        sub = w.reads.subset(sel)
        t0 = time.time()
        ro, ho, look = ox.align(sub.codes, sub.offsets, sub.lens, sub.z, z_default=lim["z"],
                                max_gapo=lim["max_gapo"], max_gape=lim["max_gape"],
                                seed_len=lim["seed_len"], seed_z=lim["seed_z"],
                                indel_end_skip=lim["indel_end_skip"], hit_cap=hit_cap, threads=threads)
        t_align = time.time() - t0
        cpu_v = sel.size / t_align
        sel1 = sel[: min(1000, sel.size)]
        sub1 = w.reads.subset(sel1)
        t0 = time.time()
        ox.align(sub1.codes, sub1.offsets, sub1.lens, sub1.z, z_default=lim["z"], max_gapo=lim["max_gapo"],
                 max_gape=lim["max_gape"], seed_len=lim["seed_len"], seed_z=lim["seed_z"],
                 indel_end_skip=lim["indel_end_skip"], hit_cap=hit_cap, threads=1)
        cpu_v1 = sel1.size / (time.time() - t0)
        # parity of the timed outputs on the sample
        rg, hg = out["persistent"]
        rg, hg = rg[sel], hg[sel]
        ok = all(np.array_equal(rg[f], ro[f]) for f in ("c0", "c1", "n_hits", "d_best", "flags"))
        valid = np.arange(hit_cap)[None, :] < rg["n_hits"][:, None]
        for f in ("k", "l", "aligned_len", "strand", "n_diff", "n_mm", "n_gapo", "n_gape"):
            ok = ok and np.array_equal(np.where(valid, hg[f], 0), np.where(valid, ho[f], 0))
        line["roofline"] = roofline(float(look.mean()), n, ms_head, probes, index_bytes, args.workload)
        line["cpu_baseline"] = {"value": cpu_v, "unit": "reads/s", "cores": threads, "kind": "oracle",
                                "value_1thread": cpu_v1,
                                "sample": f"{sel.size} seeded reads of the {n}-read batch, "
                                          f"oracle index build ({t_index:.1f} s) not timed"}
        line["parity"] = {"sampled_reads": int(sel.size), "bit_exact": bool(ok)}
    # SA walk of every hit of the timed run (positions of hits of width <= 16)
    rg, hg = out["persistent"]
    valid = np.arange(hit_cap)[None, :] < rg["n_hits"][:, None]
    hits_all = hg[valid]
    dh = torch.from_numpy(hits_all.view(np.uint8).copy()).to(dev)
    pos = torch.empty(max(1, hits_all.size * 16), dtype=torch.int64, device=dev)
    npos = torch.empty(max(1, hits_all.size), dtype=torch.int32, device=dev)
    sa_ms = []
    with torch.cuda.stream(stream):
        for it in range(args.warmup + args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            dix.sa_to_pos(dh, hits_all.size, 16, pos, npos, stream)
            e1.record(stream)
            e1.synchronize()
            if it >= args.warmup:
                sa_ms.append(e0.elapsed_time(e1))
    np_h = npos.cpu().numpy().view(np.uint32)[:hits_all.size]
    n_pos = int(np_h[np_h <= 16].sum())
    line["sa_to_pos"] = {"hits": int(hits_all.size), "positions": n_pos, "ms": float(np.mean(sa_ms)),
                         "positions_per_s": n_pos / (np.mean(sa_ms) / 1000)}
    if rank == 0:
        line["accuracy"] = accuracy_report(w, out["persistent"], pos, npos, hit_cap, valid)
    if not use_oracle and rank == 0 and not args.no_oracle:
        line["parity"] = property_checks(w, out["persistent"], pos, npos, hit_cap, hits_all.size, valid)
    if use_oracle:
        # positions of the sampled reads' hits against the oracle's full suffix arrays
        sel_hits = hg[sel][np.arange(hit_cap)[None, :] < rg[sel]["n_hits"][:, None]]
        pos_h = pos.cpu().numpy().view(np.uint64)[:hits_all.size * 16].reshape(-1, 16)
        idx_valid = np.nonzero(valid.reshape(-1))[0]
        row_of = np.full(valid.size, -1, np.int64)
        row_of[idx_valid] = np.arange(idx_valid.size)
        flat_sel = (sel[:, None] * hit_cap + np.arange(hit_cap)[None, :])[np.arange(hit_cap)[None, :] < rg[sel]["n_hits"][:, None]]
        rows = row_of[flat_sel]
        import oracle
        oh = np.zeros(sel_hits.size, oracle.HIT_DTYPE)
        for f in ("k", "l", "aligned_len", "strand"):
            oh[f] = sel_hits[f]
        opos, onpos = ox.positions(oh, 16)
        okp = True
        for j, rrow in enumerate(rows):
            w_ = int(sel_hits[j]["l"]) - int(sel_hits[j]["k"]) + 1
            if w_ <= 16:
                okp = okp and int(np_h[rrow]) == int(onpos[j]) and np.array_equal(pos_h[rrow, :w_], opos[j, :w_])
            else:
                okp = okp and int(np_h[rrow]) == 0xFFFFFFFF
        line["parity"]["positions_bit_exact"] = bool(okp)
        line["parity"]["positions_hits_checked"] = int(sel_hits.size)
    if args.serve_seconds > 0:
        line["serving"] = serving_phase(aln, dix, w, args.serve_lambda, args.serve_seconds, slots=args.serve_slots,
                                        batch_reads=args.serve_batch_reads)
        line["p99_ms"] = line["serving"]["p99_ms"]
    if args.human and ws == 1:
        args._probes = probes
        del al, dix, res, hits, d
        torch.cuda.empty_cache()
        line["human"] = human_phase(args, aln, torch, dev, stream, flush)
        if "serving" in line["human"]:
            line["p99_ms"] = line["human"]["serving"]["p99_ms"]
            line["p99_source"] = "human.serving (3.1 Gbp text, lambda = %g req/s)" % args.human_serve_lambda
    line["wall_s"] = time.time() - t_all
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="chr100", choices=["chr100", "tiny36", "human_mixed", "human_pairs"])
    ap.add_argument("--ref-len", type=int, default=0, help="reference length (default: the workload's)")
    ap.add_argument("--oracle-max-bp", type=int, default=400_000_000,
                    help="above this text size the oracle is not built; sampled hits are checked by properties")
    ap.add_argument("--kmer-k", type=int, default=10)
    ap.add_argument("--blocks-per-sm", type=int, default=0)
    ap.add_argument("--work-limit", type=int, default=0, help="node expansions per read (0 = library default)")
    ap.add_argument("--autotune", action="store_true", help="choose blocks per SM and stack depth with aln_autotune first")
    ap.add_argument("--index-cache", default="", help="load the index image from this file, or build and save it")
    ap.add_argument("--graph", action="store_true", help="time the persistent form as CUDA-graph replays")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-sample", type=int, default=2000)
    ap.add_argument("--gather-probe", type=int, default=1,
                    help="1: measure the random 64-byte gather rate over a 4 GiB buffer (aln_gather_probe)")
    ap.add_argument("--no-oracle", action="store_true")
    ap.add_argument("--reads", type=int, default=0, help="use only the first N reads (profiling runs)")
    ap.add_argument("--serve-seconds", type=float, default=15.0)
    ap.add_argument("--serve-lambda", type=float, default=100.0)
    ap.add_argument("--serve-slots", type=int, default=3, help="server: batches in flight")
    ap.add_argument("--serve-batch-reads", type=int, default=1 << 19, help="server: reads per batch")
    ap.add_argument("--human", type=int, default=1,
                    help="1: also run the 3.1 Gbp paired and mixed-length batches, oracle-checked, and serving on it")
    ap.add_argument("--human-ref", type=int, default=0, help="human-scale text length (default 3.1 Gbp)")
    ap.add_argument("--human-reads", type=int, default=1_000_000, help="reads per human-scale batch")
    ap.add_argument("--human-steps", type=int, default=3)
    ap.add_argument("--human-warmup", type=int, default=3)
    ap.add_argument("--human-serve-seconds", type=float, default=60.0)
    ap.add_argument("--human-serve-lambda", type=float, default=50.0)
    ap.add_argument("--l2-window", type=int, default=0,
                    help="1: hold the prefix-trie tables in L2's persisting set during the search (l2_window)")
    ap.add_argument("--index-build", default="gpu", choices=["gpu", "host"],
                    help="build the index with fm_index_build_gpu (default) or on the host cores")
    args = ap.parse_args()
    if args.gpus > 1 and "RANK" not in os.environ:
        # one process per GPU: re-launch this command under torch.distributed.run
        import socket
        sk = socket.socket()
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
        sk.close()
        cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={args.gpus}",
               "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.abspath(__file__), *sys.argv[1:]]
        os.execv(sys.executable, cmd)
    if args.warmup < 3 and args.impl == "gb300":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
