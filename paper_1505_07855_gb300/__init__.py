"""GB300-native BWA-aln inexact FM-index search (the hot path of BarraCUDA).

Python binding of the C ABI in include/aln_gb300.h.  PyTorch supplies device
memory and streams; the index build runs in the library's host C++ and every
step of the search runs in its sm_103a kernels.  There is no CPU fallback.

Typical use::

    idx = Index.build(text_codes)            # fm_index_build
    dix = idx.to_device(0)                   # fm_index_to_device
    al = Aligner(dix)
    res, hits = al.align(codes, offsets, lens, Params(z=2))   # aln_search
    pos, npos = al.positions(hits_device, n, 16)              # sa_to_pos
"""
from __future__ import annotations

import ctypes
import dataclasses

import numpy as np

from . import _lib
from ._lib import (  # noqa: F401
    ALN_ELIMIT, ALN_OK, AlnError, CAND_CAP, FLAG_BAD_LIMIT, FLAG_CAND_OVERFLOW, FLAG_HIT_OVERFLOW,
    FLAG_INCOMPLETE, FLAG_LOOP_LIMIT, FLAG_MANY_BEST, FLAG_READ_TOO_LONG, FLAG_STACK_OVERFLOW, FLAG_WORK_LIMIT,
    HIT_DTYPE, MAX_HIT_CAP, MAX_READ_LEN, MAX_Z, MODE_PERSISTENT, MODE_PLAIN, POS_BAD_HIT,
    POS_TOO_WIDE, POS_WALK_LIMIT, RES_DTYPE, SMEM_STACK_CHOICES, HEAVY_AFTER_DEFAULT, HEAVY_PASSES, STATUS_LOOP_LIMIT, STRATA_BEST1,
    STRATA_FULL, STRATA_SCORE, check, lib, library_path, PAIR_DTYPE, PAIR_MAPPED1, PAIR_MAPPED2, PAIR_PLACED1, PAIR_PLACED2,
    PAIR_UNIQUE, PAIR_PROPER, PAIR_DISCORDANT, PAIR_STATS_FIELDS,
)

__all__ = ["Index", "DeviceIndex", "Params", "Aligner", "pack_reads", "gather_probe", "scratch_bytes",
           "HIT_DTYPE", "RES_DTYPE"]


def _ptr(a) -> int | None:
    """Address of a numpy array or a torch tensor (None for None)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return int(a.data_ptr())


class Index:
    """Host FM-index of X and of X reversed (fm_index_build / load)."""

    def __init__(self, handle: int):
        self._h = ctypes.c_void_p(handle)

    @classmethod
    def build(cls, text: np.ndarray, n_seed: int = 0, sa_sample: int = 32, kmer_k: int = 0,
              threads: int = 0, device: int | None = None, stream=None) -> "Index":
        """fm_index_build on the host, or fm_index_build_gpu on CUDA device
        ``device`` (same index, byte for byte)."""
        t = np.ascontiguousarray(text, dtype=np.uint8)
        opts = _lib.fm_build_opts(n_seed, sa_sample, kmer_k, threads, 0)
        out = ctypes.c_void_p()
        if device is None:
            check(lib().fm_index_build(_ptr(t), t.size, ctypes.byref(opts), ctypes.byref(out)),
                  "fm_index_build")
        else:
            check(lib().fm_index_build_gpu(_ptr(t), t.size, ctypes.byref(opts), device, _stream_ptr(stream),
                                           ctypes.byref(out)), "fm_index_build_gpu")
        return cls(out.value)

    @classmethod
    def load(cls, path: str) -> "Index":
        out = ctypes.c_void_p()
        check(lib().fm_index_load(path.encode(), ctypes.byref(out)), "fm_index_load")
        return cls(out.value)

    def save(self, path: str) -> None:
        check(lib().fm_index_save(self._h, path.encode()), "fm_index_save")

    def info(self) -> dict:
        i = _lib.fm_index_info_t()
        check(lib().fm_index_info(self._h, ctypes.byref(i)), "fm_index_info")
        return _info_dict(i)

    def to_device(self, device: int = 0, stream=None) -> "DeviceIndex":
        out = ctypes.c_void_p()
        check(lib().fm_index_to_device(self._h, device, _stream_ptr(stream), ctypes.byref(out)),
              "fm_index_to_device")
        return DeviceIndex(out.value, device)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib().fm_index_free(h)
            self._h = None


def _info_dict(i) -> dict:
    return {"n": i.n, "primary": list(i.primary), "C": [list(i.C[0]), list(i.C[1])],
            "occ_bytes": i.occ_bytes, "sa_bytes": i.sa_bytes, "kmer_bytes": i.kmer_bytes,
            "sa_sample": i.sa_sample, "kmer_k": i.kmer_k}


def _stream_ptr(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


class DeviceIndex:
    """Device-resident index image (fm_index_to_device)."""

    def __init__(self, handle: int, device: int):
        self._h = ctypes.c_void_p(handle)
        self.device = device

    def info(self) -> dict:
        i = _lib.fm_index_info_t()
        check(lib().fm_dindex_info(self._h, ctypes.byref(i)), "fm_dindex_info")
        return _info_dict(i)

    def search(self, bases, nmask, offsets, lens, z, n_reads: int, params: "Params",
               res_out, hits_out, stream=None, status=None, scratch=None) -> None:
        """aln_search on device buffers (torch tensors or raw addresses).  status:
        a device word receiving ALN_STATUS_* bits; scratch: a device buffer of at
        least scratch_bytes(n_reads) bytes for the persistent form's pre-pass."""
        b = _lib.aln_batch(_ptr(bases), _ptr(nmask), _ptr(offsets), _ptr(lens), _ptr(z))
        nbytes = 0 if scratch is None else scratch.numel() * scratch.element_size()
        r = _lib.aln_result(_ptr(res_out), _ptr(hits_out), _ptr(status), _ptr(scratch), nbytes)
        p = params.c()
        check(lib().aln_search(self._h, ctypes.byref(b), n_reads, ctypes.byref(p), ctypes.byref(r),
                               _stream_ptr(stream)), "aln_search")

    def sa_to_pos(self, hits, n_hits: int, max_width: int, pos_out, npos_out, stream=None) -> None:
        check(lib().sa_to_pos(self._h, _ptr(hits), n_hits, max_width, _ptr(pos_out), _ptr(npos_out),
                              _stream_ptr(stream)), "sa_to_pos")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib().fm_dindex_free(h)
            self._h = None


def scratch_bytes(n_reads: int) -> int:
    """aln_search_scratch_bytes: bytes of caller scratch the persistent form uses."""
    return int(lib().aln_search_scratch_bytes(n_reads))


def gather_probe(buf, n_gathers: int, seed: int, sink, stream=None) -> None:
    """aln_gather_probe: n_gathers random 64-byte block reads of the device tensor
    buf; sink (a device int32/uint32 tensor of one element) is XORed with the XOR
    of every gathered block's 16 words."""
    check(lib().aln_gather_probe(_ptr(buf), buf.numel() * buf.element_size(), n_gathers, seed, _ptr(sink),
                                 _stream_ptr(stream)), "aln_gather_probe")


@dataclasses.dataclass
class Params:
    """Search limits (aln_params)."""
    z: int = 2
    max_gapo: int = 1
    max_gape: int = 2
    seed_len: int = 0
    seed_z: int = 0
    indel_end_skip: int = 5
    hit_cap: int = 32
    mode: int = MODE_PLAIN
    strata: int = STRATA_BEST1
    work_limit: int = 0
    blocks_per_sm: int = 0
    smem_stack: int = 0
    loop_limit: int = 0
    help_after: int = 0
    l2_window: int = 0
    heavy_after: int = 0
    score_mm: int = 0
    score_gapo: int = 0
    score_gape: int = 0
    max_best: int = 0

    def c(self) -> _lib.aln_params:
        return _lib.aln_params(self.z, self.max_gapo, self.max_gape, self.seed_len, self.seed_z,
                               self.indel_end_skip, self.hit_cap, self.mode, self.strata,
                               self.blocks_per_sm, self.smem_stack, self.l2_window, self.work_limit,
                               self.loop_limit, self.help_after, self.heavy_after, self.score_mm,
                               self.score_gapo, self.score_gape, self.max_best)

    @classmethod
    def from_limits(cls, lim: dict, **kw) -> "Params":
        """Params from a limits dict; keyword arguments override its entries."""
        d = dict(z=lim["z"], max_gapo=lim["max_gapo"], max_gape=lim["max_gape"],
                 seed_len=lim["seed_len"], seed_z=lim["seed_z"], indel_end_skip=lim["indel_end_skip"])
        d.update(kw)
        return cls(**d)


def pack_reads(codes: np.ndarray, offsets: np.ndarray, lens: np.ndarray):
    """aln_pack_reads: codes 0..4 -> (bases u32, nmask u32, offsets u64), host arrays."""
    codes = np.ascontiguousarray(codes, dtype=np.uint8)
    offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
    lens = np.ascontiguousarray(lens, dtype=np.uint16)
    total = int(lens.astype(np.int64).sum())
    bases = np.zeros(max(1, (total + 15) // 16), np.uint32)
    nmask = np.zeros(max(1, (total + 31) // 32), np.uint32)
    offs = np.zeros(lens.size, np.uint64)
    check(lib().aln_pack_reads(_ptr(codes), _ptr(offsets), _ptr(lens), lens.size, _ptr(bases),
                               _ptr(nmask), _ptr(offs)), "aln_pack_reads")
    return bases, nmask, offs


class Aligner:
    """Device buffers (torch) around a DeviceIndex for host-array convenience calls."""

    def __init__(self, dindex: DeviceIndex):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("Aligner needs a CUDA device; there is no CPU path")
        self.dix = dindex
        self.torch = torch
        self.dev = torch.device("cuda", dindex.device)
        self.status = torch.zeros(1, dtype=torch.int32, device=self.dev)  # ALN_STATUS_* of the last search

    def upload(self, codes, offsets, lens, z=None):
        """Pack reads on the host and copy them to the device."""
        t = self.torch
        bases, nmask, offs = pack_reads(codes, offsets, lens)
        d = {
            "bases": t.from_numpy(bases.view(np.int32)).to(self.dev),
            "nmask": t.from_numpy(nmask.view(np.int32)).to(self.dev),
            "offsets": t.from_numpy(offs.view(np.int64)).to(self.dev),
            "lens": t.from_numpy(np.ascontiguousarray(lens, np.uint16).view(np.int16)).to(self.dev),
            "z": None if z is None else t.from_numpy(np.ascontiguousarray(z, np.uint8)).to(self.dev),
            "n": int(np.asarray(lens).size),
        }
        return d

    def outputs(self, n: int, hit_cap: int):
        t = self.torch
        res = t.empty(max(1, n) * RES_DTYPE.itemsize, dtype=t.uint8, device=self.dev)
        hits = t.empty(max(1, n * hit_cap) * HIT_DTYPE.itemsize, dtype=t.uint8, device=self.dev)
        return res, hits

    def search_device(self, d, params: Params, res, hits, stream=None, scratch=None):
        self.dix.search(d["bases"], d["nmask"], d["offsets"], d["lens"], d["z"], d["n"], params,
                        res, hits, stream, status=self.status, scratch=scratch)

    def last_status(self) -> int:
        """ALN_STATUS_* bits of the last search (synchronises with the device)."""
        return int(self.status.item())

    def check_status(self, where: str = "aln_search") -> None:
        """Raise AlnError(ALN_ELIMIT) if the last search stopped at its loop bound."""
        st = self.last_status()
        if st & STATUS_LOOP_LIMIT:
            raise AlnError(ALN_ELIMIT, where, "the persistent loop reached params.loop_limit; "
                                              "unfinished reads carry ALN_FLAG_LOOP_LIMIT")

    def autotune(self, d, params: Params, res, hits, stream=None) -> tuple:
        """aln_autotune on an uploaded sample: returns (params with the fastest
        blocks_per_sm and smem_stack, its time in ms)."""
        b = _lib.aln_batch(_ptr(d["bases"]), _ptr(d["nmask"]), _ptr(d["offsets"]), _ptr(d["lens"]), _ptr(d["z"]))
        r = _lib.aln_result(_ptr(res), _ptr(hits), _ptr(self.status), None, 0)
        p = params.c()
        ms = ctypes.c_float()
        check(lib().aln_autotune(self.dix._h, ctypes.byref(b), d["n"], ctypes.byref(p), ctypes.byref(r),
                                 _stream_ptr(stream), ctypes.byref(ms)), "aln_autotune")
        return dataclasses.replace(params, blocks_per_sm=p.blocks_per_sm, smem_stack=p.smem_stack), ms.value

    def capture(self, d, params: Params, res, hits):
        """Capture one search of the uploaded batch d into a CUDA graph; replay it
        with graph.replay() for every new batch copied into the same buffers.
        The graph owns a queue counter of its own and a scratch buffer (kept on
        the graph object as ``aln_scratch``) for the D pre-pass and visit order,
        so a replay runs the same four kernels as aln_search.  Replays of one
        graph must not overlap each other."""
        t = self.torch
        scratch = t.empty(scratch_bytes(d["n"]), dtype=t.uint8, device=self.dev)
        side = t.cuda.Stream(device=self.dev)
        side.wait_stream(t.cuda.current_stream(self.dev))
        with t.cuda.stream(side):  # warm-up outside the capture
            self.search_device(d, params, res, hits, side, scratch=scratch)
        t.cuda.current_stream(self.dev).wait_stream(side)
        t.cuda.synchronize(self.dev)
        g = t.cuda.CUDAGraph()
        with t.cuda.graph(g):
            self.search_device(d, params, res, hits, t.cuda.current_stream(self.dev), scratch=scratch)
        g.aln_scratch = scratch
        return g

    def align(self, codes, offsets, lens, params: Params, z=None, stream=None, check_status: bool = True):
        """Host arrays in, numpy (res[n], hits[n, hit_cap]) out.  Raises
        AlnError(ALN_ELIMIT) if the search stopped at its loop bound (unless
        check_status is False: the flagged results are returned)."""
        d = self.upload(codes, offsets, lens, z)
        n = d["n"]
        res, hits = self.outputs(n, params.hit_cap)
        self.search_device(d, params, res, hits, stream)
        self.torch.cuda.synchronize(self.dev)
        if check_status:
            self.check_status()
        r = res.cpu().numpy().view(RES_DTYPE)[:n]
        h = hits.cpu().numpy().view(HIT_DTYPE)[:n * params.hit_cap].reshape(n, params.hit_cap)
        return r, h

    def compact(self, res, hits, n: int, hit_cap: int, offsets, dense, scratch, stream=None) -> None:
        """aln_compact_hits on device buffers: offsets (n + 1 uint32), dense hits
        (its capacity is its size in hits), scratch (aln_compact_scratch_bytes)."""
        check(lib().aln_compact_hits(_ptr(res), _ptr(hits), n, hit_cap, _ptr(offsets), _ptr(dense),
                                     dense.numel() * dense.element_size() // HIT_DTYPE.itemsize, _ptr(scratch),
                                     scratch.numel() * scratch.element_size(), _stream_ptr(stream)),
              "aln_compact_hits")

    def compact_scratch(self, n: int):
        """A device buffer for aln_compact_hits' scratch."""
        t = self.torch
        return t.empty(int(lib().aln_compact_scratch_bytes(n)), dtype=t.uint8, device=self.dev)

    def pair(self, res, n_reads: int, hit_cap: int, hits, max_width: int = 16, max_place: int = 16,
             stream=None):
        """Pairing of reads 2p / 2p+1 from a search's device outputs (res, hits):
        aln_compact_hits, sa_to_pos of the dense hits, aln_pair_resolve.
        Returns numpy (pairs PAIR_DTYPE[n_reads // 2], stats dict)."""
        t = self.torch
        n_pairs = n_reads // 2
        off = t.empty(n_reads + 1, dtype=t.int32, device=self.dev)
        dense = t.empty(max(1, n_reads * hit_cap) * HIT_DTYPE.itemsize, dtype=t.uint8, device=self.dev)
        self.compact(res, hits, n_reads, hit_cap, off, dense, self.compact_scratch(n_reads), stream)
        t.cuda.synchronize(self.dev)
        total = int(off[n_reads].item())
        pos = t.empty(max(1, total * max_width), dtype=t.int64, device=self.dev)
        npos = t.empty(max(1, total), dtype=t.int32, device=self.dev)
        if total:
            self.dix.sa_to_pos(dense, total, max_width, pos, npos, stream)
        out = t.empty(max(1, n_pairs) * PAIR_DTYPE.itemsize, dtype=t.uint8, device=self.dev)
        stats = t.zeros(8, dtype=t.int32, device=self.dev)
        scratch = t.empty(int(lib().aln_pair_scratch_bytes()), dtype=t.uint8, device=self.dev)
        check(lib().aln_pair_resolve(_ptr(res), _ptr(off), _ptr(dense), _ptr(pos), _ptr(npos), max_width, n_pairs,
                                     max_place, _ptr(out), _ptr(stats), _ptr(scratch),
                                     scratch.numel(), _stream_ptr(stream)), "aln_pair_resolve")
        t.cuda.synchronize(self.dev)
        st = stats.cpu().numpy().view(np.uint32)
        return (out.cpu().numpy().view(PAIR_DTYPE)[:n_pairs].copy(),
                dict(zip(PAIR_STATS_FIELDS, (int(x) for x in st[:6]))))

    def positions(self, hits_np: np.ndarray, max_width: int = 16, stream=None):
        """sa_to_pos for a host array of hits; returns (pos[n, max_width], npos[n])."""
        t = self.torch
        h = np.ascontiguousarray(hits_np, dtype=HIT_DTYPE).reshape(-1)
        n = h.size
        dh = t.from_numpy(h.view(np.uint8)).to(self.dev)
        pos = t.zeros(max(1, n * max_width), dtype=t.int64, device=self.dev)
        npos = t.zeros(max(1, n), dtype=t.int32, device=self.dev)
        self.dix.sa_to_pos(dh, n, max_width, pos, npos, stream)
        t.cuda.synchronize(self.dev)
        return (pos.cpu().numpy().view(np.uint64)[:n * max_width].reshape(n, max_width),
                npos.cpu().numpy().view(np.uint32)[:n])


class Server:
    """Continuous-batching request loop on a resident index (aln_server_*)."""

    def __init__(self, dindex: DeviceIndex, params: Params, n_slots: int = 3,
                 max_batch_reads: int = 1 << 18, max_batch_bases: int = 0, device_mem_budget: int = 0,
                 coalesce_us: int = 200):
        self.dix = dindex
        self.params = params
        cfg = _lib.aln_server_config()
        cfg.device = dindex.device
        cfg.n_slots = n_slots
        cfg.max_batch_reads = max_batch_reads
        cfg.max_batch_bases = max_batch_bases or max_batch_reads * 256
        cfg.device_mem_budget = device_mem_budget
        cfg.coalesce_us = coalesce_us
        cfg.params = params.c()
        out = ctypes.c_void_p()
        check(lib().aln_server_create(dindex._h, ctypes.byref(cfg), ctypes.byref(out)), "aln_server_create")
        self._h = out

    def submit(self, codes, offsets, lens, z=None) -> int:
        codes = np.ascontiguousarray(codes, dtype=np.uint8)
        offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
        lens = np.ascontiguousarray(lens, dtype=np.uint16)
        zz = None if z is None else np.ascontiguousarray(z, dtype=np.uint8)
        rid = ctypes.c_uint64()
        check(lib().aln_server_submit(self._h, _ptr(codes), _ptr(offsets), _ptr(lens), _ptr(zz), lens.size,
                                      ctypes.byref(rid)), "aln_server_submit")
        return rid.value

    def poll(self, rid: int, n_reads: int, wait_ms: int = 60000):
        """Results of a finished request as (res, hits, latency_ms), or None if not done."""
        res = np.zeros(max(1, n_reads), RES_DTYPE)
        hits = np.zeros(max(1, n_reads * self.params.hit_cap), HIT_DTYPE)
        lat = ctypes.c_double()
        rc = lib().aln_server_poll(self._h, rid, wait_ms, _ptr(res), _ptr(hits), ctypes.byref(lat))
        if rc == _lib.ALN_EAGAIN:
            return None
        check(rc, "aln_server_poll")
        return res[:n_reads], hits[:n_reads * self.params.hit_cap].reshape(n_reads, self.params.hit_cap), lat.value

    def stats(self) -> dict:
        st = _lib.aln_server_stats_t()
        check(lib().aln_server_stats(self._h, ctypes.byref(st)), "aln_server_stats")
        return {f: getattr(st, f) for f, _ in st._fields_ if f != "reserved"}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().aln_server_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()
