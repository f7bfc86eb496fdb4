"""CPU oracle for the BWA-aln inexact FM-index search (test infrastructure).

Only the tests, the smoke check and the benchmark's CPU-baseline leg may use this
package.  It wraps ``aln_oracle.c`` (plain C: naive suffix sort, prefix-count
Occ, greedy D scan, recursive exhaustive DFS, iterative deepening) through
ctypes and shares nothing with the CUDA library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "aln_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liborc.so")

HIT_DTYPE = np.dtype([("k", "<u4"), ("l", "<u4"), ("aligned_len", "<u2"), ("strand", "u1"),
                      ("n_diff", "u1"), ("n_mm", "u1"), ("n_gapo", "u1"), ("n_gape", "u1"),
                      ("pad", "u1")])
RES_DTYPE = np.dtype([("c0", "<u4"), ("c1", "<u4"), ("n_hits", "u1"), ("flags", "u1"),
                      ("d_best", "u1"), ("pad", "u1")])
assert HIT_DTYPE.itemsize == 16 and RES_DTYPE.itemsize == 12

PAIR_DTYPE = np.dtype([("pos", "<u8", (2,)), ("insert", "<u4"), ("n_proper", "<u2"), ("strand", "u1", (2,)),
                       ("flags", "u1"), ("pad", "u1", (3,)), ("pad2", "<u4")])
assert PAIR_DTYPE.itemsize == 32
PAIR_MAPPED1, PAIR_MAPPED2, PAIR_PLACED1, PAIR_PLACED2 = 0x01, 0x02, 0x04, 0x08
PAIR_UNIQUE, PAIR_PROPER, PAIR_DISCORDANT = 0x10, 0x20, 0x40

FLAG_HIT_OVERFLOW = 0x01
FLAG_READ_TOO_LONG = 0x08
FLAG_BAD_LIMIT = 0x10
FLAG_MANY_BEST = 0x80
BEST1, FULL, SCORE = 0, 1, 2


class _Params(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int) for f in ("z", "max_gapo", "max_gape", "seed_len", "seed_z",
                                            "indel_end_skip", "hit_cap", "strata", "use_d",
                                            "sc_mm", "sc_gapo", "sc_gape", "max_best")]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into oracle/_build/liborc.so."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-D_POSIX_C_SOURCE=200809L", "-shared",
                               "-fPIC", "-pthread", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        P, u64, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int
        L.orc_build.restype = P
        L.orc_build.argtypes = [P, u64, u64, i32, i32]
        L.orc_free.argtypes = [P]
        L.orc_n.restype = u64
        L.orc_n.argtypes = [P]
        for name in ("orc_get_text", "orc_get_sa", "orc_get_bwt", "orc_get_C"):
            getattr(L, name).argtypes = [P, i32, P]
        L.orc_primary.restype = u64
        L.orc_primary.argtypes = [P, i32]
        L.orc_occ.restype = u64
        L.orc_occ.argtypes = [P, i32, i32, ctypes.c_int64]
        L.orc_exact.restype = i32
        L.orc_exact.argtypes = [P, i32, P, i32, P, P]
        L.orc_align.restype = i32
        L.orc_align.argtypes = [P, P, P, P, P, u64, ctypes.POINTER(_Params), i32, P, P, P]
        L.orc_dscan.restype = i32
        L.orc_dscan.argtypes = [P, i32, P, i32, P]
        L.orc_pair_resolve.restype = i32
        L.orc_pair_resolve.argtypes = [P, P, P, ctypes.c_uint32, u64, i32, P, P]
        L.orc_mix64.restype = u64
        L.orc_mix64.argtypes = [u64]
        L.orc_positions.restype = i32
        L.orc_positions.argtypes = [P, P, u64, ctypes.c_uint32, P, P]
        _lib = L
    return _lib


def mix64(x: int) -> int:
    """The oracle's SplitMix64 output function on state x + 0x9E3779B97F4A7C15."""
    return int(lib().orc_mix64(x & 0xFFFFFFFFFFFFFFFF))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def default_threads() -> int:
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()


class OracleIndex:
    """Index of X (which=0) and of X reversed (which=1), built by naive suffix sort.
    ``bucket_k``: leading symbols the sort groups suffixes by before sorting each
    group with the byte-wise comparator (0 = chosen from the text length)."""

    def __init__(self, text: np.ndarray, n_seed: int = 0, threads: int | None = None, bucket_k: int = 0):
        text = np.ascontiguousarray(text, dtype=np.uint8)
        self._text_keep = text
        self.threads = threads or default_threads()
        h = lib().orc_build(_ptr(text), text.size, n_seed, self.threads, bucket_k)
        if not h:
            raise MemoryError("oracle index build failed")
        self._h = h
        self.n = int(lib().orc_n(h))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_free(h)
            self._h = None

    def text(self, which: int = 0) -> np.ndarray:
        out = np.empty(self.n, np.uint8)
        lib().orc_get_text(self._h, which, _ptr(out))
        return out

    def sa(self, which: int = 0) -> np.ndarray:
        out = np.empty(self.n + 1, np.uint32)
        lib().orc_get_sa(self._h, which, _ptr(out))
        return out

    def bwt(self, which: int = 0) -> np.ndarray:
        out = np.empty(self.n + 1, np.uint8)
        lib().orc_get_bwt(self._h, which, _ptr(out))
        return out

    def C(self, which: int = 0) -> np.ndarray:
        out = np.empty(4, np.uint64)
        lib().orc_get_C(self._h, which, _ptr(out))
        return out

    def primary(self, which: int = 0) -> int:
        return int(lib().orc_primary(self._h, which))

    def occ(self, which: int, c: int, r: int) -> int:
        return int(lib().orc_occ(self._h, which, c, r))

    def exact(self, which: int, pattern) -> tuple[int, int] | None:
        p = np.ascontiguousarray(pattern, dtype=np.uint8)
        k = ctypes.c_uint64()
        l = ctypes.c_uint64()
        ok = lib().orc_exact(self._h, which, _ptr(p), p.size, ctypes.byref(k), ctypes.byref(l))
        return (k.value, l.value) if ok else None

    def dscan(self, strand: int, read) -> np.ndarray:
        r = np.ascontiguousarray(read, dtype=np.uint8)
        D = np.zeros(r.size + 1, np.int32)
        if lib().orc_dscan(self._h, strand, _ptr(r), r.size, _ptr(D)) != 0:
            raise ValueError("read too long")
        return D

    def align(self, codes, offsets, lens, z=None, *, z_default=2, max_gapo=1, max_gape=2,
              seed_len=0, seed_z=0, indel_end_skip=5, hit_cap=32, strata=BEST1, use_d=True,
              threads: int | None = None, score=(3, 11, 4), max_best=0):
        """Search a batch.  Returns (res[n] RES_DTYPE, hits[n, hit_cap] HIT_DTYPE,
        lookups[n] uint64).  strata SCORE: hits ranked by the penalties `score`
        (mismatch, gap open, gap extension); res["pad"] holds the best score."""
        codes = np.ascontiguousarray(codes, dtype=np.uint8)
        offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
        lens = np.ascontiguousarray(lens, dtype=np.uint16)
        n = lens.size
        zp = None
        if z is not None:
            z = np.ascontiguousarray(z, dtype=np.uint8)
            zp = _ptr(z)
        p = _Params(z_default, max_gapo, max_gape, seed_len, seed_z, indel_end_skip, hit_cap,
                    strata, 1 if use_d else 0, score[0], score[1], score[2], max_best)
        res = np.zeros(n, RES_DTYPE)
        hits = np.zeros((n, max(1, hit_cap)), HIT_DTYPE)
        look = np.zeros(n, np.uint64)
        rc = lib().orc_align(self._h, _ptr(codes), _ptr(offsets), _ptr(lens), zp, n,
                             ctypes.byref(p), threads or self.threads, _ptr(res), _ptr(hits),
                             _ptr(look))
        if rc != 0:
            raise ValueError("bad oracle parameters")
        return res, hits[:, :hit_cap], look

    def pair_resolve(self, res: np.ndarray, hits: np.ndarray, max_place: int = 16):
        """Pairing of reads 2p (mate 1) and 2p+1 (mate 2) from their search results
        (res[n], hits[n, hit_cap], n even).  Returns (pairs PAIR_DTYPE[n / 2],
        stats dict: n_unique, q1, q2, q3, lo, hi)."""
        res = np.ascontiguousarray(res, dtype=RES_DTYPE)
        hits = np.ascontiguousarray(hits, dtype=HIT_DTYPE)
        n = res.size
        if n % 2 or hits.shape[0] != n:
            raise ValueError("pairs need an even number of reads and hits[n, hit_cap]")
        out = np.zeros(n // 2, PAIR_DTYPE)
        st = np.zeros(8, np.uint32)
        if lib().orc_pair_resolve(self._h, _ptr(res), _ptr(hits), hits.shape[1], n // 2, max_place, _ptr(out),
                                  _ptr(st)) != 0:
            raise ValueError("bad pairing arguments")
        return out, dict(zip(("n_unique", "q1", "q2", "q3", "lo", "hi"), (int(x) for x in st[:6])))

    def positions(self, hits: np.ndarray, max_width: int = 16):
        """Per hit: sorted forward-strand positions (array of max_width) and count."""
        h = np.ascontiguousarray(hits, dtype=HIT_DTYPE).reshape(-1)
        pos = np.zeros((h.size, max_width), np.uint64)
        npos = np.zeros(h.size, np.uint32)
        lib().orc_positions(self._h, _ptr(h), h.size, max_width, _ptr(pos), _ptr(npos))
        return pos, npos
