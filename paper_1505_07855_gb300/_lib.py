"""ctypes binding of libaln_gb300.so: the C ABI of include/aln_gb300.h with the
same names.  Argument marshalling only; every step of the search runs in the
library's CUDA kernels.  There is no fallback: if the library is missing or
fails to load, every entry point raises."""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

ALN_OK = 0
STATUS = {0: "ALN_OK", -1: "ALN_EINVAL", -2: "ALN_ENOMEM", -3: "ALN_EDEVICE", -4: "ALN_ELIMIT",
          -5: "ALN_EOVERFLOW", -6: "ALN_EIO", -7: "ALN_EAGAIN"}
ALN_EAGAIN = -7
MAX_READ_LEN = 255
MAX_Z = 7
MAX_HIT_CAP = 255
CAND_CAP = 512
FLAG_HIT_OVERFLOW = 0x01
FLAG_STACK_OVERFLOW = 0x02
FLAG_CAND_OVERFLOW = 0x04
FLAG_READ_TOO_LONG = 0x08
FLAG_BAD_LIMIT = 0x10
FLAG_WORK_LIMIT = 0x20
FLAG_LOOP_LIMIT = 0x40
FLAG_MANY_BEST = 0x80
FLAG_INCOMPLETE = FLAG_STACK_OVERFLOW | FLAG_CAND_OVERFLOW | FLAG_WORK_LIMIT | FLAG_LOOP_LIMIT
STATUS_LOOP_LIMIT = 0x1
ALN_ELIMIT = -4
SMEM_STACK_CHOICES = (4, 8, 12)
HEAVY_PASSES = 5
HEAVY_AFTER_DEFAULT = 65536
MODE_PLAIN, MODE_PERSISTENT = 0, 1
STRATA_BEST1, STRATA_FULL, STRATA_SCORE = 0, 1, 2
POS_TOO_WIDE = 0xFFFFFFFF
POS_WALK_LIMIT = 0xFFFFFFFE
POS_BAD_HIT = 0xFFFFFFFD

PAIR_MAPPED1, PAIR_MAPPED2, PAIR_PLACED1, PAIR_PLACED2 = 0x01, 0x02, 0x04, 0x08
PAIR_UNIQUE, PAIR_PROPER, PAIR_DISCORDANT = 0x10, 0x20, 0x40
PAIR_DTYPE = np.dtype([("pos", "<u8", (2,)), ("insert", "<u4"), ("n_proper", "<u2"), ("strand", "u1", (2,)),
                       ("flags", "u1"), ("reserved", "u1", (7,))])
PAIR_STATS_FIELDS = ("n_unique", "q1", "q2", "q3", "lo", "hi")

# numpy views of aln_hit (16 B) and aln_read_result (12 B)
HIT_DTYPE = np.dtype([("k", "<u4"), ("l", "<u4"), ("aligned_len", "<u2"), ("strand", "u1"),
                      ("n_diff", "u1"), ("n_mm", "u1"), ("n_gapo", "u1"), ("n_gape", "u1"),
                      ("reserved", "u1")])
RES_DTYPE = np.dtype([("c0", "<u4"), ("c1", "<u4"), ("n_hits", "u1"), ("flags", "u1"),
                      ("d_best", "u1"), ("best_score", "u1")])


class fm_build_opts(ctypes.Structure):
    _fields_ = [("n_seed", ctypes.c_uint64), ("sa_sample", ctypes.c_uint32),
                ("kmer_k", ctypes.c_uint32), ("n_threads", ctypes.c_int32),
                ("reserved", ctypes.c_uint32)]


class fm_index_info_t(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint64), ("primary", ctypes.c_uint64 * 2),
                ("C", (ctypes.c_uint64 * 4) * 2), ("occ_bytes", ctypes.c_uint64),
                ("sa_bytes", ctypes.c_uint64), ("kmer_bytes", ctypes.c_uint64),
                ("sa_sample", ctypes.c_uint32), ("kmer_k", ctypes.c_uint32)]


class aln_batch(ctypes.Structure):
    _fields_ = [("bases", ctypes.c_void_p), ("nmask", ctypes.c_void_p), ("offset", ctypes.c_void_p),
                ("len", ctypes.c_void_p), ("z", ctypes.c_void_p)]


class aln_params(ctypes.Structure):
    _fields_ = [("z", ctypes.c_uint8), ("max_gapo", ctypes.c_uint8), ("max_gape", ctypes.c_uint8),
                ("seed_len", ctypes.c_uint8), ("seed_z", ctypes.c_uint8),
                ("indel_end_skip", ctypes.c_uint8), ("hit_cap", ctypes.c_uint8),
                ("mode", ctypes.c_uint8), ("strata", ctypes.c_uint8),
                ("blocks_per_sm", ctypes.c_uint8), ("smem_stack", ctypes.c_uint8),
                ("l2_window", ctypes.c_uint8), ("work_limit", ctypes.c_uint32),
                ("loop_limit", ctypes.c_uint32), ("help_after", ctypes.c_uint32),
                ("heavy_after", ctypes.c_uint32), ("score_mm", ctypes.c_uint8), ("score_gapo", ctypes.c_uint8),
                ("score_gape", ctypes.c_uint8), ("max_best", ctypes.c_uint8)]


class aln_result(ctypes.Structure):
    _fields_ = [("reads", ctypes.c_void_p), ("hits", ctypes.c_void_p), ("status", ctypes.c_void_p),
                ("scratch", ctypes.c_void_p), ("scratch_bytes", ctypes.c_uint64)]


class aln_server_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("n_slots", ctypes.c_uint32),
                ("max_batch_reads", ctypes.c_uint32), ("max_batch_bases", ctypes.c_uint64),
                ("device_mem_budget", ctypes.c_uint64), ("coalesce_us", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32), ("params", aln_params)]


class aln_server_stats_t(ctypes.Structure):
    _fields_ = [("requests_done", ctypes.c_uint64), ("reads_done", ctypes.c_uint64),
                ("batches", ctypes.c_uint64), ("queued_reads", ctypes.c_uint64),
                ("p50_ms", ctypes.c_double), ("p95_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("seconds", ctypes.c_double), ("n_slots", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


assert ctypes.sizeof(aln_params) == 32 and ctypes.sizeof(fm_build_opts) == 24
assert PAIR_DTYPE.itemsize == 32
assert ctypes.sizeof(fm_index_info_t) == 120 and ctypes.sizeof(aln_result) == 40
assert ctypes.sizeof(aln_server_config) == 72 and ctypes.sizeof(aln_server_stats_t) == 72

# name -> (restype, argtypes); the exported ABI
P, u8p = ctypes.c_void_p, ctypes.c_void_p
SIGNATURES = {
    "fm_index_build": (ctypes.c_int, [P, ctypes.c_uint64, ctypes.POINTER(fm_build_opts), ctypes.POINTER(P)]),
    "fm_index_build_gpu": (ctypes.c_int, [P, ctypes.c_uint64, ctypes.POINTER(fm_build_opts), ctypes.c_int, P,
                                          ctypes.POINTER(P)]),
    "fm_index_free": (None, [P]),
    "fm_index_info": (ctypes.c_int, [P, ctypes.POINTER(fm_index_info_t)]),
    "fm_index_save": (ctypes.c_int, [P, ctypes.c_char_p]),
    "fm_index_load": (ctypes.c_int, [ctypes.c_char_p, ctypes.POINTER(P)]),
    "fm_index_to_device": (ctypes.c_int, [P, ctypes.c_int, P, ctypes.POINTER(P)]),
    "fm_dindex_free": (None, [P]),
    "fm_dindex_info": (ctypes.c_int, [P, ctypes.POINTER(fm_index_info_t)]),
    "aln_search": (ctypes.c_int, [P, ctypes.POINTER(aln_batch), ctypes.c_uint32,
                                  ctypes.POINTER(aln_params), ctypes.POINTER(aln_result), P]),
    "aln_search_scratch_bytes": (ctypes.c_uint64, [ctypes.c_uint32]),
    "sa_to_pos": (ctypes.c_int, [P, P, ctypes.c_uint32, ctypes.c_uint32, P, P, P]),
    "aln_compact_scratch_bytes": (ctypes.c_uint64, [ctypes.c_uint32]),
    "aln_pair_scratch_bytes": (ctypes.c_uint64, []),
    "aln_pair_resolve": (ctypes.c_int, [P, P, P, P, P, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, P, P, P,
                                        ctypes.c_uint64, P]),
    "aln_compact_hits": (ctypes.c_int, [P, P, ctypes.c_uint32, ctypes.c_uint32, P, P, ctypes.c_uint64, P,
                                        ctypes.c_uint64, P]),
    "aln_autotune": (ctypes.c_int, [P, ctypes.POINTER(aln_batch), ctypes.c_uint32, ctypes.POINTER(aln_params),
                                    ctypes.POINTER(aln_result), P, ctypes.POINTER(ctypes.c_float)]),
    "aln_search_noalloc": (ctypes.c_int, [P, ctypes.POINTER(aln_batch), ctypes.c_uint32,
                                          ctypes.POINTER(aln_params), ctypes.POINTER(aln_result), P]),
    "aln_gather_probe": (ctypes.c_int, [P, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32, P, P]),
    "aln_pack_reads": (ctypes.c_int, [P, P, P, ctypes.c_uint32, P, P, P]),
    "aln_server_create": (ctypes.c_int, [P, ctypes.POINTER(aln_server_config), ctypes.POINTER(P)]),
    "aln_server_submit": (ctypes.c_int, [P, P, P, P, P, ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint64)]),
    "aln_server_poll": (ctypes.c_int, [P, ctypes.c_uint64, ctypes.c_int, P, P, ctypes.POINTER(ctypes.c_double)]),
    "aln_server_stats": (ctypes.c_int, [P, ctypes.POINTER(aln_server_stats_t)]),
    "aln_server_destroy": (None, [P]),
    "aln_last_error": (ctypes.c_char_p, []),
    "aln_version": (ctypes.c_int, []),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = True):
    """Load the library (building it first if it is absent)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(f"libaln_gb300.so not built ({path}); run __graft_entry__.build()")
            _build.build()
        L = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class AlnError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str | None = None):
        if msg is None:
            msg = lib().aln_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS.get(status, status)}: {msg}")
        self.status = status


def check(status: int, where: str) -> None:
    if status != ALN_OK:
        raise AlnError(status, where)
