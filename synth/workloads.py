"""Named synthetic workloads.  Each returns the reference text (codes 0..4), its N
mask, the reads and the search limits.  Sizes can be scaled down for tests; the
recipe (distributions, rates, structure) stays the same.

Workloads (full sizes):
  tiny36   -- 1 Mbp i.i.d. text, 10 000 x 36 bp, 1 % substitutions, 0.05 % 1-bp
              indels, 2 % of reads with one N; z=2, gap opens <= 1, gap ext <= 2,
              no indel within 5 bp of an end.
  chr100   -- 100 Mbp order-3 Markov text (41 % GC) with 5 % of it copies of 50
              repeat families (300-6000 bp, 2-15 % divergence); 1 M x 100 bp,
              substitutions 0.5 % -> 2 % along the read, 0.02 % indels of 1-3 bp;
              z=4, seed 32 with <= 2 seed differences, gap opens <= 1, gap ext <= 6.
  human_mixed -- 3.1 Gbp i.i.d. text with 45 % repeats (500 families) and 1 % N as
              runs of 100-10 000 bp; reads of length uniform in {36,50,76,100,150,250},
              errors as tiny36, z = min(6, ceil(0.04 len)).
  human_pairs -- same text, pairs of 2 x 100 bp, fragment ~ Normal(500, 50),
              0.1 % chimeric pairs, errors as tiny36, z=4.
"""
from __future__ import annotations

import dataclasses
import numpy as np

from .gen import (Rng, Reads, reference_iid, reference_markov3, overlay_repeats,
                  overlay_n_runs, simulate_reads, simulate_pairs)


def z_for_length(m: int) -> int:
    """z = min(6, ceil(0.04 * m)) in integer arithmetic."""
    return min(6, (4 * m + 99) // 100)


@dataclasses.dataclass
class Workload:
    name: str
    text: np.ndarray          # uint8 codes 0..4
    nmask: np.ndarray | None  # bool, True where the generator wrote N
    reads: Reads
    params: dict              # search limits
    mates: tuple | None = None  # (mate1, mate2) for paired workloads
    meta: dict = dataclasses.field(default_factory=dict)


LIMITS = {
    "tiny36": dict(z=2, max_gapo=1, max_gape=2, seed_len=0, seed_z=0, indel_end_skip=5),
    "chr100": dict(z=4, max_gapo=1, max_gape=6, seed_len=32, seed_z=2, indel_end_skip=5),
    "human_mixed": dict(z=6, max_gapo=1, max_gape=2, seed_len=0, seed_z=0, indel_end_skip=5),
    "human_pairs": dict(z=4, max_gapo=1, max_gape=2, seed_len=0, seed_z=0, indel_end_skip=5),
}

FULL = {
    "tiny36": dict(ref_len=1_000_000, n_reads=10_000),
    "chr100": dict(ref_len=100_000_000, n_reads=1_000_000),
    "human_mixed": dict(ref_len=3_100_000_000, n_reads=10_000_000),
    "human_pairs": dict(ref_len=3_100_000_000, n_reads=5_000_000),
}


def _tiny36(ref_len, n_reads, seed):
    rng = Rng(seed, "tiny36")
    text = reference_iid(ref_len, rng.sub("ref"))
    reads = simulate_reads(text, n_reads, 36, rng.sub("reads"), sub_rate=(0.01, 0.01),
                           indel_rate=0.0005, indel_lens=(1,), n_frac=0.02, z=2)
    return Workload("tiny36", text, None, reads, dict(LIMITS["tiny36"]))


def _chr100(ref_len, n_reads, seed):
    rng = Rng(seed, "chr100")
    text = reference_markov3(ref_len, rng.sub("ref"), gc=0.41)
    rep = overlay_repeats(text, rng.sub("rep"), 0.05, 50, (300, 6000), (0.02, 0.15))
    reads = simulate_reads(text, n_reads, 100, rng.sub("reads"), sub_rate=(0.005, 0.02),
                           indel_rate=0.0002, indel_lens=(1, 2, 3), n_frac=0.0, z=4)
    return Workload("chr100", text, None, reads, dict(LIMITS["chr100"]), meta={"repeats": rep})


def _human_text(ref_len, seed):
    rng = Rng(seed, "human")
    text = reference_iid(ref_len, rng.sub("ref"))
    rep = overlay_repeats(text, rng.sub("rep"), 0.45, 500, (300, 6000), (0.02, 0.15))
    nmask = overlay_n_runs(text, rng.sub("nruns"), 0.01, (100, 10_000))
    return text, nmask, rep


def _human_mixed(ref_len, n_reads, seed):
    text, nmask, rep = _human_text(ref_len, seed)
    rng = Rng(seed, "human_mixed")
    reads = simulate_reads(text, n_reads, (36, 50, 76, 100, 150, 250), rng.sub("reads"),
                           sub_rate=(0.01, 0.01), indel_rate=0.0005, indel_lens=(1,),
                           n_frac=0.02, z_of_len=z_for_length, nmask=nmask)
    return Workload("human_mixed", text, nmask, reads, dict(LIMITS["human_mixed"]),
                    meta={"repeats": rep})


def _human_pairs(ref_len, n_pairs, seed):
    text, nmask, rep = _human_text(ref_len, seed)
    rng = Rng(seed, "human_pairs")
    m1, m2 = simulate_pairs(text, n_pairs, 100, rng.sub("pairs"), nmask=nmask,
                            sub_rate=(0.01, 0.01), indel_rate=0.0005, indel_lens=(1,),
                            n_frac=0.02, z=4)
    # both mates in one batch: pair p -> reads 2p (mate 1) and 2p+1 (mate 2)
    order = np.empty(2 * n_pairs, dtype=np.int64)
    both = Reads.concat([m1, m2])
    order[0::2] = np.arange(n_pairs)
    order[1::2] = n_pairs + np.arange(n_pairs)
    reads = both.subset(order)
    return Workload("human_pairs", text, nmask, reads, dict(LIMITS["human_pairs"]),
                    mates=(m1, m2), meta={"repeats": rep})


def human_workloads(ref_len: int | None = None, n_mixed: int = 1_000_000, n_pairs: int = 500_000,
                    seed: int = 0) -> tuple[Workload, Workload]:
    """The mixed-length and the paired workload over one shared human-scale text
    (generated once): the same reads as ``workload("human_mixed", ...)`` and
    ``workload("human_pairs", ...)`` with these sizes."""
    ref_len = ref_len or FULL["human_mixed"]["ref_len"]
    text, nmask, rep = _human_text(ref_len, seed)
    rng = Rng(seed, "human_mixed")
    reads = simulate_reads(text, n_mixed, (36, 50, 76, 100, 150, 250), rng.sub("reads"),
                           sub_rate=(0.01, 0.01), indel_rate=0.0005, indel_lens=(1,),
                           n_frac=0.02, z_of_len=z_for_length, nmask=nmask)
    mixed = Workload("human_mixed", text, nmask, reads, dict(LIMITS["human_mixed"]), meta={"repeats": rep})
    rng = Rng(seed, "human_pairs")
    m1, m2 = simulate_pairs(text, n_pairs, 100, rng.sub("pairs"), nmask=nmask,
                            sub_rate=(0.01, 0.01), indel_rate=0.0005, indel_lens=(1,),
                            n_frac=0.02, z=4)
    order = np.empty(2 * n_pairs, dtype=np.int64)
    order[0::2] = np.arange(n_pairs)
    order[1::2] = n_pairs + np.arange(n_pairs)
    pairs = Workload("human_pairs", text, nmask, Reads.concat([m1, m2]).subset(order),
                     dict(LIMITS["human_pairs"]), mates=(m1, m2), meta={"repeats": rep})
    return mixed, pairs


WORKLOADS = {"tiny36": _tiny36, "chr100": _chr100, "human_mixed": _human_mixed,
             "human_pairs": _human_pairs}


def workload(name: str, ref_len: int | None = None, n_reads: int | None = None,
             seed: int = 0) -> Workload:
    """Build a named workload; ``ref_len``/``n_reads`` default to the full sizes."""
    full = FULL[name]
    return WORKLOADS[name](ref_len or full["ref_len"], n_reads or full["n_reads"], seed)
