"""Seeded synthetic inputs (references and reads) shared by the CUDA path's tests
and bench and by the oracle's tests.

This package holds no step of the alignment method: it only draws reference
texts and simulated reads, deterministically per seed, from its own
counter-based generator (SplitMix64).  See ``synth.gen`` and ``synth.workloads``.
"""
from .gen import (  # noqa: F401
    Rng,
    mix64,
    Reads,
    reference_iid,
    reference_markov3,
    overlay_repeats,
    overlay_n_runs,
    simulate_reads,
    simulate_pairs,
    revcomp_codes,
)
from .workloads import workload, WORKLOADS, z_for_length  # noqa: F401
