"""Helpers for comparing the CUDA path with the oracle element by element."""
import numpy as np

import oracle
import paper_1505_07855_gb300 as aln

HIT_FIELDS = ("k", "l", "aligned_len", "strand", "n_diff", "n_mm", "n_gapo", "n_gape")
RES_FIELDS = ("c0", "c1", "n_hits", "d_best")


def oracle_align(ox, reads, params: dict, hit_cap, strata, z=None, threads=None, **kw):
    return ox.align(reads.codes, reads.offsets, reads.lens, z if z is not None else None,
                    z_default=params["z"], max_gapo=params["max_gapo"], max_gape=params["max_gape"],
                    seed_len=params["seed_len"], seed_z=params["seed_z"],
                    indel_end_skip=params["indel_end_skip"], hit_cap=hit_cap, strata=strata,
                    threads=threads, **kw)


def compare(res_g, hits_g, res_o, hits_o, idx=None, what=""):
    """Bit-exact comparison; returns the number of reads compared.  GPU results
    must carry no implementation-limit flag."""
    n = res_g.shape[0]
    rows = np.arange(n) if idx is None else np.asarray(idx)
    inc = res_g["flags"] & aln.FLAG_INCOMPLETE
    assert not inc.any(), f"{what}: {int((inc != 0).sum())} reads hit an implementation limit"
    for f in RES_FIELDS:
        g = res_g[f]
        o = res_o[f]
        bad = np.nonzero(g != o)[0]
        assert bad.size == 0, f"{what}: field {f} differs at read {rows[bad[0]]}: gpu {g[bad[0]]} oracle {o[bad[0]]}"
    bad = np.nonzero(res_g["flags"] != res_o["flags"])[0]
    assert bad.size == 0, f"{what}: flags differ at read {rows[bad[0]]}"
    bad = np.nonzero(res_g["best_score"] != res_o["pad"])[0]  # the best score (score-ordered mode; else 0)
    assert bad.size == 0, f"{what}: best score differs at read {rows[bad[0]]}"
    cap = hits_g.shape[1]
    valid = np.arange(cap)[None, :] < res_g["n_hits"][:, None]
    for f in HIT_FIELDS:
        g = np.where(valid, hits_g[f], 0)
        o = np.where(valid, hits_o[f], 0)
        bad = np.argwhere(g != o)
        assert bad.size == 0, (f"{what}: hit field {f} differs at read {rows[bad[0][0]]} hit {bad[0][1]}: "
                               f"gpu {g[tuple(bad[0])]} oracle {o[tuple(bad[0])]}")
    return n
