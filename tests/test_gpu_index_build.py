"""fm_index_build_gpu (the index built on the GPU) gives the host builder's index
image byte for byte: the suffix array is unique and every table of the image is
a function of it.  The host builder is itself checked against the oracle's naive
suffix sort (test_capi_host.py), so equality here ties the GPU builder to the
oracle too; one case also compares the decoded BWT with the oracle's directly."""
import numpy as np
import pytest

import oracle
import paper_1505_07855_gb300 as aln
from synth import Rng, reference_iid, workload
from test_capi_host import _decode_bwt, _read_index_file

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _texts():
    r = Rng(77, "gpu-build")
    t = {}
    for n in (1, 2, 3, 20, 191, 192, 193, 383, 384, 385, 4095, 4096, 4097, 50_000):
        t[f"iid{n}"] = reference_iid(n, r.sub(str(n)))
    t["allA3000"] = np.zeros(3000, np.uint8)                 # deep doubling: one long run
    t["alpha2_9000"] = reference_iid(9000, r.sub("a2")) % 2  # long repeats everywhere
    per = reference_iid(37, r.sub("per"))
    t["periodic"] = np.tile(per, 400)                        # period 37 over 14 800 bases
    nt = reference_iid(30_000, r.sub("n"))
    nt[1000:1600] = 4
    nt[29_990:] = 4
    t["nruns"] = nt
    return t


CASES = [(name, k, s) for name in _texts() for (k, s) in ((0, 32), (5, 4))] + \
        [("iid50000", 10, 1), ("iid50000", 12, 1024), ("nruns", 8, 32)]


@pytest.mark.parametrize("name,kmer_k,sa_sample", CASES)
def test_gpu_build_equals_host_build(cuda, tmp_path, name, kmer_k, sa_sample):
    text = _texts()[name]
    seed = 99 if name == "nruns" else 0
    host = aln.Index.build(text, n_seed=seed, sa_sample=sa_sample, kmer_k=kmer_k)
    gpu = aln.Index.build(text, n_seed=seed, sa_sample=sa_sample, kmer_k=kmer_k, device=0)
    a, b = str(tmp_path / "host.fmi"), str(tmp_path / "gpu.fmi")
    host.save(a)
    gpu.save(b)
    assert open(a, "rb").read() == open(b, "rb").read()


def test_gpu_build_repeat_recipe_against_oracle(cuda, tmp_path):
    """The 3.1 Gbp recipe (repeat families, N runs) at 4 Mbp: the GPU image's BWT,
    C, primary row and sampled SA against the oracle's naive construction, and the
    whole image against the host builder's."""
    w = workload("human_pairs", ref_len=4_000_000, n_reads=10, seed=6)
    gpu = aln.Index.build(w.text, n_seed=5, kmer_k=10, device=0)
    host = aln.Index.build(w.text, n_seed=5, kmer_k=10)
    a, b = str(tmp_path / "host.fmi"), str(tmp_path / "gpu.fmi")
    host.save(a)
    gpu.save(b)
    assert open(a, "rb").read() == open(b, "rb").read()
    img = _read_index_file(b)
    ox = oracle.OracleIndex(w.text, n_seed=5)
    for which in (0, 1):
        t = img["t"][which]
        bwt = ox.bwt(which)
        exp = np.where(bwt == 4, 0, bwt).astype(np.uint8)
        assert np.array_equal(_decode_bwt(t), exp)
        assert t["primary"] == ox.primary(which) and list(t["C"]) == ox.C(which).tolist()
        assert np.array_equal(t["sa"], ox.sa(which)[::32])
