"""Host-side checks of the C ABI (no GPU): the library loads and exports every
function declared in include/*.h; the host index builder's suffix arrays, BWT,
C array, sampled SA and k-mer table (read back through the documented save
format) equal the oracle's independent naive construction; read packing;
argument validation."""
import ctypes
import glob
import os
import re
import struct

import numpy as np
import pytest

import oracle
import paper_1505_07855_gb300 as aln
from synth import Rng, reference_iid, workload

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", src, re.M):
            if not m.group(0).lstrip().startswith(("#", "typedef", "return")):
                names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol():
    L = aln.lib()
    names = _declared_functions()
    assert {"fm_index_build", "fm_index_to_device", "aln_search", "sa_to_pos"} <= names
    for n in sorted(names):
        assert hasattr(L, n), f"{n} declared but not exported"
    assert set(aln._lib.SIGNATURES) == names
    assert L.aln_version() >= 100


def _read_index_file(path):
    """Parse the fm_index_save format: magic, (sa_sample, kmer_k, n_seed), then per
    text (n, primary, C[4]) and three length-prefixed u32 vectors."""
    with open(path, "rb") as f:
        data = f.read()
    assert data[:8] == b"ALNFMIX4"
    off = 8
    sa_sample, kmer_k, n_seed = struct.unpack_from("<3Q", data, off)
    off += 24
    texts = []
    for _ in range(2):
        n, primary, *C = struct.unpack_from("<6Q", data, off)
        off += 48
        vecs = []
        for _v in range(3):
            (sz,) = struct.unpack_from("<Q", data, off)
            off += 8
            vecs.append(np.frombuffer(data, dtype="<u4", count=sz, offset=off).copy())
            off += 4 * sz
        texts.append(dict(n=n, primary=primary, C=C, blocks=vecs[0].reshape(-1, 16), sa=vecs[1],
                          kmer=vecs[2]))
    assert off == len(data)
    return dict(sa_sample=sa_sample, kmer_k=kmer_k, n_seed=n_seed, t=texts)


def _decode_bwt(t):
    """Symbols of the saved blocks: per half of a block (96 rows), 3 words of
    low bits then 3 words of high bits, bit j of word g = the half's symbol
    32 g + j."""
    b = t["blocks"]
    halves = b[:, 4:].reshape(-1, 2, 2, 3)  # block, half, plane, group
    bits = (halves[..., None] >> np.arange(32, dtype=np.uint32)) & 1  # block, half, plane, group, bit
    sym = bits[:, :, 0] | (bits[:, :, 1] << 1)  # block, half, group, bit
    return sym.reshape(-1)[: t["n"] + 1].astype(np.uint8)


@pytest.mark.parametrize("name,n,kmer_k,sample", [("iid", 1, 0, 1), ("iid", 191, 3, 4),
                                                   ("iid", 192, 2, 32), ("iid", 5000, 5, 32),
                                                   ("hp", 3000, 4, 8), ("markov", 200_000, 8, 32)])
def test_host_index_matches_oracle(tmp_path, name, n, kmer_k, sample):
    if name == "iid":
        t = reference_iid(n, Rng(n, "ib"))
    elif name == "hp":  # long exact repeats: needs many doubling rounds
        t = np.tile(np.array([0, 0, 0, 1], np.uint8), n // 4)
        t[::97] = 4
    else:
        t = workload("chr100", ref_len=n, n_reads=1).text
    idx = aln.Index.build(t, n_seed=99, sa_sample=sample, kmer_k=kmer_k, threads=4)
    path = str(tmp_path / "ix.bin")
    idx.save(path)
    f = _read_index_file(path)
    ox = oracle.OracleIndex(t, n_seed=99)
    info = idx.info()
    assert info["n"] == t.size and info["kmer_k"] == kmer_k
    for w in range(2):
        T = f["t"][w]
        sa = ox.sa(w)
        bwt = ox.bwt(w)
        assert T["primary"] == ox.primary(w) == info["primary"][w]
        assert T["C"] == ox.C(w).tolist() == info["C"][w]
        dec = _decode_bwt(T)
        exp = bwt.copy()
        exp[exp == 4] = 0  # $ stored as A
        assert np.array_equal(dec, exp)
        # block counts: occurrences before the block's middle row, $ and the
        # padding after the last row counted as A
        nb = T["blocks"].shape[0]
        padded = np.zeros(nb * 192, np.uint8)
        padded[: exp.size] = exp
        rows = np.arange(nb) * 192 + 96
        cs = np.zeros((padded.size + 1, 4), np.int64)
        for c in range(4):
            cs[1:, c] = np.cumsum(padded == c)
        assert np.array_equal(T["blocks"][:, :4], cs[rows])
        assert np.array_equal(T["sa"], sa[::sample])
        if kmer_k:
            km = T["kmer"].reshape(-1, 2)
            assert km.shape[0] == (4 ** (kmer_k + 1) - 4) // 3
            rng = np.random.default_rng(n + w)
            for j in range(1, kmer_k + 1):
                off = (4 ** j - 4) // 3
                for kid in list(rng.integers(0, 4 ** j, 60)) + [0, 4 ** j - 1]:
                    # processing order: first symbol in the top bits; pattern = reversed
                    q = [(int(kid) >> (2 * (j - 1 - u))) & 3 for u in range(j)]
                    iv = ox.exact(w, np.array(q[::-1], np.uint8))
                    exp_iv = (0, 0) if iv is None else (iv[0], iv[1] + 1)
                    assert tuple(km[off + kid]) == exp_iv
    # load round trip
    idx2 = aln.Index.load(path)
    assert idx2.info() == info
    p2 = str(tmp_path / "ix2.bin")
    idx2.save(p2)
    assert open(p2, "rb").read() == open(path, "rb").read()


def test_load_rejects_bad_files(tmp_path):
    t = reference_iid(1000, Rng(1, "x"))
    idx = aln.Index.build(t)
    p = str(tmp_path / "a.bin")
    idx.save(p)
    data = open(p, "rb").read()
    for bad in (data[:20], data[:-4], b"XXXXXXXX" + data[8:]):
        q = str(tmp_path / "bad.bin")
        open(q, "wb").write(bad)
        with pytest.raises(aln.AlnError) as e:
            aln.Index.load(q)
        assert e.value.status == -6
    with pytest.raises(aln.AlnError):
        aln.Index.load(str(tmp_path / "missing.bin"))


def test_build_argument_errors():
    with pytest.raises(aln.AlnError) as e:
        aln.Index.build(np.zeros(0, np.uint8))
    assert e.value.status == -1
    with pytest.raises(aln.AlnError):
        aln.Index.build(np.zeros(10, np.uint8), sa_sample=3)
    with pytest.raises(aln.AlnError):
        aln.Index.build(np.zeros(10, np.uint8), kmer_k=13)
    L = aln.lib()
    b = aln._lib.aln_batch()
    p = aln.Params().c()
    r = aln._lib.aln_result()
    assert L.aln_search(None, ctypes.byref(b), 1, ctypes.byref(p), ctypes.byref(r), None) == -1
    assert L.sa_to_pos(None, None, 1, 16, None, None, None) == -1
    assert b"null" in L.aln_last_error()
    # the persistent form's caller scratch: 256 bytes of counters + 20 bytes per read,
    # then (from the next 256-byte boundary) a fixed block for the heavy phase
    heavy = L.aln_search_scratch_bytes(0) - 256
    assert heavy > 0
    for n in (1000, 0xFFFFFFFF):
        assert L.aln_search_scratch_bytes(n) == (256 + 20 * n + 255) // 256 * 256 + heavy
    assert L.aln_version() == 200


def test_pack_reads_layout():
    rng = np.random.default_rng(5)
    lens = rng.integers(0, 70, 50).astype(np.uint16)
    codes = rng.integers(0, 5, int(lens.sum())).astype(np.uint8)
    offs = np.zeros(50, np.uint64)
    offs[1:] = np.cumsum(lens[:-1].astype(np.uint64))
    bases, nmask, po = aln.pack_reads(codes, offs, lens)
    j = 0
    for r in range(50):
        assert po[r] == j
        for t in range(int(lens[r])):
            c = int(codes[int(offs[r]) + t])
            isn = (int(nmask[j // 32]) >> (j % 32)) & 1
            b = (int(bases[j // 16]) >> (2 * (j % 16))) & 3
            assert isn == (c == 4)
            if c < 4:
                assert b == c
            j += 1


def test_server_argument_errors():
    L = aln.lib()
    cfg = aln._lib.aln_server_config()
    out = ctypes.c_void_p()
    assert L.aln_server_create(None, ctypes.byref(cfg), ctypes.byref(out)) == -1
    rid = ctypes.c_uint64()
    assert L.aln_server_submit(None, None, None, None, None, 0, ctypes.byref(rid)) == -1
    assert L.aln_server_poll(None, 1, 0, None, None, None) == -1
    L.aln_server_destroy(None)


def _header_macros():
    vals = {}
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for m in re.finditer(r"^#define\s+ALN_(\w+)\s+(.+?)\s*$", src, re.M):
            vals[m.group(1)] = m.group(2)
    return vals


def test_binding_constants_equal_the_header_macros():
    """Every constant of the binding named after a header macro (ALN_X -> X or
    ALN_X) carries the macro's value, so the two cannot drift apart."""
    macros = _header_macros()
    checked = 0
    for name, text in macros.items():
        py_name = name if hasattr(aln._lib, name) else "ALN_" + name
        if not hasattr(aln._lib, py_name):
            continue
        py = getattr(aln._lib, py_name)
        text = text.rstrip("uU")
        if text.startswith("{"):
            assert tuple(int(v) for v in text.strip("{}").split(",")) == tuple(py), name
        elif re.fullmatch(r"\(?-?(0x[0-9A-Fa-f]+|\d+)u?\)?", text):
            assert int(text.strip("()").rstrip("uU"), 0) == py, name
        else:
            continue
        checked += 1
    assert checked >= 20
    assert aln.HEAVY_PASSES == int(macros["HEAVY_PASSES"])
