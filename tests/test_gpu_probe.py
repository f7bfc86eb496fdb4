"""aln_gather_probe, the random 64-byte block-read rate that bounds the LF step
over an index larger than L2 (Sec. 2: every processed base reads index data at
a data-dependent position).  The kernel's checksum is compared with the same
gathers recomputed here from the probe's stated definition (block
b(g) = (lowbias32(g + seed * 0x9E3779B9) * n_blocks) >> 32, XOR of its 16
words), with a ragged gather count; invalid arguments are refused before any
launch."""
import numpy as np
import pytest

import paper_1505_07855_gb300 as aln

pytestmark = pytest.mark.gpu

M32 = np.uint64(0xFFFFFFFF)


def _lowbias32(x):
    x = x.astype(np.uint64) & M32
    x ^= x >> np.uint64(16)
    x = (x * np.uint64(0x7FEB352D)) & M32
    x ^= x >> np.uint64(15)
    x = (x * np.uint64(0x846CA68B)) & M32
    x ^= x >> np.uint64(16)
    return x


def _expected(words: np.ndarray, n_gathers: int, seed: int) -> int:
    n_blocks = words.size // 16
    g = np.arange(n_gathers, dtype=np.uint64)
    salt = (np.uint64(seed) * np.uint64(0x9E3779B9)) & M32
    b = (_lowbias32((g + salt) & M32) * np.uint64(n_blocks)) >> np.uint64(32)
    blk = np.bitwise_xor.reduce(words.reshape(n_blocks, 16), axis=1)
    return int(np.bitwise_xor.reduce(blk[b.astype(np.int64)]))


def _torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.mark.parametrize("n_blocks,n_gathers,seed", [(1, 1, 0), (1000, 100_003, 7), (16384, 1_000_000, 12345)])
def test_probe_checksum(n_blocks, n_gathers, seed):
    torch = _torch()
    rng = np.random.default_rng(n_blocks + seed)
    words = rng.integers(0, 2**32, size=n_blocks * 16, dtype=np.uint64).astype(np.uint32)
    buf = torch.from_numpy(words.view(np.int32)).cuda()
    sink = torch.zeros(1, dtype=torch.int32, device="cuda")
    aln.gather_probe(buf, n_gathers, seed, sink)
    torch.cuda.synchronize()
    got = int(sink.cpu().numpy().view(np.uint32)[0])
    assert got == _expected(words, n_gathers, seed)


def test_probe_zero_gathers_leaves_sink():
    torch = _torch()
    buf = torch.ones(64, dtype=torch.int32, device="cuda")
    sink = torch.full((1,), 5, dtype=torch.int32, device="cuda")
    aln.gather_probe(buf, 0, 1, sink)
    torch.cuda.synchronize()
    assert int(sink.item()) == 5


def test_probe_rejects_bad_arguments():
    torch = _torch()
    buf = torch.zeros(4096, dtype=torch.uint8, device="cuda")
    sink = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(aln.AlnError):  # not 64-byte aligned
        aln.gather_probe(buf[16:], 10, 0, sink)
    with pytest.raises(aln.AlnError):  # host memory
        aln.gather_probe(torch.zeros(4096, dtype=torch.uint8), 10, 0, sink)
    with pytest.raises(aln.AlnError):  # host sink
        aln.gather_probe(buf, 10, 0, torch.zeros(1, dtype=torch.int32))
    with pytest.raises(aln.AlnError):  # smaller than one block
        aln.gather_probe(buf[:32], 10, 0, sink)
    with pytest.raises(aln.AlnError):  # n_gathers out of range
        aln.gather_probe(buf, 1 << 32, 0, sink)
