"""Deterministic generators for synthetic DNA references and reads.

Randomness comes only from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used counter-style: output
``i`` of stream ``key`` is ``mix64(key + (i + 1) * GOLDEN)``.  Everything is
computed in uint64 / integer arithmetic or in float64 comparisons of exact
dyadic values, so the same seed gives the same bytes on x86-64 and AArch64.

Base codes: A=0, C=1, G=2, T=3, N=4.
"""
from __future__ import annotations

import dataclasses
import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_U30, _U27, _U31 = np.uint64(30), np.uint64(27), np.uint64(31)


def mix64(z):
    """SplitMix64 output function applied to state ``z + GOLDEN`` (uint64 array or int)."""
    scalar = np.isscalar(z) or isinstance(z, int)
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = z + GOLDEN
        z = (z ^ (z >> _U30)) * _M1
        z = (z ^ (z >> _U27)) * _M2
        z = z ^ (z >> _U31)
    return int(z) if scalar else z


def _fnv1a64(name: str) -> int:
    h = 0xCBF29CE484222325
    for ch in name.encode():
        h ^= ch
        h = (h * 0x100000001B3) & 0xFFFFFFFFFFFFFFFF
    return h


class Rng:
    """Counter-based SplitMix64 streams keyed by (seed, name)."""

    def __init__(self, seed: int, name: str = ""):
        self.key = mix64(np.uint64((seed & 0xFFFFFFFFFFFFFFFF) ^ _fnv1a64(name)))

    def sub(self, name: str) -> "Rng":
        r = Rng.__new__(Rng)
        r.key = mix64(np.uint64(self.key ^ _fnv1a64(name)))
        return r

    def u64_at(self, idx) -> np.ndarray:
        idx = np.asarray(idx, dtype=np.uint64)
        with np.errstate(over="ignore"):
            return mix64(np.uint64(self.key) + (idx + np.uint64(1)) * GOLDEN)

    def u64(self, n: int, start: int = 0) -> np.ndarray:
        return self.u64_at(np.arange(start, start + n, dtype=np.uint64))

    @staticmethod
    def to_unit(u: np.ndarray) -> np.ndarray:
        """uint64 -> float64 in [0, 1) using the top 53 bits (exact)."""
        return (u >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)

    @staticmethod
    def to_below(u: np.ndarray, bound) -> np.ndarray:
        """uint64 -> integer in [0, bound) by the multiply-shift (Lemire) map on the top 32 bits."""
        hi = (u >> np.uint64(32)).astype(np.uint64)
        return ((hi * np.asarray(bound, dtype=np.uint64)) >> np.uint64(32)).astype(np.int64)


def revcomp_codes(codes: np.ndarray) -> np.ndarray:
    """Reverse complement of a code array; N (4) stays N."""
    r = codes[::-1].copy()
    m = r < 4
    r[m] = 3 - r[m]
    return r


# --------------------------------------------------------------------------- references


def reference_iid(n: int, rng: Rng, chunk: int = 1 << 26) -> np.ndarray:
    """Uniform i.i.d. ACGT text of length n (32 bases per 64-bit draw)."""
    out = np.empty(n, dtype=np.uint8)
    shifts = (np.arange(32, dtype=np.uint64) * np.uint64(2))
    words_per_chunk = chunk // 32
    pos = 0
    w = 0
    while pos < n:
        cnt = min(words_per_chunk, (n - pos + 31) // 32)
        u = rng.u64(cnt, start=w)
        b = ((u[:, None] >> shifts[None, :]) & np.uint64(3)).astype(np.uint8).reshape(-1)
        take = min(n - pos, b.size)
        out[pos:pos + take] = b[:take]
        pos += take
        w += cnt
    return out


def _markov3_table(rng: Rng, gc: float):
    """Order-3 transition table: composition (A=T=(1-gc)/2, C=G=gc/2) perturbed by
    seeded factors in [0.8, 1.2] per (context, base) and renormalised per context."""
    base_p = np.array([(1 - gc) / 2, gc / 2, gc / 2, (1 - gc) / 2])
    f = 0.8 + 0.4 * Rng.to_unit(rng.u64(256)).reshape(64, 4)
    t = base_p[None, :] * f
    return t / t.sum(axis=1, keepdims=True)


def _stationary_gc(t: np.ndarray) -> float:
    # 64-state chain over contexts (b0 b1 b2) -> (b1 b2 b3)
    P = np.zeros((64, 64))
    for ctx in range(64):
        for b in range(4):
            P[ctx, ((ctx << 2) | b) & 63] += t[ctx, b]
    pi = np.full(64, 1 / 64)
    for _ in range(2000):
        pi = pi @ P
    pi /= pi.sum()
    p_next = pi @ t
    return float(p_next[1] + p_next[2])


def reference_markov3(n: int, rng: Rng, gc: float = 0.41, gc_window=(0.405, 0.415),
                      segment: int = 8192) -> np.ndarray:
    """Order-3 Markov text.  The table is redrawn (new sub-seed) until its stationary
    GC and the realised GC both fall inside ``gc_window``.  The text is generated as
    independent chains of ``segment`` bases (each started from a composition-drawn
    3-base context) so that the generation vectorises over segments."""
    for attempt in range(1000):
        r = rng.sub(f"table{attempt}")
        t = _markov3_table(r, gc)
        if not (gc_window[0] <= _stationary_gc(t) <= gc_window[1]):
            continue
        cum = np.cumsum(t, axis=1)
        cum[:, 3] = 1.0
        nseg = (n + segment - 1) // segment
        draws = r.sub("walk")
        out = np.empty((nseg, segment), dtype=np.uint8)
        base_cum = np.cumsum([(1 - gc) / 2, gc / 2, gc / 2, (1 - gc) / 2])
        seg_idx = np.arange(nseg, dtype=np.uint64)
        ctx = np.zeros(nseg, dtype=np.int64)
        for j in range(3):  # initial context
            u = Rng.to_unit(draws.u64_at(seg_idx * np.uint64(segment + 3) + np.uint64(j)))
            b = np.searchsorted(base_cum, u, side="right").clip(0, 3)
            ctx = ((ctx << 2) | b) & 63
        for j in range(segment):
            u = Rng.to_unit(draws.u64_at(seg_idx * np.uint64(segment + 3) + np.uint64(3 + j)))
            c = cum[ctx]
            b = (u[:, None] >= c).sum(axis=1).clip(0, 3)
            out[:, j] = b
            ctx = ((ctx << 2) | b) & 63
        text = out.reshape(-1)[:n].copy()
        real_gc = float(np.isin(text, (1, 2)).mean())
        if gc_window[0] <= real_gc <= gc_window[1]:
            return text
    raise RuntimeError("no Markov table met the GC window")


def overlay_repeats(text: np.ndarray, rng: Rng, frac: float, n_families: int,
                    len_range=(300, 6000), div_range=(0.02, 0.15),
                    family_source=None) -> dict:
    """Overwrite about ``frac`` of ``text`` with diverged copies of ``n_families``
    random families.  Each copy is a whole family sequence, given substitutions at a
    per-copy rate uniform in ``div_range`` and a random orientation, written at a
    uniform position.  Returns summary statistics."""
    n = text.size
    fr = rng.sub("families")
    lens = len_range[0] + Rng.to_below(fr.u64(n_families), len_range[1] - len_range[0] + 1)
    fams = []
    for f in range(n_families):
        if family_source is None:
            fams.append(reference_iid(int(lens[f]), fr.sub(f"fam{f}")))
        else:
            fams.append(family_source(int(lens[f]), fr.sub(f"fam{f}")))
    target = int(frac * n)
    cr = rng.sub("copies")
    covered = 0
    copies = 0
    while covered < target:
        u = cr.u64(4, start=copies * 4)
        f = int(Rng.to_below(u[0:1], n_families)[0])
        L = fams[f].size
        if L >= n:
            break
        pos = int(Rng.to_below(u[1:2], n - L + 1)[0])
        div = div_range[0] + (div_range[1] - div_range[0]) * float(Rng.to_unit(u[2:3])[0])
        seq = fams[f].copy()
        if int(u[3]) & 1:
            seq = revcomp_codes(seq)
        er = cr.sub(f"copy{copies}")
        e = er.u64(2 * L)
        hit = Rng.to_unit(e[:L]) < div
        seq[hit] = (seq[hit] + 1 + Rng.to_below(e[L:][hit], 3)) & 3
        text[pos:pos + L] = seq
        covered += L
        copies += 1
    return {"copies": copies, "covered": covered, "families": n_families}


def overlay_n_runs(text: np.ndarray, rng: Rng, frac: float, run_range=(100, 10000)) -> np.ndarray:
    """Write runs of N (code 4) of uniform length in ``run_range`` at uniform positions
    until about ``frac`` of the text is N.  Returns the boolean N mask."""
    n = text.size
    target = int(frac * n)
    covered = 0
    i = 0
    while covered < target:
        u = rng.u64(2, start=2 * i)
        L = int(run_range[0] + Rng.to_below(u[0:1], run_range[1] - run_range[0] + 1)[0])
        pos = int(Rng.to_below(u[1:2], max(1, n - L))[0])
        text[pos:pos + L] = 4
        covered += L
        i += 1
    return text == 4


# --------------------------------------------------------------------------- reads


@dataclasses.dataclass
class Reads:
    """A batch of reads as concatenated base codes (0..4) with per-read offsets."""
    codes: np.ndarray      # uint8, all reads back to back
    offsets: np.ndarray    # uint64, start of each read in ``codes``
    lens: np.ndarray       # uint16
    z: np.ndarray          # uint8, per-read difference limit
    true_pos: np.ndarray   # int64, forward-strand start of the origin
    true_strand: np.ndarray  # uint8, 0 = forward, 1 = reverse complement

    @property
    def n(self) -> int:
        return int(self.lens.size)

    def read(self, i: int) -> np.ndarray:
        o = int(self.offsets[i])
        return self.codes[o:o + int(self.lens[i])]

    def subset(self, idx) -> "Reads":
        idx = np.asarray(idx, dtype=np.int64)
        parts = [self.read(int(i)) for i in idx]
        lens = self.lens[idx].copy()
        offs = np.zeros(idx.size, dtype=np.uint64)
        if idx.size:
            offs[1:] = np.cumsum(lens[:-1].astype(np.uint64))
        codes = np.concatenate(parts) if parts else np.zeros(0, np.uint8)
        return Reads(codes.astype(np.uint8), offs, lens, self.z[idx].copy(),
                     self.true_pos[idx].copy(), self.true_strand[idx].copy())

    @staticmethod
    def concat(items) -> "Reads":
        items = list(items)
        lens = np.concatenate([r.lens for r in items])
        offs = np.zeros(lens.size, dtype=np.uint64)
        if lens.size:
            offs[1:] = np.cumsum(lens[:-1].astype(np.uint64))
        codes = np.concatenate([np.concatenate([r.read(i) for i in range(r.n)]) if r.n else
                                np.zeros(0, np.uint8) for r in items])
        return Reads(codes, offs, lens, np.concatenate([r.z for r in items]),
                     np.concatenate([r.true_pos for r in items]),
                     np.concatenate([r.true_strand for r in items]))


def _mask_prefix(nmask):
    """Prefix counts of an N mask (uint32: texts are < 2^32 bases)."""
    if nmask is None:
        return None
    cs = np.zeros(nmask.size + 1, dtype=np.uint32)
    np.cumsum(nmask, out=cs[1:], dtype=np.uint32)
    return cs


def _clean_starts(rng: Rng, n_reads: int, lens: np.ndarray, pad: int, n: int, nmask_cs) -> np.ndarray:
    """Uniform anchors s0 in [pad, n - len - pad] whose padded span
    [s0 - pad, s0 + len + pad) avoids N runs (resampled with fresh counters)."""
    lo = pad
    width = np.maximum(1, n - lens - 2 * pad + 1)
    starts = lo + Rng.to_below(rng.u64(n_reads), width)
    if nmask_cs is None:
        return starts
    def bad_of(s, L):
        hi = nmask_cs[np.minimum(n, s + L + pad)].astype(np.int64)
        return (hi - nmask_cs[np.maximum(0, s - pad)].astype(np.int64)) > 0
    bad = bad_of(starts, lens)
    attempt = 1
    while bad.any():
        idx = np.nonzero(bad)[0]
        u = rng.sub(f"retry{attempt}").u64_at(idx.astype(np.uint64))
        starts[idx] = lo + Rng.to_below(u, width[idx])
        bad[idx] = bad_of(starts[idx], lens[idx])
        attempt += 1
        if attempt > 1000:
            raise RuntimeError("could not place reads outside N runs")
    return starts


def simulate_reads(ref: np.ndarray, n_reads: int, lengths, rng: Rng, *,
                   sub_rate=(0.01, 0.01), indel_rate=0.0005, indel_lens=(1,),
                   n_frac=0.02, z_of_len=None, z=2, strands="both",
                   nmask: np.ndarray | None = None, starts=None, rev=None,
                   chunk: int = 1 << 16) -> Reads:
    """Simulate single-end reads.

    * Each read has an anchor s0: a forward read copies the text rightwards from s0;
      a reverse read copies the reverse complement leftwards from s0 + len - 1.
      Anchors are uniform over positions whose padded span avoids N runs (unless
      ``starts``/``rev`` are given); the strand is 50/50 (``strands="both"``).
    * Per read position j (5'->3'): an indel event with probability ``indel_rate``
      (insertion or deletion, equal odds, length uniform from ``indel_lens``), then a
      substitution with probability rising linearly from ``sub_rate[0]`` at the 5'
      end to ``sub_rate[1]`` at the 3' end.
    * With probability ``n_frac`` one uniform position becomes N.
    ``lengths`` is an int or an array of allowed lengths drawn uniformly.
    ``true_pos`` is the leftmost text position the read's bases were copied from.
    """
    n = ref.size
    if np.isscalar(lengths):
        lens = np.full(n_reads, int(lengths), dtype=np.int64)
    else:
        choices = np.asarray(lengths, dtype=np.int64)
        lens = choices[Rng.to_below(rng.sub("len").u64(n_reads), choices.size)]
    max_indel = max(indel_lens) if indel_rate > 0 else 0
    pad = 4 * max_indel + 8
    if starts is None:
        nmask_cs = _mask_prefix(nmask)
        starts = _clean_starts(rng.sub("start"), n_reads, lens, pad, n, nmask_cs)
    starts = np.asarray(starts, dtype=np.int64)
    if rev is None:
        if strands == "both":
            rev = (rng.sub("strand").u64(n_reads) & np.uint64(1)).astype(np.uint8)
        else:
            rev = np.full(n_reads, 1 if strands == "rev" else 0, dtype=np.uint8)
    rev = np.asarray(rev, dtype=np.uint8)

    offs = np.zeros(n_reads, dtype=np.uint64)
    if n_reads:
        offs[1:] = np.cumsum(lens[:-1].astype(np.uint64))
    codes = np.zeros(int(lens.sum()), dtype=np.uint8)
    true_pos = np.zeros(n_reads, dtype=np.int64)

    er_sub, er_val = rng.sub("subst"), rng.sub("substval")
    er_indel, er_n = rng.sub("indel"), rng.sub("nbase")
    maxlen = int(lens.max()) if n_reads else 0
    CTR = np.uint64(1024)  # counters reserved per read for per-base draws
    jj = np.arange(maxlen, dtype=np.int64)
    for c0 in range(0, n_reads, chunk):
        c1 = min(n_reads, c0 + chunk)
        rid = np.arange(c0, c1, dtype=np.uint64)
        ctr = rid[:, None] * CTR + jj[None, :].astype(np.uint64)
        L = lens[c0:c1]
        valid = jj[None, :] < L[:, None]
        st = starts[c0:c1]
        rv = rev[c0:c1]
        has_indel = np.zeros(c1 - c0, dtype=bool)
        ind_u = None
        if indel_rate > 0:
            ind_u = Rng.to_unit(er_indel.u64_at(ctr))
            has_indel = ((ind_u < indel_rate) & valid).any(axis=1)
        anchor = st + L - 1
        pos = np.where(rv[:, None] == 1, anchor[:, None] - jj[None, :], st[:, None] + jj[None, :])
        pos = np.clip(pos, 0, n - 1)
        win = ref[pos]
        comp = np.where(win < 4, 3 - win.astype(np.int16), 4).astype(np.uint8)  # N stays N
        win = np.where(rv[:, None] == 1, comp, win).astype(np.uint8)
        tp = st.copy()
        for r in np.nonzero(has_indel)[0]:
            gi = c0 + int(r)
            Lr = int(L[r])
            ev = np.nonzero(ind_u[r, :Lr] < indel_rate)[0]
            evu = er_indel.sub("kind").u64_at(np.uint64(gi) * CTR + ev.astype(np.uint64))
            kinds = (evu & np.uint64(1)).astype(np.int64)
            elen = np.asarray(indel_lens, dtype=np.int64)[Rng.to_below(evu, len(indel_lens))]
            ins_u = er_indel.sub("insbase").u64(64, start=gi * 64)
            events = {int(j): (int(k), int(l)) for j, k, l in zip(ev, kinds, elen)}
            out = []
            p = 0
            j = 0
            k_ins = 0
            s0 = int(st[r])
            a0 = int(anchor[r])
            while len(out) < Lr:
                if j in events:
                    kind, ln = events[j]
                    if kind == 0:
                        for _ in range(ln):
                            out.append(int(ins_u[k_ins % 64] >> np.uint64(8)) & 3)
                            k_ins += 1
                    else:
                        p += ln
                if len(out) >= Lr:
                    break
                if rv[r]:
                    b = int(ref[a0 - p])
                    out.append(3 - b if b < 4 else 4)
                else:
                    out.append(int(ref[s0 + p]))
                p += 1
                j += 1
            win[r, :Lr] = np.asarray(out[:Lr], dtype=np.uint8)
            tp[r] = (a0 - p + 1) if rv[r] else s0
        frac = jj[None, :].astype(np.float64) / np.maximum(1, (L[:, None] - 1))
        rate = sub_rate[0] + (sub_rate[1] - sub_rate[0]) * frac
        hit = (Rng.to_unit(er_sub.u64_at(ctr)) < rate) & valid
        sv = Rng.to_below(er_val.u64_at(ctr), 3).astype(np.uint8)
        win = np.where(hit, (win + 1 + sv) & 3, win).astype(np.uint8)
        gets_n = Rng.to_unit(er_n.u64_at(rid)) < n_frac
        npos = Rng.to_below(er_n.sub("pos").u64_at(rid), L)
        rows = np.nonzero(gets_n)[0]
        win[rows, npos[rows]] = 4
        flat_idx = offs[c0:c1][:, None].astype(np.int64) + jj[None, :]
        codes[flat_idx[valid]] = win[valid]
        true_pos[c0:c1] = tp
    if z_of_len is not None:
        zz = np.asarray([z_of_len(int(x)) for x in range(maxlen + 1)], dtype=np.uint8)[lens]
    else:
        zz = np.full(n_reads, z, dtype=np.uint8)
    return Reads(codes, offs, lens.astype(np.uint16), zz, true_pos, rev)


def simulate_pairs(ref: np.ndarray, n_pairs: int, length: int, rng: Rng, *,
                   frag_mean=500, frag_sd=50, frag_min=200, chimeric=0.001,
                   nmask=None, **kw) -> tuple[Reads, Reads]:
    """Paired reads.  Fragment length = mean + sd * Z rounded, where Z is the
    Irwin-Hall sum of 12 16-bit integer uniforms, centred and scaled in exact
    integer arithmetic; clamped >= max(frag_min, length).  Mate 1 is the forward read
    at the fragment start and mate 2 the reverse-complement read at its end; a random
    half of the fragments swap the two (opposite orientation).  A fraction
    ``chimeric`` of pairs take mate 2 from an unrelated uniform locus."""
    n = ref.size
    u = (rng.sub("frag").u64(12 * n_pairs).reshape(n_pairs, 12) >> np.uint64(48)).astype(np.int64)
    s = u.sum(axis=1)
    num = (2 * s - 12 * 65535) * frag_sd          # = 2 * 65536 * sd * Z
    frag = frag_mean + np.floor_divide(num + 65536, 2 * 65536)
    frag = np.maximum(frag, max(frag_min, length))
    max_indel = max(kw.get("indel_lens", (1,))) if kw.get("indel_rate", 0.0005) > 0 else 0
    pad = 4 * max_indel + 8
    nmask_cs = _mask_prefix(nmask)
    fstart = _clean_starts(rng.sub("fstart"), n_pairs, frag, pad, n, nmask_cs)
    flip = (rng.sub("forient").u64(n_pairs) & np.uint64(1)).astype(bool)
    chim = Rng.to_unit(rng.sub("chim").u64(n_pairs)) < chimeric
    cstart = _clean_starts(rng.sub("cstart"), n_pairs, np.full(n_pairs, length), pad, n, nmask_cs)
    cstrand = (rng.sub("cstrand").u64(n_pairs) & np.uint64(1)).astype(np.uint8)
    head = fstart
    tail = fstart + frag - length
    s1 = np.where(flip, tail, head)
    r1 = np.where(flip, 1, 0).astype(np.uint8)
    s2 = np.where(flip, head, tail)
    r2 = np.where(flip, 0, 1).astype(np.uint8)
    s2 = np.where(chim, cstart, s2)
    r2 = np.where(chim, cstrand, r2).astype(np.uint8)
    m1 = simulate_reads(ref, n_pairs, length, rng.sub("mate1"), starts=s1, rev=r1, **kw)
    m2 = simulate_reads(ref, n_pairs, length, rng.sub("mate2"), starts=s2, rev=r2, **kw)
    return m1, m2
