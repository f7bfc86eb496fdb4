// Device-side index image and the Occ / LF primitives (sm_103a).
//
// Paper Sec. 2: each processed base updates a lower and an upper pointer from
// index data.  Here an interval is half-open [lo, hi) over the n+1 BWT rows
// (the closed interval of the output is [lo, hi-1]); extending by base c gives
//     lo' = C1[c] + occ_before(c, lo),  hi' = C1[c] + occ_before(c, hi),
// with C1[c] = C[c] + 1 and occ_before(c, j) = number of c in B[0 .. j-1].
// It is empty ("the pointers cross") iff hi' <= lo'.
//
// Block layout (64 bytes per 192 rows): cnt[4] = occurrences of A, C, G, T
// before the block's middle row (192 b + 96), $ and end padding counted as A;
// then 12 words of symbols (A=00 C=01 G=10 T=11), 6 for each half of the block:
// the low-bit planes of symbols 0-31, 32-63, 64-95 of the half, then the
// high-bit planes.  A row at offset o in the block counts forwards over symbols
// [96, o) or backwards over [o, 96), inside one half: 3 masks, 9 popcounts.
#pragma once

#include <cstdint>

namespace aln {

constexpr uint32_t kRowsPerBlock = 192;
constexpr uint32_t kHalfRows = 96;

struct DText {
    const uint4 *blocks;     // 4 x uint4 per 64-byte block: counts, then 12 symbol words
    const uint32_t *sa_samp; // SA[r] for r % sa_sample == 0
    const uint2 *kmer;       // (lo, hi) per k-mer, or nullptr
    uint32_t C1[5];          // C[c] + 1; C1[4] = n + 1
    uint32_t primary;        // row of $ (stored as A)
    uint32_t n;              // text length; rows 0..n
};

struct DIndex {
    DText t[2];              // t[0] = X, t[1] = X reversed
    uint32_t kmer_k;
    uint32_t sa_shift;       // log2(sa_sample)
};

__device__ __forceinline__ uint4 ld_nc(const uint4 *p) {
    uint4 v;
    asm volatile("ld.global.nc.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

// The half of a block a row at offset o counts over: the 4 counts and the 6
// symbol words of its half (block words 4..9 below the middle, 10..15 above),
// read as 3 of the block's 4 quads.
struct HalfBlock {
    uint32_t cnt[4];
    uint32_t w[6];
};

__device__ __forceinline__ void load_half(const uint4 *blocks, uint32_t b, uint32_t o, HalfBlock &H) {
    const uint4 *p = blocks + 4ull * b;
    const bool up = o >= kHalfRows;
    const uint4 q0 = ld_nc(p), q2 = ld_nc(p + 2), qx = ld_nc(p + (up ? 3 : 1));
    H.cnt[0] = q0.x; H.cnt[1] = q0.y; H.cnt[2] = q0.z; H.cnt[3] = q0.w;
    if (up) {
        H.w[0] = q2.z; H.w[1] = q2.w; H.w[2] = qx.x; H.w[3] = qx.y; H.w[4] = qx.z; H.w[5] = qx.w;
    } else {
        H.w[0] = qx.x; H.w[1] = qx.y; H.w[2] = qx.z; H.w[3] = qx.w; H.w[4] = q2.x; H.w[5] = q2.y;
    }
}

// Symbols of a half as bit planes: w[g] holds the low bits and w[3 + g] the
// high bits of the half's symbols 32 g .. 32 g + 31 (bit j = symbol 32 g + j).
// Counting symbols before (or from) position x of the half needs one mask per
// 32 symbols, shared by both planes.
__device__ __forceinline__ void occ4_in_half(const HalfBlock &H, uint32_t o, uint32_t occ[4]) {
    const bool up = o >= kHalfRows;
    const int x = static_cast<int>(up ? o - kHalfRows : o);
    uint32_t nlo = 0, nhi = 0, nboth = 0;
#pragma unroll
    for (int g = 0; g < 3; g++) {
        const int k = max(x - 32 * g, 0);
        uint32_t m = __funnelshift_lc(0xFFFFFFFFu, 0u, static_cast<uint32_t>(k));  // low min(k, 32) bits
        if (!up) m = ~m;  // backwards: symbols at or after o
        const uint32_t l = H.w[g] & m, h = H.w[3 + g] & m;
        nlo += __popc(l);
        nhi += __popc(h);
        nboth += __popc(l & h);
    }
    const uint32_t nsym = up ? static_cast<uint32_t>(x) : kHalfRows - static_cast<uint32_t>(x);
    const uint32_t cT = nboth, cG = nhi - nboth, cC = nlo - nboth;
    const uint32_t cA = nsym - cT - cG - cC;
    if (up) {
        occ[0] = H.cnt[0] + cA; occ[1] = H.cnt[1] + cC; occ[2] = H.cnt[2] + cG; occ[3] = H.cnt[3] + cT;
    } else {
        occ[0] = H.cnt[0] - cA; occ[1] = H.cnt[1] - cC; occ[2] = H.cnt[2] - cG; occ[3] = H.cnt[3] - cT;
    }
}

// The symbol at offset o of the block, from its half.
__device__ __forceinline__ uint32_t sym_in_half(const HalfBlock &H, uint32_t o) {
    const uint32_t x = o >= kHalfRows ? o - kHalfRows : o;
    const uint32_t g = x >> 5, j = x & 31u;
    const uint32_t l = g == 0 ? H.w[0] : (g == 1 ? H.w[1] : H.w[2]);
    const uint32_t h = g == 0 ? H.w[3] : (g == 1 ? H.w[4] : H.w[5]);
    return ((l >> j) & 1u) | (((h >> j) & 1u) << 1);
}

// Extend [lo, hi) by every base: children (lo4[c], hi4[c]).  Both half-block
// reads are issued before either is used (a second read of the same half is an
// L1 hit).
__device__ __forceinline__ void lf4(const DText &T, uint32_t lo, uint32_t hi, uint32_t lo4[4], uint32_t hi4[4]) {
    if (lo == 0 && hi == T.n + 1) {  // the empty string: children are the C ranges
#pragma unroll
        for (int c = 0; c < 4; c++) {
            lo4[c] = T.C1[c];
            hi4[c] = T.C1[c + 1];
        }
        return;
    }
    const uint32_t blo = lo / kRowsPerBlock, bhi = hi / kRowsPerBlock;
    const uint32_t ol = lo - blo * kRowsPerBlock, oh = hi - bhi * kRowsPerBlock;
    HalfBlock Hl, Hh;
    load_half(T.blocks, blo, ol, Hl);  // both reads issued before either is used
    load_half(T.blocks, bhi, oh, Hh);
    uint32_t olo[4], ohi[4];
    occ4_in_half(Hl, ol, olo);
    occ4_in_half(Hh, oh, ohi);
    olo[0] -= (lo > T.primary) ? 1u : 0u;
    ohi[0] -= (hi > T.primary) ? 1u : 0u;
#pragma unroll
    for (int c = 0; c < 4; c++) {
        lo4[c] = T.C1[c] + olo[c];
        hi4[c] = T.C1[c] + ohi[c];
    }
}

// Extend [lo, hi) by base c.
__device__ __forceinline__ void lf1(const DText &T, uint32_t c, uint32_t &lo, uint32_t &hi) {
    uint32_t lo4[4], hi4[4];
    lf4(T, lo, hi, lo4, hi4);
    lo = lo4[c];
    hi = hi4[c];
}

// LF(r) = C1[B[r]] + occ_before(B[r], r) for a row r != primary: the row of the
// suffix that starts one text position earlier.
__device__ __forceinline__ uint32_t lf_row(const DText &T, uint32_t r) {
    const uint32_t b = r / kRowsPerBlock, o = r - b * kRowsPerBlock;
    HalfBlock H;
    load_half(T.blocks, b, o, H);
    const uint32_t c = sym_in_half(H, o);
    uint32_t occ[4];
    occ4_in_half(H, o, occ);
    uint32_t v = occ[c];
    if (c == 0) v -= (r > T.primary) ? 1u : 0u;
    return T.C1[c] + v;
}

}  // namespace aln
