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
// then 12 words of 2-bit symbols (A=00 C=01 G=10 T=11), 16 per word.  A row at
// offset o in the block counts forwards over symbols [96, o) or backwards over
// [o, 96): at most 6 words, merged two words per popcount.
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

struct Block {
    uint32_t cnt[4];
    uint32_t w[12];
};

__device__ __forceinline__ uint4 ld_nc(const uint4 *p) {
    uint4 v;
    asm volatile("ld.global.nc.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

__device__ __forceinline__ void load_block(const uint4 *blocks, uint32_t b, Block &B) {
    const uint4 *p = blocks + 4ull * b;
    uint4 q0 = ld_nc(p), q1 = ld_nc(p + 1), q2 = ld_nc(p + 2), q3 = ld_nc(p + 3);
    B.cnt[0] = q0.x; B.cnt[1] = q0.y; B.cnt[2] = q0.z; B.cnt[3] = q0.w;
    B.w[0] = q1.x; B.w[1] = q1.y; B.w[2] = q1.z; B.w[3] = q1.w;
    B.w[4] = q2.x; B.w[5] = q2.y; B.w[6] = q2.z; B.w[7] = q2.w;
    B.w[8] = q3.x; B.w[9] = q3.y; B.w[10] = q3.z; B.w[11] = q3.w;
}

// Mask of the low k symbols (k = 0..16) of a word, lo bit of each symbol only.
__device__ __forceinline__ uint32_t sym_mask(int k) {
    k = k < 0 ? 0 : (k > 16 ? 16 : k);
    return __funnelshift_lc(0xFFFFFFFFu, 0u, 2u * static_cast<uint32_t>(k)) & 0x55555555u;
}

// The half of a block a row at offset o counts over: the 4 counts and the 6
// symbol words of its half (words 0..5 backwards from the middle, 6..11
// forwards), read as 3 of the block's 4 quads.
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

// occ_before(c, 192 b + o) from the row's half block (before the $ correction).
__device__ __forceinline__ void occ4_in_half(const HalfBlock &H, uint32_t o, uint32_t occ[4]) {
    const bool up = o >= kHalfRows;
    const int x = static_cast<int>(up ? o - kHalfRows : o);
    uint32_t nlo = 0, nhi = 0, nboth = 0;
#pragma unroll
    for (int pr = 0; pr < 3; pr++) {
        const uint32_t wa = H.w[2 * pr], wb = H.w[2 * pr + 1];
        uint32_t ma = sym_mask(x - 32 * pr), mb = sym_mask(x - 32 * pr - 16);
        if (!up) {
            ma ^= 0x55555555u;
            mb ^= 0x55555555u;
        }
        const uint32_t la = wa & ma, ha = (wa >> 1) & ma;
        const uint32_t lb = wb & mb, hb = (wb >> 1) & mb;
        nlo += __popc(la | (lb << 1));
        nhi += __popc(ha | (hb << 1));
        nboth += __popc((la & ha) | ((lb & hb) << 1));
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

// occ_before(c, 192 b + o) for all four bases (before the $ correction).
__device__ __forceinline__ void occ4_in_block(const Block &B, uint32_t o, uint32_t occ[4]) {
    const bool up = o >= kHalfRows;
    const int x = static_cast<int>(up ? o - kHalfRows : o);
    uint32_t nlo = 0, nhi = 0, nboth = 0;
#pragma unroll
    for (int pr = 0; pr < 3; pr++) {
        const uint32_t wa = up ? B.w[6 + 2 * pr] : B.w[2 * pr];
        const uint32_t wb = up ? B.w[7 + 2 * pr] : B.w[2 * pr + 1];
        uint32_t ma = sym_mask(x - 32 * pr), mb = sym_mask(x - 32 * pr - 16);
        if (!up) {  // backwards: symbols at or after o
            ma ^= 0x55555555u;
            mb ^= 0x55555555u;
        }
        const uint32_t la = wa & ma, ha = (wa >> 1) & ma;
        const uint32_t lb = wb & mb, hb = (wb >> 1) & mb;
        nlo += __popc(la | (lb << 1));
        nhi += __popc(ha | (hb << 1));
        nboth += __popc((la & ha) | ((lb & hb) << 1));
    }
    const uint32_t nsym = up ? static_cast<uint32_t>(x) : kHalfRows - static_cast<uint32_t>(x);
    const uint32_t cT = nboth, cG = nhi - nboth, cC = nlo - nboth;
    const uint32_t cA = nsym - cT - cG - cC;
    if (up) {
        occ[0] = B.cnt[0] + cA; occ[1] = B.cnt[1] + cC; occ[2] = B.cnt[2] + cG; occ[3] = B.cnt[3] + cT;
    } else {
        occ[0] = B.cnt[0] - cA; occ[1] = B.cnt[1] - cC; occ[2] = B.cnt[2] - cG; occ[3] = B.cnt[3] - cT;
    }
}

// Extend [lo, hi) by every base: children (lo4[c], hi4[c]).  Both block reads
// are issued before either is used; a second read of the same block is skipped.
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
    Block B;
    load_block(T.blocks, b, B);
    const uint32_t c = (B.w[o >> 4] >> (2 * (o & 15u))) & 3u;
    uint32_t occ[4];
    occ4_in_block(B, o, occ);
    uint32_t v = occ[c];
    if (c == 0) v -= (r > T.primary) ? 1u : 0u;
    return T.C1[c] + v;
}

}  // namespace aln
