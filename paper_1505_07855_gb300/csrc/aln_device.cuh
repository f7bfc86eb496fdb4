// Device-side index image and the Occ / LF primitives (sm_103a).
//
// Paper Sec. 2: each processed base updates a lower and an upper pointer from
// index data.  Here an interval is half-open [lo, hi) over the n+1 BWT rows
// (the closed interval of the output is [lo, hi-1]); extending by base c gives
//     lo' = C1[c] + occ_before(c, lo),  hi' = C1[c] + occ_before(c, hi),
// with C1[c] = C[c] + 1 and occ_before(c, j) = number of c in B[0 .. j-1].
// It is empty ("the pointers cross") iff hi' <= lo'.
#pragma once

#include <cstdint>

namespace aln {

constexpr uint32_t kRowsPerBlock = 192;

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

// Counts of A, C, G, T among the first r (0..191) symbols of a block.
// Symbol bits (hi, lo): A=00 C=01 G=10 T=11.
__device__ __forceinline__ void count4_prefix(const Block &B, uint32_t r, uint32_t out[4]) {
    const uint32_t full = r >> 4, rem = r & 15u;
    uint32_t nlo = 0, nhi = 0, nboth = 0;
#pragma unroll
    for (uint32_t t = 0; t < 12; t++) {
        uint32_t m = (t < full) ? 0x55555555u : ((t == full) ? (((1u << (2 * rem)) - 1u) & 0x55555555u) : 0u);
        uint32_t lo = B.w[t] & m, hi = (B.w[t] >> 1) & m;
        nlo += __popc(lo);
        nhi += __popc(hi);
        nboth += __popc(lo & hi);
    }
    out[3] = nboth;
    out[2] = nhi - nboth;
    out[1] = nlo - nboth;
    out[0] = r - out[1] - out[2] - out[3];
}

// Count of symbol c among the first r symbols of a block.
__device__ __forceinline__ uint32_t count1_prefix(const Block &B, uint32_t r, uint32_t c) {
    const uint32_t full = r >> 4, rem = r & 15u;
    const uint32_t pat = c * 0x55555555u;  // c replicated in every 2-bit lane
    uint32_t n = 0;
#pragma unroll
    for (uint32_t t = 0; t < 12; t++) {
        uint32_t m = (t < full) ? 0x55555555u : ((t == full) ? (((1u << (2 * rem)) - 1u) & 0x55555555u) : 0u);
        uint32_t x = B.w[t] ^ pat;
        n += __popc(~(x | (x >> 1)) & m);
    }
    return n;
}

// occ_before for all four symbols at rows lo and hi (one or two block reads).
__device__ __forceinline__ void occ4_pair(const DText &T, uint32_t lo, uint32_t hi, uint32_t olo[4],
                                          uint32_t ohi[4]) {
    const uint32_t blo = lo / kRowsPerBlock, bhi = hi / kRowsPerBlock;
    Block Bl, Bh;
    load_block(T.blocks, blo, Bl);
    if (bhi != blo) load_block(T.blocks, bhi, Bh);
    count4_prefix(Bl, lo - blo * kRowsPerBlock, olo);
    if (bhi != blo) {
        count4_prefix(Bh, hi - bhi * kRowsPerBlock, ohi);
#pragma unroll
        for (int c = 0; c < 4; c++) ohi[c] += Bh.cnt[c];
    } else {
        count4_prefix(Bl, hi - blo * kRowsPerBlock, ohi);
#pragma unroll
        for (int c = 0; c < 4; c++) ohi[c] += Bl.cnt[c];
    }
#pragma unroll
    for (int c = 0; c < 4; c++) olo[c] += Bl.cnt[c];
    olo[0] -= (lo > T.primary) ? 1u : 0u;
    ohi[0] -= (hi > T.primary) ? 1u : 0u;
}

// Extend [lo, hi) by every base: children (lo4[c], hi4[c]).
__device__ __forceinline__ void lf4(const DText &T, uint32_t lo, uint32_t hi, uint32_t lo4[4], uint32_t hi4[4]) {
    if (lo == 0 && hi == T.n + 1) {  // the empty string: children are the C ranges
#pragma unroll
        for (int c = 0; c < 4; c++) {
            lo4[c] = T.C1[c];
            hi4[c] = T.C1[c + 1];
        }
        return;
    }
    uint32_t olo[4], ohi[4];
    occ4_pair(T, lo, hi, olo, ohi);
#pragma unroll
    for (int c = 0; c < 4; c++) {
        lo4[c] = T.C1[c] + olo[c];
        hi4[c] = T.C1[c] + ohi[c];
    }
}

// Extend [lo, hi) by base c.
__device__ __forceinline__ void lf1(const DText &T, uint32_t c, uint32_t &lo, uint32_t &hi) {
    if (lo == 0 && hi == T.n + 1) {
        lo = T.C1[c];
        hi = T.C1[c + 1];
        return;
    }
    const uint32_t blo = lo / kRowsPerBlock, bhi = hi / kRowsPerBlock;
    Block Bl, Bh;
    load_block(T.blocks, blo, Bl);
    if (bhi != blo) load_block(T.blocks, bhi, Bh);
    uint32_t a = Bl.cnt[c] + count1_prefix(Bl, lo - blo * kRowsPerBlock, c);
    uint32_t b = (bhi != blo) ? Bh.cnt[c] + count1_prefix(Bh, hi - bhi * kRowsPerBlock, c)
                              : Bl.cnt[c] + count1_prefix(Bl, hi - blo * kRowsPerBlock, c);
    if (c == 0) {
        a -= (lo > T.primary) ? 1u : 0u;
        b -= (hi > T.primary) ? 1u : 0u;
    }
    lo = T.C1[c] + a;
    hi = T.C1[c] + b;
}

// BWT symbol at row r (r != primary) and occ_before of it at r: one LF step of
// the row itself, LF(r) = C1[B[r]] + occ_before(B[r], r).
__device__ __forceinline__ uint32_t lf_row(const DText &T, uint32_t r) {
    const uint32_t b = r / kRowsPerBlock, o = r - b * kRowsPerBlock;
    Block B;
    load_block(T.blocks, b, B);
    const uint32_t c = (B.w[o >> 4] >> (2 * (o & 15u))) & 3u;
    uint32_t v = B.cnt[c] + count1_prefix(B, o, c);
    if (c == 0) v -= (r > T.primary) ? 1u : 0u;
    return T.C1[c] + v;
}

}  // namespace aln
