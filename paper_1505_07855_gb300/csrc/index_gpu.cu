// GPU construction of the FM-index of X and of X reversed (paper Sec. 2: the
// reference is encoded offline so that all suffixes with the same starting
// subsequence share one contiguous location).  Produces exactly the image the
// host builder (index_build.cpp) produces: the suffix array is unique, and the
// Occ blocks, sampled SA and prefix-trie table are functions of it.
//
// Suffix array by prefix doubling (Manber and Myers 1993, restricted to the
// groups not yet sorted as in Larsson and Sadakane 2007):
//   round 0: every suffix is keyed by its first 21 symbols (3 bits each, a real
//            symbol c as c+1, past the end 0) and the (key, start) pairs are
//            radix-sorted; equal keys form groups, and a suffix's rank is the
//            row of its group's first member;
//   round h: the members of groups with two or more suffixes are keyed by
//            (rank of the suffix, rank of the suffix h positions later), sorted,
//            and split where the key changes; ranks are updated after every key
//            of the round has been read; h doubles, until no group is left.
// A member of a group shares h real symbols with another suffix, so s + h <= n
// and rank[n] (the suffix "$") is 0.
//
// Device primitives written for this file: a tiled scan (sum or max) and an LSD
// radix sort of (u64 key, u32 value) pairs, 8-bit digits, 4096-element tiles,
// stable ranking inside a tile by warp match + per-warp digit counters, and a
// shared-memory staging pass so that each digit's run is written contiguously.
#include <cuda_runtime.h>

#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "aln_internal.h"
#include "aln_scan.cuh"

namespace aln {
namespace {

using scan::OpAdd;
using scan::OpMax;
using scan::block_exclusive;
using scan::device_scan;
using scan::scan_temp_words;

// ------------------------------------------------------------------ radix sort

constexpr int kRsThreads = 256;
constexpr int kRsWarps = kRsThreads / 32;
constexpr int kRsRounds = 16;                                   // rounds of 32 items per warp
constexpr uint32_t kRsTile = kRsThreads * kRsRounds;            // 4096 items per tile
constexpr int kRsBins = 256;
constexpr size_t kRsSmem = (kRsWarps * kRsBins + 2 * kRsBins) * 4 + kRsTile * (8 + 4);

__global__ void __launch_bounds__(kRsThreads) rs_hist_kernel(const uint64_t *keys, uint64_t n, uint32_t shift,
                                                             uint32_t *counts, uint64_t n_tiles) {
    __shared__ uint32_t h[kRsBins];
    h[threadIdx.x] = 0;
    __syncthreads();
    const uint64_t base = static_cast<uint64_t>(blockIdx.x) * kRsTile;
#pragma unroll 4
    for (int i = 0; i < kRsRounds; i++) {
        const uint64_t j = base + static_cast<uint64_t>(i) * kRsThreads + threadIdx.x;
        if (j < n) atomicAdd(&h[(keys[j] >> shift) & 255u], 1u);
    }
    __syncthreads();
    counts[static_cast<uint64_t>(threadIdx.x) * n_tiles + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter of one tile by the digit at `shift`.  offs: exclusive scan of
// the digit-major counts (global start of digit d's part of tile t).
__global__ void __launch_bounds__(kRsThreads) rs_scatter_kernel(const uint64_t *kin, const uint32_t *vin,
                                                                uint64_t *kout, uint32_t *vout, uint64_t n,
                                                                uint32_t shift, const uint32_t *offs,
                                                                uint64_t n_tiles) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint64_t *sk = reinterpret_cast<uint64_t *>(smem_raw);
    uint32_t *sv = reinterpret_cast<uint32_t *>(sk + kRsTile);
    uint32_t *whist = sv + kRsTile;            // [warp][digit]: running count, then offset in the tile's digit
    uint32_t *tdig = whist + kRsWarps * kRsBins;  // local start of each digit in the tile
    uint32_t *wt = tdig + kRsBins;                // scan scratch (8 words used)
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kRsWarps * kRsBins; i += kRsThreads) whist[i] = 0;
    __syncthreads();
    const uint64_t base = static_cast<uint64_t>(blockIdx.x) * kRsTile;
    const uint32_t lt = (1u << lane) - 1u;
    uint64_t k[kRsRounds];
    uint32_t v[kRsRounds], pos[kRsRounds];
    uint32_t *wh = whist + warp * kRsBins;
#pragma unroll
    for (int r = 0; r < kRsRounds; r++) {
        const uint64_t j = base + static_cast<uint64_t>(warp) * (32 * kRsRounds) + 32u * r + lane;
        const bool valid = j < n;
        k[r] = valid ? kin[j] : 0ull;
        v[r] = valid ? vin[j] : 0u;
        const uint32_t d = valid ? static_cast<uint32_t>((k[r] >> shift) & 255u) : 256u;
        const uint32_t peers = __match_any_sync(0xFFFFFFFFu, d);
        const uint32_t before = valid ? wh[d] : 0u;
        __syncwarp();
        if (valid && lane == static_cast<uint32_t>(__ffs(peers) - 1)) wh[d] = before + __popc(peers);
        __syncwarp();
        pos[r] = before + __popc(peers & lt);
    }
    __syncthreads();
    // per digit (one thread each): offsets of the warps inside the tile's digit run
    uint32_t tot = 0;
    {
        const uint32_t d = threadIdx.x;
        for (int w = 0; w < kRsWarps; w++) {
            const uint32_t c = whist[w * kRsBins + d];
            whist[w * kRsBins + d] = tot;
            tot += c;
        }
    }
    __syncthreads();
    tdig[threadIdx.x] = block_exclusive(tot, wt, nullptr, OpAdd());
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kRsRounds; r++) {
        const uint64_t j = base + static_cast<uint64_t>(warp) * (32 * kRsRounds) + 32u * r + lane;
        if (j < n) {
            const uint32_t d = static_cast<uint32_t>((k[r] >> shift) & 255u);
            const uint32_t lp = tdig[d] + wh[d] + pos[r];
            sk[lp] = k[r];
            sv[lp] = v[r];
        }
    }
    __syncthreads();
    const uint32_t cnt = static_cast<uint32_t>(n - base < kRsTile ? n - base : kRsTile);
#pragma unroll 4
    for (int i = 0; i < kRsRounds; i++) {
        const uint32_t t = i * kRsThreads + threadIdx.x;
        if (t < cnt) {
            const uint64_t key = sk[t];
            const uint32_t d = static_cast<uint32_t>((key >> shift) & 255u);
            const uint64_t g = static_cast<uint64_t>(offs[static_cast<uint64_t>(d) * n_tiles + blockIdx.x]) + (t - tdig[d]);
            kout[g] = key;
            vout[g] = sv[t];
        }
    }
}

struct SortBufs {
    uint64_t *k[2];
    uint32_t *v[2];
    uint32_t *counts;  // kRsBins * tiles
    uint32_t *scan_tmp;
};

// Sort n pairs in (k[0], v[0]) by the low `bits` bits of the key (stable LSD);
// returns the index (0 or 1) of the buffers holding the result.
int radix_sort(SortBufs &B, uint64_t n, uint32_t bits, cudaStream_t st) {
    int cur = 0;
    if (n <= 1) return cur;
    const uint64_t tiles = (n + kRsTile - 1) / kRsTile;
    for (uint32_t shift = 0; shift < bits; shift += 8) {
        rs_hist_kernel<<<static_cast<unsigned>(tiles), kRsThreads, 0, st>>>(B.k[cur], n, shift, B.counts, tiles);
        device_scan(B.counts, B.counts, kRsBins * tiles, false, B.scan_tmp, st, OpAdd());
        rs_scatter_kernel<<<static_cast<unsigned>(tiles), kRsThreads, kRsSmem, st>>>(
            B.k[cur], B.v[cur], B.k[cur ^ 1], B.v[cur ^ 1], n, shift, B.counts, tiles);
        cur ^= 1;
    }
    return cur;
}

// ------------------------------------------------------------------ suffix array kernels

__device__ __forceinline__ uint64_t splitmix64_dev(uint64_t z) {
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// x[i] = text[i] (an N, or anything above 3, replaced by splitmix64(seed ^ i) & 3),
// xr[n-1-i] = x[i].
__global__ void text_kernel(const uint8_t *text, uint64_t n, uint64_t seed, uint8_t *x, uint8_t *xr) {
    for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        const uint8_t t = text[i];
        const uint8_t c = t < 4 ? t : static_cast<uint8_t>(splitmix64_dev(seed ^ i) & 3u);
        x[i] = c;
        xr[n - 1 - i] = c;
    }
}

// Round 0 keys: suffix i (0..n) keyed by its first 21 symbols.
__global__ void key21_kernel(const uint8_t *y, uint64_t n, uint64_t *key, uint32_t *val) {
    const uint64_t N = n + 1;
    for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i < N;
         i += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        uint64_t k = 0;
#pragma unroll
        for (int t = 0; t < 21; t++) {
            const uint64_t p = i + t;
            k = (k << 3) | (p < n ? static_cast<uint64_t>(y[p]) + 1u : 0u);
        }
        key[i] = k;
        val[i] = static_cast<uint32_t>(i);
    }
}

// head[i] = i where key[i] starts a run of equal keys, else 0 (max-scan input).
__global__ void run_head_kernel(const uint64_t *key, uint64_t m, uint32_t *head) {
    for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i < m;
         i += static_cast<uint64_t>(gridDim.x) * blockDim.x)
        head[i] = (i == 0 || key[i] != key[i - 1]) ? static_cast<uint32_t>(i) : 0u;
}

// After a sort of the active rows: the suffix order goes back into sa at the
// rows the active set occupies, and each suffix's rank becomes the row of the
// first member of its new run.  A == nullptr: the active set is every row.
__global__ void place_rank_kernel(const uint32_t *A, const uint32_t *v, const uint32_t *start, uint64_t m,
                                  uint32_t *sa, uint32_t *rank) {
    for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i < m;
         i += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        const uint32_t row = A ? A[i] : static_cast<uint32_t>(i);
        const uint32_t s = v[i];
        sa[row] = s;
        rank[s] = A ? A[start[i]] : start[i];
    }
}

// active[i] = 1 if row i's run has two or more members (keys sorted).
__global__ void active_kernel(const uint64_t *key, uint64_t m, uint32_t *active) {
    for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i < m;
         i += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        const bool head = i == 0 || key[i] != key[i - 1];
        const bool next_head = i + 1 == m || key[i + 1] != key[i];
        active[i] = (head && next_head) ? 0u : 1u;
    }
}

// Compaction: rows of active runs, in order.  pos = inclusive scan of the
// flags; flags are recomputed from the keys (the flag array was scanned in place).
__global__ void compact_kernel(const uint64_t *key, const uint32_t *A, const uint32_t *pos, uint64_t m,
                               uint32_t *A2) {
    for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i < m;
         i += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        const bool head = i == 0 || key[i] != key[i - 1];
        const bool next_head = i + 1 == m || key[i + 1] != key[i];
        if (!(head && next_head)) A2[pos[i] - 1] = A ? A[i] : static_cast<uint32_t>(i);
    }
}

// Keys of a doubling round: (rank of the suffix, rank of the suffix h later).
__global__ void round_key_kernel(const uint32_t *A, uint64_t m, const uint32_t *sa, const uint32_t *rank,
                                 uint64_t h, uint64_t n, uint32_t b, uint64_t *key, uint32_t *val) {
    for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i < m;
         i += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        const uint32_t s = sa[A[i]];
        const uint64_t s2 = static_cast<uint64_t>(s) + h;
        const uint32_t r2 = s2 <= n ? rank[s2] : 0u;  // s + h <= n for every member of a group
        key[i] = (static_cast<uint64_t>(rank[s]) << b) | r2;
        val[i] = s;
    }
}

// ------------------------------------------------------------------ index image kernels

// One warp per Occ block of 192 rows: the symbol of row r is y[sa[r] - 1] ($
// and padding as A); ballots give the bit planes of each half (3 words of low
// bits, then 3 of high bits), and the counts of the block and of its first half
// (rows < N only) go to bcount / hcount (column c at c * nb).
__global__ void pack_kernel(const uint8_t *y, const uint32_t *sa, uint64_t N, uint64_t nb, uint32_t *blocks,
                            uint32_t *bcount, uint32_t *hcount) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t warps = static_cast<uint64_t>(gridDim.x) * (blockDim.x >> 5);
    for (uint64_t b = (blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x) >> 5; b < nb; b += warps) {
        uint32_t c4[4] = {0, 0, 0, 0}, h4[4] = {0, 0, 0, 0};
        uint32_t w[12];
#pragma unroll
        for (int u = 0; u < 6; u++) {
            const uint64_t r = b * static_cast<uint64_t>(kBlockRows) + 32u * u + lane;
            const bool valid = r < N;
            uint32_t sym = 0;
            if (valid) {
                const uint32_t s = sa[r];
                sym = s == 0 ? 0u : y[s - 1];
            }
            const uint32_t lo = __ballot_sync(0xFFFFFFFFu, sym & 1u);
            const uint32_t hi = __ballot_sync(0xFFFFFFFFu, (sym >> 1) & 1u);
            const uint32_t vm = __ballot_sync(0xFFFFFFFFu, valid);
            const int half = u / 3, g = u % 3;
            w[6 * half + g] = lo;
            w[6 * half + 3 + g] = hi;
            const uint32_t nT = __popc(lo & hi & vm), nG = __popc(hi & ~lo & vm), nC = __popc(lo & ~hi & vm);
            const uint32_t nA = __popc(vm) - nT - nG - nC;
            c4[0] += nA; c4[1] += nC; c4[2] += nG; c4[3] += nT;
            if (half == 0) {
                h4[0] += nA; h4[1] += nC; h4[2] += nG; h4[3] += nT;
            }
        }
        if (lane < 12) {
            uint32_t val = w[0];
#pragma unroll
            for (int q = 1; q < 12; q++)
                if (lane == static_cast<uint32_t>(q)) val = w[q];
            blocks[b * 16 + 4 + lane] = val;
        }
        if (lane < 4) {
            const uint32_t cc = lane == 0 ? c4[0] : (lane == 1 ? c4[1] : (lane == 2 ? c4[2] : c4[3]));
            const uint32_t hh = lane == 0 ? h4[0] : (lane == 1 ? h4[1] : (lane == 2 ? h4[2] : h4[3]));
            bcount[static_cast<uint64_t>(lane) * nb + b] = cc;
            hcount[static_cast<uint64_t>(lane) * nb + b] = hh;
        }
    }
}

// Counts before each block's middle row: the exclusive prefix of the earlier
// blocks' counts plus the block's first half; padding rows of the first half
// (stored as A) are counted as A.
__global__ void counts_kernel(const uint32_t *bpre, const uint32_t *hcount, uint64_t N, uint64_t nb,
                              uint32_t *blocks) {
    for (uint64_t b = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; b < nb;
         b += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        const uint64_t mid = b * static_cast<uint64_t>(kBlockRows) + static_cast<uint64_t>(kBlockRows) / 2;
        const uint64_t over = mid > N ? mid - N : 0;
        const uint32_t pad = static_cast<uint32_t>(over < static_cast<uint64_t>(kBlockRows) / 2 ? over : static_cast<uint64_t>(kBlockRows) / 2);
#pragma unroll
        for (int c = 0; c < 4; c++)
            blocks[b * 16 + c] = bpre[c * nb + b] + hcount[c * nb + b] + (c == 0 ? pad : 0u);
    }
}

__global__ void sample_kernel(const uint32_t *sa, uint64_t ns, uint32_t sample, uint32_t *out) {
    for (uint64_t t = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; t < ns;
         t += static_cast<uint64_t>(gridDim.x) * blockDim.x)
        out[t] = sa[t * sample];
}

__global__ void primary_count_kernel(const uint32_t *sa, const uint8_t *y, uint64_t n, unsigned long long *primary,
                                     unsigned long long *cnt) {
    __shared__ unsigned long long c[4];
    if (threadIdx.x < 4) c[threadIdx.x] = 0;
    __syncthreads();
    uint32_t loc[4] = {0, 0, 0, 0};
    for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i <= n;
         i += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        if (sa[i] == 0) *primary = i;
        if (i < n) loc[y[i]]++;
    }
#pragma unroll
    for (int q = 0; q < 4; q++) atomicAdd(&c[q], static_cast<unsigned long long>(loc[q]));
    __syncthreads();
    if (threadIdx.x < 4) atomicAdd(&cnt[threadIdx.x], c[threadIdx.x]);
}

// The first min(k, n - s) symbols of the suffix at row r as a base-4 number,
// first symbol lowest (the order the search processes them), with the count of
// available symbols in bits 24..27.
__global__ void kmer_id_kernel(const uint8_t *y, const uint32_t *sa, uint64_t n, uint32_t k, uint32_t *id) {
    for (uint64_t r = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; r <= n;
         r += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        const uint64_t s = sa[r];
        const uint32_t avail = static_cast<uint32_t>(n - s < k ? n - s : k);
        uint32_t v = 0;
        for (uint32_t u = 0; u < avail; u++) v |= static_cast<uint32_t>(y[s + u]) << (2 * u);
        id[r] = v | (avail << 24);
    }
}

// Prefix-trie table: for every level j, the run of rows whose j-prefix is the
// string with index i sets entry (lo, hi) = (first row, last row + 1).
__global__ void kmer_table_kernel(const uint32_t *id, uint64_t N, uint32_t k, uint32_t *kmer) {
    for (uint64_t r = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; r < N;
         r += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        const uint32_t cur = id[r];
        const uint32_t prv = r > 0 ? id[r - 1] : 0u, nxt = r + 1 < N ? id[r + 1] : 0u;
        for (uint32_t j = 1; j <= k; j++) {
            if ((cur >> 24) < j) break;
            const uint32_t mask = (1u << (2 * j)) - 1u;
            const uint32_t me = cur & mask;
            const uint64_t off = ((1ull << (2 * j)) - 4) / 3 + me;
            const bool first = r == 0 || (prv >> 24) < j || (prv & mask) != me;
            const bool last = r + 1 == N || (nxt >> 24) < j || (nxt & mask) != me;
            if (first) kmer[2 * off] = static_cast<uint32_t>(r);
            if (last) kmer[2 * off + 1] = static_cast<uint32_t>(r + 1);
        }
    }
}

unsigned grid_for(uint64_t n, int threads) {
    const uint64_t g = (n + threads - 1) / threads;
    return static_cast<unsigned>(g < 65536ull * 16 ? (g ? g : 1) : 65536ull * 16);
}

// Device memory of one build, freed on destruction.
struct DevMem {
    std::vector<void *> ptrs;
    cudaError_t err = cudaSuccess;
    template <class T>
    T *alloc(uint64_t count) {
        void *p = nullptr;
        if (err == cudaSuccess) {
            err = cudaMalloc(&p, (count ? count : 1) * sizeof(T));
            if (err == cudaSuccess) ptrs.push_back(p);
            else p = nullptr;
        }
        return static_cast<T *>(p);
    }
    ~DevMem() {
        for (void *p : ptrs) cudaFree(p);
    }
};

}  // namespace

// Suffix array of y$ (y on the device, codes 0..3, length n) into sa (n + 1 rows).
// rank, A, A2, tmp: n + 1 words each.
static cudaError_t gpu_suffix_array(const uint8_t *y, uint64_t n, uint32_t *sa, uint32_t *rank, uint32_t *A,
                                    uint32_t *A2, uint32_t *tmp, SortBufs &B, cudaStream_t st) {
    const uint64_t N = n + 1;
    const int T = 256;
    cudaError_t e;
    key21_kernel<<<grid_for(N, T), T, 0, st>>>(y, n, B.k[0], B.v[0]);
    int c = radix_sort(B, N, 63, st);
    uint64_t m = N;
    const uint32_t *Acur = nullptr;  // round 0: the active rows are all rows
    uint32_t b = 1;
    while (b < 32 && (1ull << b) < N) b++;
    uint64_t h = 21;
    for (int round = 0;; round++) {
        // ranks: the row of the first member of each run of equal keys
        run_head_kernel<<<grid_for(m, T), T, 0, st>>>(B.k[c], m, tmp);
        device_scan(tmp, tmp, m, true, B.scan_tmp, st, OpMax());
        place_rank_kernel<<<grid_for(m, T), T, 0, st>>>(Acur, B.v[c], tmp, m, sa, rank);
        // rows of runs with two or more members stay active
        active_kernel<<<grid_for(m, T), T, 0, st>>>(B.k[c], m, tmp);
        device_scan(tmp, tmp, m, true, B.scan_tmp, st, OpAdd());
        uint32_t *Anext = (Acur == A) ? A2 : A;
        compact_kernel<<<grid_for(m, T), T, 0, st>>>(B.k[c], Acur, tmp, m, Anext);
        uint32_t m2 = 0;
        if ((e = cudaMemcpyAsync(&m2, tmp + (m - 1), 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
        if (m2 == 0) break;
        if (round >= 34 || h > 2 * N) return cudaErrorUnknown;  // cannot happen: runs share h real symbols
        Acur = Anext;
        m = m2;
        round_key_kernel<<<grid_for(m, T), T, 0, st>>>(Acur, m, sa, rank, h, n, b, B.k[0], B.v[0]);
        c = radix_sort(B, m, 2 * b, st);
        h *= 2;
    }
    return cudaGetLastError();
}

}  // namespace aln

using namespace aln;

extern "C" int fm_index_build_gpu(const uint8_t *text, uint64_t n, const fm_build_opts *opts, int device,
                                  void *stream, fm_index **out) {
    if (!text || !out) return fail(ALN_EINVAL, "fm_index_build_gpu: null argument");
    *out = nullptr;
    if (n < 1 || n >= 0xFFFFFFFFULL) return fail(ALN_EINVAL, "fm_index_build_gpu: n must be in [1, 2^32-2]");
    fm_build_opts o{};
    if (opts) o = *opts;
    if (o.sa_sample == 0) o.sa_sample = 32;
    if (o.sa_sample > 1024 || (o.sa_sample & (o.sa_sample - 1)))
        return fail(ALN_EINVAL, "fm_index_build_gpu: sa_sample must be a power of two <= 1024");
    if (o.kmer_k > ALN_MAX_KMER_K) return fail(ALN_EINVAL, "fm_index_build_gpu: kmer_k too large");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return fail(ALN_EINVAL, "fm_index_build_gpu: bad device ordinal");
    }
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const uint64_t N = n + 1;
    const uint64_t tiles = (N + kRsTile - 1) / kRsTile;
    const uint64_t nb = N / kBlockRows + 1;
    const uint64_t ns = n / o.sa_sample + 1;
    const uint64_t kwords = o.kmer_k ? 2 * (((1ull << (2 * (o.kmer_k + 1))) - 4) / 3) : 0;
    int rc = ALN_OK;
    fm_index *ix = nullptr;
    {
        DevMem M;
        uint8_t *x = M.alloc<uint8_t>(n), *xr = M.alloc<uint8_t>(n);
        const uint64_t W = N > 4 * nb ? N : 4 * nb;  // A, A2, tmp also hold 4 count columns of nb blocks
        uint32_t *sa = M.alloc<uint32_t>(N), *rank = M.alloc<uint32_t>(N), *A = M.alloc<uint32_t>(W);
        uint32_t *A2 = M.alloc<uint32_t>(W), *tmp = M.alloc<uint32_t>(W);
        SortBufs B;
        B.k[0] = M.alloc<uint64_t>(N);
        B.k[1] = M.alloc<uint64_t>(N);
        B.v[0] = M.alloc<uint32_t>(N);
        B.v[1] = M.alloc<uint32_t>(N);
        B.counts = M.alloc<uint32_t>(kRsBins * tiles);
        const uint64_t scan_n = kRsBins * tiles > N ? kRsBins * tiles : N;
        B.scan_tmp = M.alloc<uint32_t>(scan_temp_words(scan_n));
        uint32_t *blocks = M.alloc<uint32_t>(nb * 16), *samp = M.alloc<uint32_t>(ns);
        uint32_t *kmer = M.alloc<uint32_t>(kwords);
        unsigned long long *misc = M.alloc<unsigned long long>(8);
        cudaError_t e = M.err;
        if (e == cudaSuccess) {  // N replacement and the reversed text (the input copy is freed at once)
            uint8_t *d_text = nullptr;
            e = cudaMalloc(&d_text, n);
            if (e == cudaSuccess) e = cudaMemcpyAsync(d_text, text, n, cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess) text_kernel<<<grid_for(n, 256), 256, 0, st>>>(d_text, n, o.n_seed, x, xr);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (d_text) cudaFree(d_text);
        }
        if (e == cudaSuccess) e = cudaFuncSetAttribute(rs_scatter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                       static_cast<int>(kRsSmem));
        if (e == cudaSuccess) {
            try {
                ix = new fm_index();
            } catch (const std::bad_alloc &) {
                ix = nullptr;
            }
            if (!ix) rc = fail(ALN_ENOMEM, "fm_index_build_gpu: host allocation failed");
        }
        for (int w = 0; w < 2 && e == cudaSuccess && rc == ALN_OK; w++) {
            const uint8_t *y = w ? xr : x;
            e = gpu_suffix_array(y, n, sa, rank, A, A2, tmp, B, st);
            if (e != cudaSuccess) break;
            // Occ blocks: bit planes and counts, then the counts before each middle row
            cudaMemsetAsync(blocks, 0, nb * 16 * 4, st);
            pack_kernel<<<grid_for(nb * 32, 256), 256, 0, st>>>(y, sa, N, nb, blocks, A, A2);
            for (int cc = 0; cc < 4; cc++)
                device_scan(A + cc * nb, tmp + cc * nb, nb, false, B.scan_tmp, st, OpAdd());
            counts_kernel<<<grid_for(nb, 256), 256, 0, st>>>(tmp, A2, N, nb, blocks);
            sample_kernel<<<grid_for(ns, 256), 256, 0, st>>>(sa, ns, o.sa_sample, samp);
            cudaMemsetAsync(misc, 0, 8 * sizeof(unsigned long long), st);
            primary_count_kernel<<<grid_for(N, 256) < 4096 ? grid_for(N, 256) : 4096, 256, 0, st>>>(sa, y, n, misc,
                                                                                                  misc + 1);
            if (o.kmer_k) {
                kmer_id_kernel<<<grid_for(N, 256), 256, 0, st>>>(y, sa, n, o.kmer_k, tmp);
                cudaMemsetAsync(kmer, 0, kwords * 4, st);
                kmer_table_kernel<<<grid_for(N, 256), 256, 0, st>>>(tmp, N, o.kmer_k, kmer);
            }
            if ((e = cudaGetLastError()) != cudaSuccess) break;
            HostText &Tt = ix->t[w];
            unsigned long long hm[5];
            try {
                Tt.blocks.resize(nb * 16);
                Tt.sa_samp.resize(ns);
                Tt.kmer.resize(kwords);
            } catch (const std::bad_alloc &) {
                rc = fail(ALN_ENOMEM, "fm_index_build_gpu: host allocation failed");
                break;
            }
            if ((e = cudaMemcpyAsync(Tt.blocks.data(), blocks, nb * 16 * 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess) break;
            if ((e = cudaMemcpyAsync(Tt.sa_samp.data(), samp, ns * 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess) break;
            if (kwords && (e = cudaMemcpyAsync(Tt.kmer.data(), kmer, kwords * 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
                break;
            if ((e = cudaMemcpyAsync(hm, misc, 5 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
                break;
            if ((e = cudaStreamSynchronize(st)) != cudaSuccess) break;
            Tt.n = n;
            Tt.primary = hm[0];
            Tt.C[0] = 0;
            for (int cc = 1; cc < 4; cc++) Tt.C[cc] = Tt.C[cc - 1] + hm[cc];
        }
        if (rc == ALN_OK && e != cudaSuccess)
            rc = fail(e == cudaErrorMemoryAllocation ? ALN_ENOMEM : ALN_EDEVICE,
                      std::string("fm_index_build_gpu: ") + cudaGetErrorString(e));
    }
    cudaSetDevice(prev);
    if (rc != ALN_OK) {
        delete ix;
        cudaGetLastError();
        return rc;
    }
    ix->sa_sample = o.sa_sample;
    ix->kmer_k = o.kmer_k;
    ix->n_seed = o.n_seed;
    *out = ix;
    return ALN_OK;
}
