// Pairing of mates after the search (sm_103a): the pipeline's pairing stage
// (paper Sec. 2 and the pipeline of Sec. 3: the pairing stage combines the two
// mates' hits using the fragment length, and needs their positions).
//
// Input: the search's per-read results, its hits compacted by aln_compact_hits
// (offsets + dense hits) and their positions from sa_to_pos.  Read 2p is mate 1
// and read 2p+1 mate 2 of pair p.  The rule (stated in include/aln_gb300.h):
//   placements of a mate = the positions of its best-stratum hits; a mate is
//   placed when it has 1..max_place of them and all were written;
//   insert of a combination with opposite strands = end of the reverse
//   placement - start of the forward one;
//   window = [q1 - 2 IQR, q3 + 2 IQR] (clamped to 1..65535) from the integer
//   quartiles of the unique pairs' inserts (both mates one placement);
//   the choice = the proper combination smallest by (n_diff sum, |insert - q2|,
//   insert, pos1, pos2, strand1, len1, len2).
// Three kernels: a histogram of the unique pairs' inserts (65536 bins), one
// block that finds the quartiles by a scan of the histogram, one thread per
// pair that enumerates its combinations.
#include <cuda_runtime.h>

#include <string>

#include "aln_internal.h"
#include "aln_scan.cuh"

namespace aln {
namespace {

constexpr uint32_t kIsizeBins = ALN_PAIR_ISIZE_MAX + 1;
constexpr int kMaxPlace = 64;

struct Place {
    uint64_t pos;
    uint32_t len;
    uint32_t strand;
    uint32_t n_diff;
};

struct PairIn {
    const aln_read_result *reads;
    const uint32_t *off;
    const aln_hit *hits;
    const uint64_t *pos;
    const uint32_t *npos;
    uint32_t W;
};

// Placements of read r (at most cap); -1 if the read is not placed.
__device__ int placements(const PairIn &in, uint64_t r, uint32_t max_place, Place *out) {
    const aln_read_result R = in.reads[r];
    if (R.n_hits == 0 || R.c0 < 1 || R.c0 > max_place) return -1;
    int k = 0;
    for (uint32_t h = in.off[r]; h < in.off[r + 1]; h++) {
        const aln_hit H = in.hits[h];
        if (H.n_diff != R.d_best) continue;
        const uint32_t np = in.npos[h];
        const uint64_t width = static_cast<uint64_t>(H.l) - H.k + 1;
        if (np > in.W || np != width) return -1;  // positions missing (too wide, walk bound)
        for (uint32_t j = 0; j < np; j++) {
            if (k == static_cast<int>(max_place)) return -1;
            out[k].pos = in.pos[static_cast<uint64_t>(h) * in.W + j];
            out[k].len = H.aligned_len;
            out[k].strand = H.strand;
            out[k].n_diff = H.n_diff;
            k++;
        }
    }
    return static_cast<uint32_t>(k) == R.c0 ? k : -1;
}

__device__ __forceinline__ long long insert_of(const Place &a, const Place &b, bool &fr) {
    fr = a.strand != b.strand;
    if (!fr) return 0;
    const Place &f = a.strand == 0 ? a : b, &v = a.strand == 0 ? b : a;
    return static_cast<long long>(v.pos) + v.len - static_cast<long long>(f.pos);
}

// The single placement of a read with c0 == 1, if it has one.
__device__ bool unique_place(const PairIn &in, uint64_t r, Place &p) {
    const aln_read_result R = in.reads[r];
    if (R.c0 != 1 || R.n_hits == 0) return false;
    const uint32_t h = in.off[r];
    if (h >= in.off[r + 1]) return false;
    const aln_hit H = in.hits[h];
    if (H.n_diff != R.d_best || H.k != H.l || in.npos[h] != 1) return false;
    p.pos = in.pos[static_cast<uint64_t>(h) * in.W];
    p.len = H.aligned_len;
    p.strand = H.strand;
    p.n_diff = H.n_diff;
    return true;
}

__global__ void pair_hist_kernel(PairIn in, uint64_t n_pairs, uint32_t *hist) {
    for (uint64_t p = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; p < n_pairs;
         p += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        Place a, b;
        if (!unique_place(in, 2 * p, a) || !unique_place(in, 2 * p + 1, b)) continue;
        bool fr;
        const long long x = insert_of(a, b, fr);
        if (fr && x >= 1 && x <= ALN_PAIR_ISIZE_MAX) atomicAdd(&hist[x], 1u);
    }
}

// One block of 1024 threads: each owns 64 consecutive bins; the block scan of
// their counts gives each thread the rank of its first bin, and the thread whose
// bins contain rank t reports the value s[t].
constexpr int kWinThreads = 1024;
constexpr int kBinsPerThread = kIsizeBins / kWinThreads;

__global__ void __launch_bounds__(kWinThreads) pair_window_kernel(const uint32_t *hist, aln_pair_stats *st) {
    __shared__ uint32_t wt[32];
    __shared__ uint32_t q[3];
    uint32_t local = 0;
    for (int i = 0; i < kBinsPerThread; i++) local += hist[threadIdx.x * kBinsPerThread + i];
    uint32_t u = 0;
    const uint32_t before = scan::block_exclusive(local, wt, &u, scan::OpAdd());
    const uint32_t target[3] = {u / 4, u / 2, static_cast<uint32_t>((3ull * u) / 4)};
    uint32_t run = before;
    for (int i = 0; i < kBinsPerThread; i++) {
        const uint32_t c = hist[threadIdx.x * kBinsPerThread + i];
#pragma unroll
        for (int t = 0; t < 3; t++)
            if (c && target[t] >= run && target[t] < run + c) q[t] = threadIdx.x * kBinsPerThread + i;
        run += c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        aln_pair_stats s{};
        s.n_unique = u;
        s.lo = 1;
        s.hi = ALN_PAIR_ISIZE_MAX;
        if (u >= 8) {
            s.q1 = q[0];
            s.q2 = q[1];
            s.q3 = q[2];
            const long long iqr = static_cast<long long>(s.q3) - s.q1;
            const long long lo = static_cast<long long>(s.q1) - 2 * iqr, hi = static_cast<long long>(s.q3) + 2 * iqr;
            s.lo = static_cast<uint32_t>(lo < 1 ? 1 : lo);
            s.hi = static_cast<uint32_t>(hi > ALN_PAIR_ISIZE_MAX ? ALN_PAIR_ISIZE_MAX : hi);
        }
        *st = s;
    }
}

__global__ void pair_kernel(PairIn in, uint64_t n_pairs, uint32_t max_place, const aln_pair_stats *stp,
                            aln_pair_result *out) {
    const aln_pair_stats st = *stp;
    Place pa[kMaxPlace], pb[kMaxPlace];
    for (uint64_t p = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; p < n_pairs;
         p += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        aln_pair_result o{};
        o.pos[0] = o.pos[1] = ~0ull;
        o.strand[0] = o.strand[1] = 255;
        if (in.reads[2 * p].n_hits) o.flags |= ALN_PAIR_MAPPED1;
        if (in.reads[2 * p + 1].n_hits) o.flags |= ALN_PAIR_MAPPED2;
        const int na = placements(in, 2 * p, max_place, pa);
        const int nb = placements(in, 2 * p + 1, max_place, pb);
        if (na > 0) o.flags |= ALN_PAIR_PLACED1;
        if (nb > 0) o.flags |= ALN_PAIR_PLACED2;
        if (na > 0 && nb > 0) {
            if (na == 1 && nb == 1) {
                bool fr;
                const long long x = insert_of(pa[0], pb[0], fr);
                if (fr && x >= 1 && x <= ALN_PAIR_ISIZE_MAX) o.flags |= ALN_PAIR_UNIQUE;
            }
            uint32_t nproper = 0;
            int bi = -1, bj = -1;
            long long bx = 0;
            for (int i = 0; i < na; i++) {
                for (int j = 0; j < nb; j++) {
                    bool fr;
                    const long long x = insert_of(pa[i], pb[j], fr);
                    if (!fr || x < static_cast<long long>(st.lo) || x > static_cast<long long>(st.hi)) continue;
                    nproper++;
                    bool better = bi < 0;
                    if (!better) {
                        const uint32_t d = pa[i].n_diff + pb[j].n_diff, db = pa[bi].n_diff + pb[bj].n_diff;
                        const long long e = x > st.q2 ? x - st.q2 : st.q2 - x;
                        const long long eb = bx > st.q2 ? bx - st.q2 : st.q2 - bx;
                        if (d != db) better = d < db;
                        else if (e != eb) better = e < eb;
                        else if (x != bx) better = x < bx;
                        else if (pa[i].pos != pa[bi].pos) better = pa[i].pos < pa[bi].pos;
                        else if (pb[j].pos != pb[bj].pos) better = pb[j].pos < pb[bj].pos;
                        else if (pa[i].strand != pa[bi].strand) better = pa[i].strand < pa[bi].strand;
                        else if (pa[i].len != pa[bi].len) better = pa[i].len < pa[bi].len;
                        else better = pb[j].len < pb[bj].len;
                    }
                    if (better) {
                        bi = i;
                        bj = j;
                        bx = x;
                    }
                }
            }
            o.n_proper = static_cast<uint16_t>(nproper > 65535 ? 65535 : nproper);
            if (bi >= 0) {
                o.flags |= ALN_PAIR_PROPER;
                o.pos[0] = pa[bi].pos;
                o.pos[1] = pb[bj].pos;
                o.strand[0] = static_cast<uint8_t>(pa[bi].strand);
                o.strand[1] = static_cast<uint8_t>(pb[bj].strand);
                o.insert = static_cast<uint32_t>(bx);
            } else {
                o.flags |= ALN_PAIR_DISCORDANT;
            }
        }
        out[p] = o;
    }
}

}  // namespace
}  // namespace aln

using namespace aln;

extern "C" uint64_t aln_pair_scratch_bytes(void) { return 4ull * kIsizeBins; }

extern "C" int aln_pair_resolve(const aln_read_result *reads, const uint32_t *hit_off, const aln_hit *hits,
                                const uint64_t *pos, const uint32_t *npos, uint32_t max_width, uint32_t n_pairs,
                                uint32_t max_place, aln_pair_result *out, aln_pair_stats *stats, void *scratch,
                                uint64_t scratch_bytes, void *stream) {
    if (!stats || !scratch || (n_pairs && (!reads || !hit_off || !hits || !pos || !npos || !out)))
        return fail(ALN_EINVAL, "aln_pair_resolve: null argument");
    if (max_width < 1 || max_width > 64) return fail(ALN_EINVAL, "aln_pair_resolve: max_width must be 1..64");
    if (max_place < 1 || max_place > max_width || max_place > static_cast<uint32_t>(kMaxPlace))
        return fail(ALN_EINVAL, "aln_pair_resolve: max_place must be 1..max_width");
    if (scratch_bytes < aln_pair_scratch_bytes()) return fail(ALN_EINVAL, "aln_pair_resolve: scratch too small");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    uint32_t *hist = static_cast<uint32_t *>(scratch);
    PairIn in{reads, hit_off, hits, pos, npos, max_width};
    cudaMemsetAsync(hist, 0, 4ull * kIsizeBins, st);
    const uint64_t g = (static_cast<uint64_t>(n_pairs) + 255) / 256;
    const unsigned grid = static_cast<unsigned>(g < 65536 ? (g ? g : 1) : 65536);
    pair_hist_kernel<<<grid, 256, 0, st>>>(in, n_pairs, hist);
    pair_window_kernel<<<1, kWinThreads, 0, st>>>(hist, stats);
    if (n_pairs) pair_kernel<<<grid, 128, 0, st>>>(in, n_pairs, max_place, stats, out);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return fail(ALN_EDEVICE, std::string("aln_pair_resolve: launch: ") + cudaGetErrorString(e));
    return ALN_OK;
}
