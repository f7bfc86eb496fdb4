// Search kernels and their launcher.
//
// Plain form: one launch per batch, one thread per read (both strands).
// Persistent form: one launch of (SMs x resident blocks); every thread pulls the
// next read from a device queue counter when it finishes one, so a few long
// reads no longer hold a whole warp's worth of short ones.
//
// Stack bound: the match child is pushed below the alternatives, so entries on
// the stack have non-decreasing difference counts from bottom to top and a
// node is only expanded when it is on top; expanding a node with d differences
// adds one entry with d and at most 9 with d+1 (4 mismatches when the read base
// is N, 1 insertion, 4 deletions), and only when no entry with d+1 is on the
// stack.  Hence at most 1 + 9*B entries for budget B; the capacity is chosen
// from z so the overflow flag cannot be raised.
#include <cuda_runtime.h>

#include <string>

#include "aln_flat.cuh"
#include "aln_search.cuh"

namespace aln {

#ifdef ALN_STATS
// Instrumented build only: event counters of the persistent kernel.
//  0 loop iterations (lane)   1 fetch iterations (lane)   2 Occ fetches
//  3 table fetches            4 warp-level fetch issues    5 lanes at those issues
//  6 reads finished           7 control rounds             8 stack pops
//  9 warp trips                10 live lanes at those trips
// 11 cycles in control         12 cycles in fetch + apply   13 cycles in the hand-over
//    (11-13 measured by lane 0 of each warp between warp re-formations)
__device__ unsigned long long g_stats[16];
#define STAT_ADD(i, v) atomicAdd(&g_stats[i], static_cast<unsigned long long>(v))
#endif

template <int STACK_CAP>
__global__ void __launch_bounds__(kThreads) aln_plain_kernel(DIndex X, ReadBatch rb, uint32_t n_reads, SearchParams p,
                                                             aln_read_result *res, aln_hit *hits) {
    __shared__ uint32_t s_bases[kReadWords * kThreads];
    __shared__ uint32_t s_nmask[kMaskWords * kThreads];
    const uint32_t r = blockIdx.x * kThreads + threadIdx.x;
    if (r >= n_reads) return;
    const uint32_t m = rb.len[r];
    const uint32_t z = rb.z ? rb.z[r] : p.z;
    ReadView rv{s_bases + threadIdx.x, s_nmask + threadIdx.x};
    if (m <= ALN_MAX_READ_LEN && m > 0) load_read(rb, rb.offset[r], m, s_bases + threadIdx.x, s_nmask + threadIdx.x);
    Search<STACK_CAP> S;
    S.run(X, rv, m, z, p, res + r, hits + static_cast<uint64_t>(r) * p.hit_cap);
}

#ifndef ALN_PERSISTENT_MIN_BLOCKS
#define ALN_PERSISTENT_MIN_BLOCKS 6  // 6 resident blocks per SM (80 registers, 8 shared stack entries) measured best
#endif

template <int STACK_CAP, int SMEM>
__global__ void __launch_bounds__(kThreads, ALN_PERSISTENT_MIN_BLOCKS) aln_persistent_kernel(DIndex X, ReadBatch rb, uint32_t n_reads,
                                                                  SearchParams p, aln_read_result *res,
                                                                  aln_hit *hits, uint32_t *queue,
                                                                  const uint32_t *order, const uint2 *dbp) {
    __shared__ uint32_t s_bases[kReadWords * kThreads];
    __shared__ uint32_t s_nmask[kMaskWords * kThreads];
    __shared__ uint4 s_stack[SMEM * kThreads];
    uint32_t *sb = s_bases + threadIdx.x, *sn = s_nmask + threadIdx.x;
    const uint32_t lane = threadIdx.x & 31u, warp_col = threadIdx.x & ~31u;
    uint4 stk[STACK_CAP - SMEM], cand[kCandCap];
    FlatLane<STACK_CAP, SMEM> L;
    L.sstk = s_stack + threadIdx.x;
    L.stk = stk;
    L.cand = cand;
    L.has_next = false;
    L.phase = PH_IDLE;
    L.r = 0xFFFFFFFFu;
    L.sp = 0;
    L.base = 0;
    L.K = X.kmer_k;
    L.role = ROLE_OWN;
    L.owner = lane;
    L.outstanding = 0;
    L.heavy_seen = false;
    L.own_rv = ReadView{sb, sn};
    L.rv = L.own_rv;
#ifdef ALN_STATS
    unsigned long long st_it = 0, st_f = 0, st_occ = 0, st_tab = 0, st_wi = 0, st_wl = 0, st_wa = 0, st_wal = 0;
    unsigned long long st_cc = 0, st_cf = 0, st_ce = 0;
#endif
    // All 32 lanes of the warp stay in the loop until every lane is free and the
    // queue is empty; each trip is: control, one converged fetch, the hand-over.
    // The trip count is warp-uniform; at p.loop_limit trips the warp stops and
    // flags what it has not finished (stop_at_limit).
    bool at_limit = false;
    for (unsigned long long it = 0;; it++) {
        if (it >= p.loop_limit) {
            at_limit = true;
            break;
        }
        FetchReq fr;
#ifdef ALN_STATS
        const unsigned long long k0 = clock64();
#endif
        L.control(X, rb, n_reads, p, res, hits, queue, order, dbp, sb, sn, fr);
        __syncwarp();
#ifdef ALN_STATS
        const unsigned long long k1 = clock64();
#endif
#ifdef ALN_STATS
        st_it++;
        {
            const unsigned busy = __ballot_sync(0xFFFFFFFFu, L.phase != PH_FREE);
            if (lane == 0) {
                st_wa++;
                st_wal += __popc(busy);
            }
        }
#endif
        if (fr.kind != F_NONE) {
#ifdef ALN_STATS
            const unsigned am = __activemask();
            st_f++;
            st_occ += fr.kind == F_OCC;
            st_tab += fr.kind == F_TABLE;
            if (lane == __ffs(am) - 1) {
                st_wi++;
                st_wl += __popc(am);
            }
#endif
            uint32_t lo4[4], hi4[4];
            fetch4(X, fr, lo4, hi4);
            L.apply(X, lo4, hi4);
        }
#ifdef ALN_STATS
        __syncwarp();
        const unsigned long long k2 = clock64();
#endif
        L.exchange(lane, s_bases, s_nmask, warp_col, p.help_after);
#ifdef ALN_STATS
        if (lane == 0) {
            st_cc += k1 - k0;
            st_cf += k2 - k1;
            st_ce += clock64() - k2;
        }
#endif
        if (__ballot_sync(0xFFFFFFFFu, L.phase != PH_FREE) == 0) break;
    }
    if (at_limit) L.stop_at_limit(lane, n_reads, p, res, queue, order);
#ifdef ALN_STATS
    STAT_ADD(0, st_it); STAT_ADD(1, st_f); STAT_ADD(2, st_occ); STAT_ADD(3, st_tab);
    STAT_ADD(4, st_wi); STAT_ADD(5, st_wl); STAT_ADD(6, L.st_reads); STAT_ADD(7, L.st_rounds);
    STAT_ADD(8, L.st_pops); STAT_ADD(9, st_wa); STAT_ADD(10, st_wal);
    STAT_ADD(11, st_cc); STAT_ADD(12, st_cf); STAT_ADD(13, st_ce);
#endif
}

#ifdef ALN_STATS
cudaError_t debug_stats(unsigned long long *out, int reset) {
    cudaError_t e = cudaMemcpyFromSymbol(out, g_stats, sizeof(g_stats));
    if (e == cudaSuccess && reset) {
        unsigned long long z[16] = {};
        e = cudaMemcpyToSymbol(g_stats, z, sizeof(z));
    }
    return e;
}
#endif

// D-array pre-pass.  Thread t runs the greedy D scan of strand t & 1 of read
// t >> 1 on that strand's other index (strand 0 on X, strand 1 on X reversed)
// and stores its breakpoints; reads the search would flag before any scan get
// zeros.  The persistent search then starts from these instead of scanning.
__global__ void __launch_bounds__(kThreads) aln_dscan_kernel(DIndex X, ReadBatch rb, uint32_t n, SearchParams p,
                                                             uint2 *dbp) {
    __shared__ uint32_t s_bases[kReadWords * kThreads];
    __shared__ uint32_t s_nmask[kMaskWords * kThreads];
    const uint64_t t = static_cast<uint64_t>(blockIdx.x) * kThreads + threadIdx.x;
    if (t >= 2ull * n) return;
    const uint32_t r = static_cast<uint32_t>(t >> 1), s = static_cast<uint32_t>(t & 1u);
    const uint32_t m = rb.len[r];
    const uint32_t z = rb.z ? rb.z[r] : p.z;
    uint2 out = make_uint2(0u, 0u);
    if (m >= 1 && m <= ALN_MAX_READ_LEN && z <= ALN_MAX_Z && z <= p.z) {
        uint32_t *sb = s_bases + threadIdx.x, *sn = s_nmask + threadIdx.x;
        load_read(rb, rb.offset[r], m, sb, sn);
        const ReadView rv{sb, sn};
        d_scan(X.t[s], rv, m, s, min(z + 1, 8u), out.x, out.y);
    }
    dbp[t] = out;
}

// Visit order for the persistent search: reads by decreasing lower bound
// D(0) = min over strands (0..8), so that the lanes of a warp tend to run the
// same number of deepening passes.  Counting sort in two launches; the order
// inside one bound is arbitrary (a read's result does not depend on it).
constexpr uint32_t kOrderBins = 16;

__device__ __forceinline__ uint32_t order_key(const uint2 *dbp, uint32_t r) {
    const uint2 a = dbp[2ull * r], b = dbp[2ull * r + 1];
    return min(d_at(a.x, a.y, 0), d_at(b.x, b.y, 0));
}

__global__ void aln_order_count_kernel(const uint2 *dbp, uint32_t n, uint32_t *counts) {
    __shared__ uint32_t h[kOrderBins];
    if (threadIdx.x < kOrderBins) h[threadIdx.x] = 0;
    __syncthreads();
    for (uint64_t r = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; r < n;
         r += static_cast<uint64_t>(gridDim.x) * blockDim.x)
        atomicAdd(&h[order_key(dbp, static_cast<uint32_t>(r))], 1u);
    __syncthreads();
    if (threadIdx.x < kOrderBins && h[threadIdx.x]) atomicAdd(&counts[threadIdx.x], h[threadIdx.x]);
}

__global__ void aln_order_scatter_kernel(const uint2 *dbp, uint32_t n, const uint32_t *counts, uint32_t *cursor,
                                         uint32_t *order) {
    __shared__ uint32_t first[kOrderBins];
    if (threadIdx.x == 0) {
        uint32_t acc = 0;
        for (int k = kOrderBins - 1; k >= 0; k--) {  // largest bound first
            first[k] = acc;
            acc += counts[k];
        }
    }
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31u;
    for (uint64_t r = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; r < n;
         r += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        const uint32_t key = order_key(dbp, static_cast<uint32_t>(r));
        const unsigned grp = __match_any_sync(__activemask(), key);  // lanes with the same bound
        const uint32_t leader = __ffs(grp) - 1;
        uint32_t off = 0;
        if (lane == leader) off = atomicAdd(&cursor[key], static_cast<uint32_t>(__popc(grp)));
        off = __shfl_sync(grp, off, leader);
        order[first[key] + off + __popc(grp & ((1u << lane) - 1u))] = static_cast<uint32_t>(r);
    }
}

int stack_cap_for(uint32_t z) { return z <= 2 ? 19 : (z <= 4 ? 37 : 64); }

template <int CAP, int SMEM>
static cudaError_t launch_cap(const DIndex &X, const ReadBatch &rb, uint32_t n, const SearchParams &p,
                              aln_read_result *res, aln_hit *hits, uint32_t mode, uint32_t *queue,
                              void *scratch, cudaStream_t st) {
    if (mode == ALN_MODE_PLAIN) {
        const uint32_t blocks = (n + kThreads - 1) / kThreads;
        aln_plain_kernel<CAP><<<blocks, kThreads, 0, st>>>(X, rb, n, p, res, hits);
    } else {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, aln_persistent_kernel<CAP, SMEM>, kThreads, 0);
        if (p.blocks_per_sm && static_cast<int>(p.blocks_per_sm) < per_sm) per_sm = p.blocks_per_sm;
        if (per_sm < 1) per_sm = 1;
        uint32_t blocks = static_cast<uint32_t>(sms * per_sm);
        const uint32_t need = (n + kThreads - 1) / kThreads;
        if (blocks > need) blocks = need ? need : 1;
        cudaMemsetAsync(queue, 0, sizeof(uint32_t), st);
        uint2 *dbp = nullptr;
        uint32_t *order = nullptr;
        if (scratch) {  // D pre-pass and visit order (layout: search_scratch_bytes)
            uint32_t *counts = static_cast<uint32_t *>(scratch), *cursor = counts + kOrderBins;
            dbp = reinterpret_cast<uint2 *>(static_cast<char *>(scratch) + 256);
            order = reinterpret_cast<uint32_t *>(static_cast<char *>(scratch) + 256 + 16ull * n);
            cudaMemsetAsync(scratch, 0, 2 * kOrderBins * sizeof(uint32_t), st);
            aln_dscan_kernel<<<static_cast<unsigned>((2ull * n + kThreads - 1) / kThreads), kThreads, 0, st>>>(
                X, rb, n, p, dbp);
            const uint32_t ob = min((n + 255u) / 256u, static_cast<uint32_t>(sms) * 8u);
            aln_order_count_kernel<<<ob, 256, 0, st>>>(dbp, n, counts);
            aln_order_scatter_kernel<<<ob, 256, 0, st>>>(dbp, n, counts, cursor, order);
        }
        aln_persistent_kernel<CAP, SMEM><<<blocks, kThreads, 0, st>>>(X, rb, n, p, res, hits, queue, order, dbp);
    }
    return cudaGetLastError();
}

// Resident blocks per SM of the persistent kernel for limit z and a shared-memory
// stack of smem entries per lane (occupancy).
template <int SMEM>
static int max_blocks_smem(uint32_t z) {
    int per_sm = 0;
    switch (stack_cap_for(z)) {
        case 19: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, aln_persistent_kernel<19, SMEM>, kThreads, 0); break;
        case 37: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, aln_persistent_kernel<37, SMEM>, kThreads, 0); break;
        default: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, aln_persistent_kernel<64, SMEM>, kThreads, 0); break;
    }
    return per_sm;
}

int persistent_max_blocks(uint32_t z, uint32_t smem) {
    switch (smem) {
        case 4: return max_blocks_smem<4>(z);
        case 12: return max_blocks_smem<12>(z);
        default: return max_blocks_smem<8>(z);
    }
}

// Shared-memory stack depths the persistent kernel is compiled for.
bool smem_stack_supported(uint32_t smem) { return smem == 0 || smem == 4 || smem == 8 || smem == 12; }

// Bytes of the optional persistent-mode scratch for n reads: order-sort counters
// (256 B), D breakpoints (2 x 8 B per read), visit order (4 B per read).
uint64_t search_scratch_bytes(uint32_t n) { return 256ull + 20ull * n; }

template <int CAP>
static cudaError_t launch_smem(const DIndex &X, const ReadBatch &rb, uint32_t n, const SearchParams &p,
                               aln_read_result *res, aln_hit *hits, uint32_t mode, uint32_t *queue, void *scratch,
                               cudaStream_t st) {
    switch (p.smem_stack) {
        case 4: return launch_cap<CAP, 4>(X, rb, n, p, res, hits, mode, queue, scratch, st);
        case 12: return launch_cap<CAP, 12>(X, rb, n, p, res, hits, mode, queue, scratch, st);
        default: return launch_cap<CAP, kSmemStackDefault>(X, rb, n, p, res, hits, mode, queue, scratch, st);
    }
}

cudaError_t launch_search(const DIndex &X, const ReadBatch &rb, uint32_t n, const SearchParams &p,
                          aln_read_result *res, aln_hit *hits, uint32_t mode, uint32_t *queue, void *scratch,
                          cudaStream_t st) {
    if (p.status) {
        const cudaError_t e = cudaMemsetAsync(p.status, 0, sizeof(uint32_t), st);
        if (e != cudaSuccess) return e;
    }
    if (n == 0) return cudaSuccess;
    switch (stack_cap_for(p.z)) {
        case 19: return launch_smem<19>(X, rb, n, p, res, hits, mode, queue, scratch, st);
        case 37: return launch_smem<37>(X, rb, n, p, res, hits, mode, queue, scratch, st);
        default: return launch_smem<64>(X, rb, n, p, res, hits, mode, queue, scratch, st);
    }
}

}  // namespace aln
