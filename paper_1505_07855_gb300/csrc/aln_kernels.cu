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

#include "aln_search.cuh"

namespace aln {

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

template <int STACK_CAP>
__global__ void __launch_bounds__(kThreads) aln_persistent_kernel(DIndex X, ReadBatch rb, uint32_t n_reads,
                                                                  SearchParams p, aln_read_result *res,
                                                                  aln_hit *hits, uint32_t *queue) {
    __shared__ uint32_t s_bases[kReadWords * kThreads];
    __shared__ uint32_t s_nmask[kMaskWords * kThreads];
    ReadView rv{s_bases + threadIdx.x, s_nmask + threadIdx.x};
    Search<STACK_CAP> S;
    // bounded: each iteration consumes one queue ticket, at most n_reads + grid
    for (uint32_t guard = 0; guard <= n_reads; guard++) {
        const uint32_t r = atomicAdd(queue, 1u);
        if (r >= n_reads) break;
        const uint32_t m = rb.len[r];
        const uint32_t z = rb.z ? rb.z[r] : p.z;
        if (m <= ALN_MAX_READ_LEN && m > 0) load_read(rb, rb.offset[r], m, s_bases + threadIdx.x, s_nmask + threadIdx.x);
        S.run(X, rv, m, z, p, res + r, hits + static_cast<uint64_t>(r) * p.hit_cap);
    }
}

int stack_cap_for(uint32_t z) { return z <= 2 ? 19 : (z <= 4 ? 37 : 64); }

template <int CAP>
static cudaError_t launch_cap(const DIndex &X, const ReadBatch &rb, uint32_t n, const SearchParams &p,
                              aln_read_result *res, aln_hit *hits, uint32_t mode, uint32_t *queue,
                              cudaStream_t st) {
    if (mode == ALN_MODE_PLAIN) {
        const uint32_t blocks = (n + kThreads - 1) / kThreads;
        aln_plain_kernel<CAP><<<blocks, kThreads, 0, st>>>(X, rb, n, p, res, hits);
    } else {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, aln_persistent_kernel<CAP>, kThreads, 0);
        if (per_sm < 1) per_sm = 1;
        uint32_t blocks = static_cast<uint32_t>(sms * per_sm);
        const uint32_t need = (n + kThreads - 1) / kThreads;
        if (blocks > need) blocks = need ? need : 1;
        cudaMemsetAsync(queue, 0, sizeof(uint32_t), st);
        aln_persistent_kernel<CAP><<<blocks, kThreads, 0, st>>>(X, rb, n, p, res, hits, queue);
    }
    return cudaGetLastError();
}

cudaError_t launch_search(const DIndex &X, const ReadBatch &rb, uint32_t n, const SearchParams &p,
                          aln_read_result *res, aln_hit *hits, uint32_t mode, uint32_t *queue, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    switch (stack_cap_for(p.z)) {
        case 19: return launch_cap<19>(X, rb, n, p, res, hits, mode, queue, st);
        case 37: return launch_cap<37>(X, rb, n, p, res, hits, mode, queue, st);
        default: return launch_cap<64>(X, rb, n, p, res, hits, mode, queue, st);
    }
}

}  // namespace aln
