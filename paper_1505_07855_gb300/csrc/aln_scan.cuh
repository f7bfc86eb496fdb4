// Device-wide scan (sum or max) of 32-bit words, written for this library:
// tiles of 4096 words, each reduced by one block, the tile reductions scanned
// recursively, then every tile scanned with its prefix.  Used by the GPU index
// builder and by the hit compaction.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace aln {
namespace scan {
namespace {  // each translation unit keeps its own copy of the kernels

constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr uint64_t kScanTile = static_cast<uint64_t>(kScanThreads) * kScanItems;

struct OpAdd {
    __device__ __forceinline__ uint32_t operator()(uint32_t a, uint32_t b) const { return a + b; }
};
struct OpMax {
    __device__ __forceinline__ uint32_t operator()(uint32_t a, uint32_t b) const { return a > b ? a : b; }
};

// Exclusive scan of one value per thread over the block; *total gets the block's
// reduction.  Identity 0 for both operators (values are unsigned).
template <class Op>
__device__ __forceinline__ uint32_t block_exclusive(uint32_t v, uint32_t *warp_tot, uint32_t *total, Op op) {
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    uint32_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xFFFFFFFFu, inc, o);
        if (lane >= static_cast<uint32_t>(o)) inc = op(inc, u);
    }
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const uint32_t nw = blockDim.x >> 5;
        uint32_t t = lane < nw ? warp_tot[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(0xFFFFFFFFu, t, o);
            if (lane >= static_cast<uint32_t>(o)) t = op(t, u);
        }
        if (lane < nw) warp_tot[lane] = t;  // inclusive over warps
    }
    __syncthreads();
    const uint32_t before = warp ? warp_tot[warp - 1] : 0u;
    const uint32_t excl_in_warp = __shfl_up_sync(0xFFFFFFFFu, inc, 1);
    const uint32_t mine = lane ? op(before, excl_in_warp) : before;
    if (total) *total = warp_tot[(blockDim.x >> 5) - 1];
    __syncthreads();
    return mine;
}

template <class Op>
__global__ void __launch_bounds__(kScanThreads) scan_reduce_kernel(const uint32_t *in, uint64_t n, uint32_t *partial, Op op) {
    __shared__ uint32_t wt[32];
    const uint64_t base = static_cast<uint64_t>(blockIdx.x) * kScanTile;
    uint32_t acc = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        const uint64_t j = base + static_cast<uint64_t>(i) * kScanThreads + threadIdx.x;
        if (j < n) acc = op(acc, in[j]);
    }
    uint32_t total = 0;
    block_exclusive(acc, wt, &total, op);
    if (threadIdx.x == 0) partial[blockIdx.x] = total;
}

// Scan of one tile: coalesced load into shared memory, 8 consecutive items per
// thread, block scan of the thread sums, coalesced store.  prefix: the
// exclusive scan of the tile reductions (nullptr: a single tile).
template <class Op>
__global__ void __launch_bounds__(kScanThreads) scan_tile_kernel(const uint32_t *in, uint32_t *out, uint64_t n,
                                                                 const uint32_t *prefix, bool inclusive, Op op) {
    __shared__ uint32_t s[kScanTile];
    __shared__ uint32_t wt[32];
    const uint64_t base = static_cast<uint64_t>(blockIdx.x) * kScanTile;
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        const uint32_t t = i * kScanThreads + threadIdx.x;
        const uint64_t j = base + t;
        s[t] = j < n ? in[j] : 0u;
    }
    __syncthreads();
    uint32_t v[kScanItems];
    uint32_t acc = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        v[i] = s[threadIdx.x * kScanItems + i];
        acc = op(acc, v[i]);
    }
    uint32_t run = block_exclusive(acc, wt, nullptr, op);
    if (prefix) run = op(prefix[blockIdx.x], run);
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        const uint32_t inc = op(run, v[i]);
        s[threadIdx.x * kScanItems + i] = inclusive ? inc : run;
        run = inc;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        const uint32_t t = i * kScanThreads + threadIdx.x;
        const uint64_t j = base + t;
        if (j < n) out[j] = s[t];
    }
}

// Scratch words a scan of n elements needs for its tile reductions (all levels).
inline uint64_t scan_temp_words(uint64_t n) {
    uint64_t w = 0;
    for (uint64_t t = (n + kScanTile - 1) / kScanTile; t > 1; t = (t + kScanTile - 1) / kScanTile) w += 2 * t;
    return w + 2;
}

// out = scan of in (in == out allowed), exclusive or inclusive, sum or max.
template <class Op>
inline void device_scan(const uint32_t *in, uint32_t *out, uint64_t n, bool inclusive, uint32_t *temp, cudaStream_t st,
                 Op op) {
    if (n == 0) return;
    const uint64_t tiles = (n + kScanTile - 1) / kScanTile;
    if (tiles == 1) {
        scan_tile_kernel<Op><<<1, kScanThreads, 0, st>>>(in, out, n, nullptr, inclusive, op);
        return;
    }
    uint32_t *partial = temp, *pre = temp + tiles;
    scan_reduce_kernel<Op><<<static_cast<unsigned>(tiles), kScanThreads, 0, st>>>(in, n, partial, op);
    device_scan(partial, pre, tiles, false, temp + 2 * tiles, st, op);
    scan_tile_kernel<Op><<<static_cast<unsigned>(tiles), kScanThreads, 0, st>>>(in, out, n, pre, inclusive, op);
}

}  // namespace
}  // namespace scan
}  // namespace aln
