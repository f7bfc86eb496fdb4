// C ABI: device index image, search dispatch and the SA-to-position walk.
#include <cuda_runtime.h>

#include <atomic>
#include <cstring>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "aln_device.cuh"
#include "aln_internal.h"
#include "aln_scan.cuh"
#include "aln_search.cuh"

namespace aln {
int persistent_max_blocks(uint32_t z, uint32_t smem);
bool smem_stack_supported(uint32_t smem);
cudaError_t launch_search(const DIndex &X, const ReadBatch &rb, uint32_t n, const SearchParams &p,
                          aln_read_result *res, aln_hit *hits, uint32_t mode, uint32_t *queue, void *scratch,
                          cudaStream_t st);
uint64_t search_scratch_bytes(uint32_t n);
}

using namespace aln;

static constexpr int kQueueSlots = 1024;    // counters handed to uncaptured calls in turn
static constexpr int kCaptureSlots = 1024;  // counters reserved one per captured call

struct fm_dindex {
    int device = 0;
    DIndex X{};
    fm_index_info_t info{};
    void *mem[2][3] = {{nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr}};
    void *kmer_all = nullptr;             // prefix-trie tables of both texts, one buffer (L2 window)
    uint64_t kmer_bytes = 0;
    uint32_t *queues = nullptr;           // persistent-mode queue counters: ring, then reserved
    std::atomic<uint32_t> next_queue{0};
    std::atomic<uint32_t> next_capture{0};
    cudaMemPool_t pool = nullptr;         // stream-ordered per-call scratch (D pre-pass, visit order)
};

// Search parameters from the ABI struct; ALN_OK or ALN_EINVAL with a message.
static int search_params(const char *who, const aln_params &P, uint32_t n_reads, SearchParams &sp) {
    if (P.z > ALN_MAX_Z) return fail(ALN_EINVAL, std::string(who) + ": z > ALN_MAX_Z");
    if (P.hit_cap < 1) return fail(ALN_EINVAL, std::string(who) + ": hit_cap must be >= 1");
    if (P.mode > ALN_MODE_PERSISTENT || P.strata > ALN_STRATA_SCORE)
        return fail(ALN_EINVAL, std::string(who) + ": bad mode or strata");
    if (P.strata == ALN_STRATA_SCORE && P.mode != ALN_MODE_PERSISTENT)
        return fail(ALN_EINVAL, std::string(who) + ": the score-ordered mode needs the persistent form");
    if (!smem_stack_supported(P.smem_stack))
        return fail(ALN_EINVAL, std::string(who) + ": smem_stack must be 0 or one of ALN_SMEM_STACK_CHOICES");
    sp.z = P.z;
    sp.max_gapo = P.max_gapo;
    sp.max_gape = P.max_gape;
    sp.seed_len = P.seed_len;
    sp.seed_z = P.seed_z;
    sp.e = P.indel_end_skip;
    sp.hit_cap = P.hit_cap;
    sp.strata = P.strata;
    sp.work_limit = P.work_limit ? P.work_limit : kDefaultWorkLimit;
    sp.blocks_per_sm = P.blocks_per_sm;
    sp.smem_stack = P.smem_stack;
    sp.help_after = P.help_after ? P.help_after : kDefaultHelpAfter;
    sp.heavy_after = P.heavy_after ? P.heavy_after : kDefaultHeavyAfter;
    sp.sc_mm = P.score_mm ? P.score_mm : 3;
    sp.sc_go = P.score_gapo ? P.score_gapo : 11;
    sp.sc_ge = P.score_gape ? P.score_gape : 4;
    sp.max_best = P.max_best;
    sp.heavy.hdr = nullptr;
    if (P.l2_window > 1) return fail(ALN_EINVAL, std::string(who) + ": l2_window must be 0 or 1");
    sp.window_base = nullptr;
    sp.window_bytes = 0;
    if (P.loop_limit) {
        sp.loop_limit = P.loop_limit;
    } else {  // 64 * n_reads * (576 + work_limit), saturating at 2^62
        const unsigned long long cap = 1ull << 62, per = 64ull * (576ull + sp.work_limit);
        sp.loop_limit = (n_reads && per > cap / n_reads) ? cap : per * (n_reads ? n_reads : 1);
    }
    sp.status = nullptr;
    return ALN_OK;
}

static void tune_forget(const fm_dindex *d);

static int cuda_fail(cudaError_t e, const char *what) {
    return fail(e == cudaErrorMemoryAllocation ? ALN_ENOMEM : ALN_EDEVICE,
                std::string(what) + ": " + cudaGetErrorString(e));
}

extern "C" void fm_dindex_free(fm_dindex *d) {
    if (!d) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(d->device);
    for (auto &row : d->mem)
        for (void *p : row)
            if (p) cudaFree(p);
    if (d->queues) cudaFree(d->queues);
    if (d->kmer_all) cudaFree(d->kmer_all);
    if (d->pool) cudaMemPoolDestroy(d->pool);
    cudaSetDevice(prev);
    tune_forget(d);
    delete d;
}

extern "C" int fm_index_to_device(const fm_index *idx, int device, void *stream, fm_dindex **out) {
    if (!idx || !out) return fail(ALN_EINVAL, "fm_index_to_device: null argument");
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return cuda_fail(e, "fm_index_to_device: no CUDA device");
    if (device < 0 || device >= ndev) return fail(ALN_EINVAL, "fm_index_to_device: bad device ordinal");
    int prev = 0;
    cudaGetDevice(&prev);
    if ((e = cudaSetDevice(device)) != cudaSuccess) return cuda_fail(e, "fm_index_to_device: cudaSetDevice");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    fm_dindex *d = new fm_dindex();
    d->device = device;
    fm_index_info(idx, &d->info);
    d->X.kmer_k = idx->kmer_k;
    uint32_t sh = 0;
    while ((1u << sh) < idx->sa_sample) sh++;
    d->X.sa_shift = sh;
    int rc = ALN_OK;
    // both prefix-trie tables in one buffer, so that one L2 access-policy window covers them
    d->kmer_bytes = (idx->t[0].kmer.size() + idx->t[1].kmer.size()) * 4;
    if (d->kmer_bytes) {
        if ((e = cudaMalloc(&d->kmer_all, d->kmer_bytes)) != cudaSuccess) rc = cuda_fail(e, "fm_index_to_device: cudaMalloc");
        for (int w = 0; w < 2 && rc == ALN_OK; w++) {
            char *dst = static_cast<char *>(d->kmer_all) + (w ? idx->t[0].kmer.size() * 4 : 0);
            if ((e = cudaMemcpyAsync(dst, idx->t[w].kmer.data(), idx->t[w].kmer.size() * 4, cudaMemcpyHostToDevice,
                                     st)) != cudaSuccess)
                rc = cuda_fail(e, "fm_index_to_device: copy");
        }
    }
    for (int w = 0; w < 2 && rc == ALN_OK; w++) {
        const HostText &T = idx->t[w];
        const void *src[3] = {T.blocks.data(), T.sa_samp.data(), nullptr};
        const size_t bytes[3] = {T.blocks.size() * 4, T.sa_samp.size() * 4, 0};
        for (int a = 0; a < 3 && rc == ALN_OK; a++) {
            if (!bytes[a]) continue;
            if ((e = cudaMalloc(&d->mem[w][a], bytes[a])) != cudaSuccess) rc = cuda_fail(e, "fm_index_to_device: cudaMalloc");
            else if ((e = cudaMemcpyAsync(d->mem[w][a], src[a], bytes[a], cudaMemcpyHostToDevice, st)) != cudaSuccess)
                rc = cuda_fail(e, "fm_index_to_device: copy");
        }
        DText &D = d->X.t[w];
        D.blocks = static_cast<const uint4 *>(d->mem[w][0]);
        D.sa_samp = static_cast<const uint32_t *>(d->mem[w][1]);
        D.kmer = d->kmer_bytes ? reinterpret_cast<const uint2 *>(static_cast<const char *>(d->kmer_all) +
                                                                (w ? idx->t[0].kmer.size() * 4 : 0))
                               : nullptr;
        for (int c = 0; c < 4; c++) D.C1[c] = static_cast<uint32_t>(T.C[c] + 1);
        D.C1[4] = static_cast<uint32_t>(T.n + 1);
        D.primary = static_cast<uint32_t>(T.primary);
        D.n = static_cast<uint32_t>(T.n);
    }
    if (rc == ALN_OK) {
        const size_t qbytes = (kQueueSlots + kCaptureSlots) * sizeof(uint32_t);
        if ((e = cudaMalloc(&d->queues, qbytes)) != cudaSuccess)
            rc = cuda_fail(e, "fm_index_to_device: cudaMalloc");
        else if ((e = cudaMemsetAsync(d->queues, 0, qbytes, st)) != cudaSuccess)
            rc = cuda_fail(e, "fm_index_to_device: memset");
    }
    if (rc == ALN_OK) {  // optional: without a pool the search scans D in its own loop
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = device;
        if (cudaMemPoolCreate(&d->pool, &props) == cudaSuccess) {
            uint64_t keep = ~0ull;  // keep freed scratch for the next call
            cudaMemPoolSetAttribute(d->pool, cudaMemPoolAttrReleaseThreshold, &keep);
        } else {
            cudaGetLastError();
            d->pool = nullptr;
        }
    }
    if (rc == ALN_OK && (e = cudaStreamSynchronize(st)) != cudaSuccess) rc = cuda_fail(e, "fm_index_to_device: sync");
    cudaSetDevice(prev);
    if (rc != ALN_OK) {
        fm_dindex_free(d);
        return rc;
    }
    *out = d;
    return ALN_OK;
}

extern "C" int fm_dindex_info(const fm_dindex *d, fm_index_info_t *info) {
    if (!d || !info) return fail(ALN_EINVAL, "fm_dindex_info: null argument");
    *info = d->info;
    return ALN_OK;
}

extern "C" uint64_t aln_search_scratch_bytes(uint32_t n_reads) { return search_scratch_bytes(n_reads); }

// The L2 access-policy window over the prefix-trie tables of both texts: at most
// the device's largest window, and the context's persisting-L2 set-aside raised
// to that size if it is smaller (a limit of this process's context).
static int l2_window_for(fm_dindex *d, SearchParams &sp) {
    static std::mutex mu;
    static uint64_t set_aside[64] = {};
    int max_window = 0, max_persist = 0;
    cudaDeviceGetAttribute(&max_window, cudaDevAttrMaxAccessPolicyWindowSize, d->device);
    cudaDeviceGetAttribute(&max_persist, cudaDevAttrMaxPersistingL2CacheSize, d->device);
    if (max_window <= 0 || max_persist <= 0) return ALN_OK;  // not supported: no window
    uint64_t bytes = d->kmer_bytes;
    if (bytes > static_cast<uint64_t>(max_window)) bytes = static_cast<uint64_t>(max_window);
    const uint64_t want = bytes < static_cast<uint64_t>(max_persist) ? bytes : static_cast<uint64_t>(max_persist);
    if (d->device >= 0 && d->device < 64) {
        std::lock_guard<std::mutex> lock(mu);
        if (set_aside[d->device] < want) {
            const cudaError_t e = cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, want);
            if (e != cudaSuccess) return cuda_fail(e, "aln_search: persisting L2 set-aside");
            set_aside[d->device] = want;
        }
        sp.window_base = d->kmer_all;
        sp.window_bytes = bytes;
        sp.window_hit_ratio = static_cast<float>(static_cast<double>(set_aside[d->device]) / static_cast<double>(bytes));
        if (sp.window_hit_ratio > 1.0f) sp.window_hit_ratio = 1.0f;
    }
    return ALN_OK;
}

extern "C" int aln_search(const fm_dindex *idx, const aln_batch *batch, uint32_t n_reads, const aln_params *params,
                          aln_result *out, void *stream) {
    if (!idx || !batch || !params || !out) return fail(ALN_EINVAL, "aln_search: null argument");
    if (n_reads && (!batch->bases || !batch->offset || !batch->len || !out->reads || !out->hits))
        return fail(ALN_EINVAL, "aln_search: null batch or result array");
    const aln_params &P = *params;
    SearchParams sp;
    int rc = search_params("aln_search", P, n_reads, sp);
    if (rc != ALN_OK) return rc;
    sp.status = out->status;
    const bool own_scratch = out->scratch && out->scratch_bytes >= search_scratch_bytes(n_reads);
    if (out->scratch && !own_scratch) return fail(ALN_EINVAL, "aln_search: scratch smaller than aln_search_scratch_bytes");
    if (own_scratch && reinterpret_cast<uintptr_t>(out->scratch) % 256)
        return fail(ALN_EINVAL, "aln_search: scratch must be 256-byte aligned");
    ReadBatch rb{batch->bases, batch->nmask, batch->offset, batch->len, batch->z};
    fm_dindex *d = const_cast<fm_dindex *>(idx);
    int prev = 0;
    cudaGetDevice(&prev);
    if (prev != idx->device) cudaSetDevice(idx->device);
    if (P.l2_window && P.mode == ALN_MODE_PERSISTENT && d->kmer_bytes) {
        rc = l2_window_for(d, sp);
        if (rc != ALN_OK) {
            if (prev != idx->device) cudaSetDevice(prev);
            return rc;
        }
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusActive;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
        cudaGetLastError();
        cs = cudaStreamCaptureStatusActive;
    }
    const bool capturing = cs != cudaStreamCaptureStatusNone;
    // Queue counter: uncaptured calls take the ring's next one; a captured call
    // keeps one of its own for every replay of its graph.
    uint32_t *queue = nullptr;
    if (P.mode == ALN_MODE_PERSISTENT && capturing) {
        const uint32_t c = d->next_capture.fetch_add(1);
        if (c >= static_cast<uint32_t>(kCaptureSlots)) {
            if (prev != idx->device) cudaSetDevice(prev);
            return fail(ALN_ELIMIT, "aln_search: every queue counter reserved for captured searches is in use");
        }
        queue = d->queues + kQueueSlots + c;
    } else {
        queue = d->queues + (d->next_queue.fetch_add(1) % kQueueSlots);
    }
    // Persistent mode: the D pre-pass and visit order need scratch; the caller's,
    // else a block of the index's pool ordered on the stream (not while capturing).
    // Without scratch the search scans D itself and visits reads in input order:
    // same results.
    void *scratch = nullptr;
    bool pooled = false;
    if (P.mode == ALN_MODE_PERSISTENT && n_reads) {
        if (own_scratch) {
            scratch = out->scratch;
        } else if (d->pool && !capturing) {
            if (cudaMallocFromPoolAsync(&scratch, search_scratch_bytes(n_reads), d->pool, st) == cudaSuccess) {
                pooled = true;
            } else {
                cudaGetLastError();
                scratch = nullptr;
            }
        }
    }
    cudaError_t e = launch_search(idx->X, rb, n_reads, sp, out->reads, out->hits, P.mode, queue, scratch, st);
    if (pooled) cudaFreeAsync(scratch, st);
    if (prev != idx->device) cudaSetDevice(prev);
    if (e != cudaSuccess) return cuda_fail(e, "aln_search: launch");
    return ALN_OK;
}

// ---------------------------------------------------------------- autotuner

namespace {
// Autotuner choices, cached per (index, sample size, limits).
struct TuneKey {
    const fm_dindex *idx;
    uint32_t n;
    uint8_t z, gapo, gape, seed_len, seed_z, e, hit_cap, strata;
    uint32_t work_limit;
    const void *zarr;
    bool operator==(const TuneKey &o) const { return std::memcmp(this, &o, sizeof(TuneKey)) == 0; }
};
struct TuneVal {
    uint8_t blocks, smem;
    uint32_t help_after;
    float ms;
};
std::mutex g_tune_mu;
std::vector<std::pair<TuneKey, TuneVal>> g_tune_cache;
}  // namespace

static void tune_forget(const fm_dindex *d) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    std::vector<std::pair<TuneKey, TuneVal>> keep;
    for (auto &kv : g_tune_cache)
        if (kv.first.idx != d) keep.push_back(kv);
    g_tune_cache.swap(keep);
}

extern "C" int aln_autotune(const fm_dindex *idx, const aln_batch *sample, uint32_t n_reads, aln_params *params,
                            aln_result *scratch, void *stream, float *best_ms) {
    if (!idx || !sample || !params || !scratch || !n_reads)
        return fail(ALN_EINVAL, "aln_autotune: null argument or empty sample");
    TuneKey key;
    std::memset(&key, 0, sizeof key);
    key.idx = idx;
    key.n = n_reads;
    key.z = params->z; key.gapo = params->max_gapo; key.gape = params->max_gape;
    key.seed_len = params->seed_len; key.seed_z = params->seed_z; key.e = params->indel_end_skip;
    key.hit_cap = params->hit_cap; key.strata = params->strata;
    key.work_limit = params->work_limit;
    key.zarr = sample->z ? static_cast<const void *>(sample->z) : nullptr;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        for (auto &kv : g_tune_cache)
            if (kv.first == key) {
                params->blocks_per_sm = kv.second.blocks;
                params->smem_stack = kv.second.smem;
                params->help_after = kv.second.help_after;
                if (best_ms) *best_ms = kv.second.ms;
                return ALN_OK;
            }
    }
    int prev = 0;
    cudaGetDevice(&prev);
    if (prev != idx->device) cudaSetDevice(idx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    aln_params p = *params;
    p.mode = ALN_MODE_PERSISTENT;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int rc = ALN_OK, best_b = 0, best_s = 0;
    const uint32_t best_h = params->help_after;
    float best = 0;
    auto timed = [&](float *ms) {
        cudaEventRecord(e0, st);
        int r = aln_search(idx, sample, n_reads, &p, scratch, stream);
        cudaEventRecord(e1, st);
        if (r == ALN_OK && cudaEventSynchronize(e1) != cudaSuccess) r = fail(ALN_EDEVICE, "aln_autotune: search failed");
        *ms = 0;
        cudaEventElapsedTime(ms, e0, e1);
        return r;
    };
    // resident blocks per SM x shared-memory stack depth (help_after and heavy_after
    // stay as given: lanes that help a read early keep its owner's expansion
    // count below heavy_after, and a heavy read then never reaches the heavy
    // phase).  A sample's time varies from run to run once its tail goes to the
    // heavy phase, so every candidate is timed twice and counts by its slower
    // run, and the default (every block that fits, 8 stack entries) is kept
    // unless a candidate beats it by more than 5 %.
    auto timed2 = [&](float *ms) {
        float a = 0, b = 0;
        int r = timed(&a);
        if (r == ALN_OK) r = timed(&b);
        *ms = a > b ? a : b;
        return r;
    };
    static const int kSmem[] = ALN_SMEM_STACK_CHOICES;
    const int maxb_default = persistent_max_blocks(params->z, 8u);
    p.smem_stack = 8;
    p.blocks_per_sm = static_cast<uint8_t>(maxb_default > 0 ? maxb_default : 1);
    best_b = p.blocks_per_sm;
    best_s = 8;
    rc = aln_search(idx, sample, n_reads, &p, scratch, stream);  // warm-up
    if (rc == ALN_OK) rc = timed2(&best);
    const float default_ms = best;
    for (int smem : kSmem) {
        const int maxb = persistent_max_blocks(params->z, static_cast<uint32_t>(smem));
        p.smem_stack = static_cast<uint8_t>(smem);
        p.blocks_per_sm = static_cast<uint8_t>(maxb > 0 ? maxb : 1);
        if (rc == ALN_OK) rc = aln_search(idx, sample, n_reads, &p, scratch, stream);  // warm-up
        for (int b = 1; b <= maxb && rc == ALN_OK; b++) {
            if (smem == 8 && b == maxb_default) continue;  // the default, timed above
            p.blocks_per_sm = static_cast<uint8_t>(b);
            float ms = 0;
            rc = timed2(&ms);
            if (rc == ALN_OK && ms < 0.95f * default_ms && ms < best) {
                best = ms;
                best_b = b;
                best_s = smem;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (prev != idx->device) cudaSetDevice(prev);
    if (rc != ALN_OK) return rc;
    params->blocks_per_sm = static_cast<uint8_t>(best_b);
    params->smem_stack = static_cast<uint8_t>(best_s);
    params->help_after = best_h;
    if (best_ms) *best_ms = best;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache.push_back({key, TuneVal{static_cast<uint8_t>(best_b), static_cast<uint8_t>(best_s), best_h, best}});
    return ALN_OK;
}

// ---------------------------------------------------------------- sa_to_pos

namespace aln {

// One thread per (hit, row slot): SA value of row k + j by an LF walk to the
// nearest sampled row, then the forward-strand start of the target.
__global__ void sa_walk_kernel(DIndex X, const aln_hit *hits, uint32_t n_hits, uint32_t max_width,
                               uint64_t *pos_out, uint32_t *n_pos_out) {
    const uint64_t tid = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x;
    const uint64_t h = tid / max_width;
    const uint32_t j = static_cast<uint32_t>(tid % max_width);
    if (h >= n_hits) return;
    const aln_hit H = hits[h];
    if (H.strand > 1 || H.l < H.k || H.l > X.t[0].n) return;  // not a hit of this index
    const uint64_t width = static_cast<uint64_t>(H.l) - H.k + 1;
    if (width > max_width || j >= width) return;
    const DText &T = X.t[H.strand ? 0 : 1];
    const uint32_t mask = (1u << X.sa_shift) - 1u;
    const uint32_t limit = 64u << X.sa_shift;
    uint32_t row = H.k + j, steps = 0;
    uint64_t sa;
    bool ok = true;
    for (;;) {
        if ((row & mask) == 0) {
            sa = static_cast<uint64_t>(T.sa_samp[row >> X.sa_shift]) + steps;
            break;
        }
        if (row == T.primary) {  // SA[primary] = 0
            sa = steps;
            break;
        }
        if (steps >= limit) {
            ok = false;
            sa = 0;
            break;
        }
        row = lf_row(T, row);
        steps++;
    }
    uint64_t p = H.strand ? sa : static_cast<uint64_t>(T.n) - sa - H.aligned_len;
    pos_out[h * max_width + j] = ok ? p : ~0ull;
    if (!ok) n_pos_out[h] = ALN_POS_WALK_LIMIT;  // racing writers store the same value
}

// One thread per hit: width flag and ascending order of its positions.
__global__ void sa_sort_kernel(const aln_hit *hits, uint32_t n_hits, uint32_t max_width, uint32_t n_text,
                               uint64_t *pos_out, uint32_t *n_pos_out) {
    const uint32_t h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= n_hits) return;
    const aln_hit H = hits[h];
    if (H.strand > 1 || H.l < H.k || H.l > n_text) {
        n_pos_out[h] = ALN_POS_BAD_HIT;
        return;
    }
    const uint64_t width = static_cast<uint64_t>(H.l) - H.k + 1;
    if (width > max_width) {
        n_pos_out[h] = ALN_POS_TOO_WIDE;
        return;
    }
    if (n_pos_out[h] == ALN_POS_WALK_LIMIT) return;
    uint64_t *p = pos_out + static_cast<uint64_t>(h) * max_width;
    for (uint32_t a = 1; a < width; a++) {  // insertion sort, width <= 64
        uint64_t v = p[a];
        uint32_t b = a;
        while (b > 0 && p[b - 1] > v) {
            p[b] = p[b - 1];
            b--;
        }
        p[b] = v;
    }
    n_pos_out[h] = static_cast<uint32_t>(width);
}

}  // namespace aln

extern "C" int sa_to_pos(const fm_dindex *idx, const aln_hit *hits, uint32_t n_hits, uint32_t max_width,
                         uint64_t *pos_out, uint32_t *n_pos_out, void *stream) {
    if (!idx || (n_hits && (!hits || !pos_out || !n_pos_out))) return fail(ALN_EINVAL, "sa_to_pos: null argument");
    if (max_width < 1 || max_width > 64) return fail(ALN_EINVAL, "sa_to_pos: max_width must be 1..64");
    if (!n_hits) return ALN_OK;
    int prev = 0;
    cudaGetDevice(&prev);
    if (prev != idx->device) cudaSetDevice(idx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaMemsetAsync(n_pos_out, 0, n_hits * sizeof(uint32_t), st);
    const uint64_t threads = static_cast<uint64_t>(n_hits) * max_width;
    sa_walk_kernel<<<static_cast<unsigned>((threads + 255) / 256), 256, 0, st>>>(idx->X, hits, n_hits, max_width,
                                                                                 pos_out, n_pos_out);
    sa_sort_kernel<<<(n_hits + 255) / 256, 256, 0, st>>>(hits, n_hits, max_width, idx->X.t[0].n, pos_out,
                                                         n_pos_out);
    cudaError_t e = cudaGetLastError();
    if (prev != idx->device) cudaSetDevice(prev);
    if (e != cudaSuccess) return cuda_fail(e, "sa_to_pos: launch");
    return ALN_OK;
}

// ---------------------------------------------------------------- aln_compact_hits

namespace aln {

__global__ void hit_count_kernel(const aln_read_result *reads, uint32_t n, uint32_t *offsets) {
    for (uint64_t r = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; r <= n;
         r += static_cast<uint64_t>(gridDim.x) * blockDim.x)
        offsets[r] = r < n ? reads[r].n_hits : 0u;
}

// One thread per read: its written hits to their place in the dense array.
__global__ void hit_gather_kernel(const aln_read_result *reads, const aln_hit *hits, uint32_t n, uint32_t hit_cap,
                                  const uint32_t *offsets, aln_hit *dense, uint64_t dense_cap) {
    for (uint64_t r = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; r < n;
         r += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        const uint32_t k = reads[r].n_hits < hit_cap ? reads[r].n_hits : hit_cap;
        const uint64_t o = offsets[r];
        for (uint32_t t = 0; t < k && o + t < dense_cap; t++) dense[o + t] = hits[r * hit_cap + t];
    }
}

}  // namespace aln

extern "C" uint64_t aln_compact_scratch_bytes(uint32_t n_reads) {
    return 4ull * scan::scan_temp_words(static_cast<uint64_t>(n_reads) + 1);
}

extern "C" int aln_compact_hits(const aln_read_result *reads, const aln_hit *hits, uint32_t n_reads, uint32_t hit_cap,
                                uint32_t *offsets, aln_hit *dense, uint64_t dense_cap, void *scratch,
                                uint64_t scratch_bytes, void *stream) {
    if (!offsets || (n_reads && (!reads || !hits)) || (dense_cap && !dense) || !scratch)
        return fail(ALN_EINVAL, "aln_compact_hits: null argument");
    if (hit_cap < 1 || hit_cap > ALN_MAX_HIT_CAP) return fail(ALN_EINVAL, "aln_compact_hits: hit_cap must be 1..255");
    if (scratch_bytes < aln_compact_scratch_bytes(n_reads))
        return fail(ALN_EINVAL, "aln_compact_hits: scratch smaller than aln_compact_scratch_bytes");
    if (static_cast<uint64_t>(n_reads) * hit_cap > 0xFFFFFFFFull)
        return fail(ALN_EINVAL, "aln_compact_hits: n_reads * hit_cap must be below 2^32");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const uint64_t m = static_cast<uint64_t>(n_reads) + 1;
    const unsigned g = static_cast<unsigned>((m + 255) / 256 < 65536 ? (m + 255) / 256 : 65536);
    hit_count_kernel<<<g, 256, 0, st>>>(reads, n_reads, offsets);
    scan::device_scan(offsets, offsets, m, false, static_cast<uint32_t *>(scratch), st, scan::OpAdd());
    if (n_reads)
        hit_gather_kernel<<<g, 256, 0, st>>>(reads, hits, n_reads, hit_cap, offsets, dense, dense_cap);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "aln_compact_hits: launch");
    return ALN_OK;
}

// ---------------------------------------------------------------- aln_search_noalloc
//
// The persistent search with its work-queue counter in a fixed, file-scope
// device array instead of memory the library allocated.  For callers that
// cannot call cudaMalloc (see the header).  Host code never dereferences the
// array's name: on the host it only stands in for the symbol, so its device
// address is looked up once per device with cudaGetSymbolAddress and that
// address is what the kernel receives.

namespace {
constexpr int kNoallocMaxDevices = 64;
static __device__ __align__(256) uint32_t g_noalloc_scratch[ALN_NOALLOC_SCRATCH_BYTES / sizeof(uint32_t)];
std::mutex g_noalloc_mu;
uint32_t *g_noalloc_ptr[kNoallocMaxDevices] = {};
}  // namespace

// Device address of the scratch array on the current device (set up on first use).
static int noalloc_scratch(int device, uint32_t **out) {
    if (device < 0 || device >= kNoallocMaxDevices)
        return fail(ALN_EINVAL, "aln_search_noalloc: device ordinal beyond the supported range");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return cuda_fail(e, "aln_search_noalloc: cudaGetSymbolAddress");
        g_noalloc_ptr[device] = static_cast<uint32_t *>(p);
    }
    *out = g_noalloc_ptr[device];
    return ALN_OK;
}

extern "C" int aln_search_noalloc(const fm_dindex *idx, const aln_batch *batch, uint32_t n_reads,
                                  const aln_params *params, aln_result *out, void *stream) {
    if (!idx || !batch || !params || !out) return fail(ALN_EINVAL, "aln_search_noalloc: null argument");
    if (n_reads > ALN_NOALLOC_MAX_READS)
        return fail(ALN_EINVAL, "aln_search_noalloc: n_reads exceeds ALN_NOALLOC_MAX_READS (the range of the "
                                "work-queue counter in the fixed scratch array)");
    if (n_reads && (!batch->bases || !batch->offset || !batch->len || !out->reads || !out->hits))
        return fail(ALN_EINVAL, "aln_search_noalloc: null batch or result array");
    aln_params P = *params;
    P.mode = ALN_MODE_PERSISTENT;  // the mode field is ignored
    SearchParams sp;
    int rc0 = search_params("aln_search_noalloc", P, n_reads, sp);
    if (rc0 != ALN_OK) return rc0;
    sp.status = out->status;
    ReadBatch rb{batch->bases, batch->nmask, batch->offset, batch->len, batch->z};
    int prev = 0;
    cudaGetDevice(&prev);
    if (prev != idx->device) cudaSetDevice(idx->device);
    uint32_t *scratch = nullptr;
    int rc = noalloc_scratch(idx->device, &scratch);
    if (rc == ALN_OK) {
        // launch_search clears the queue counter (scratch[0]) on the stream first
        cudaError_t e = launch_search(idx->X, rb, n_reads, sp, out->reads, out->hits, ALN_MODE_PERSISTENT, scratch, nullptr,
                                      static_cast<cudaStream_t>(stream));
        if (e != cudaSuccess) rc = cuda_fail(e, "aln_search_noalloc: launch");
    }
    if (prev != idx->device) cudaSetDevice(prev);
    return rc;
}

// ---------------------------------------------------------------- aln_gather_probe
//
// Random 64-byte block reads over a caller buffer: the denominator for the
// LF step's scattered block reads.  Four lanes read the four 16-byte quarters
// of one block, so one warp load instruction covers 8 blocks; each lane keeps
// kProbeInFlight loads outstanding before it consumes any.

namespace {
constexpr int kProbeThreads = 256;
constexpr int kProbeInFlight = 8;
constexpr uint32_t kProbeGathersPerWarpRound = 8u * kProbeInFlight;

// "lowbias32", a published 32-bit integer hash (two xorshift-multiply rounds).
__device__ __forceinline__ uint32_t lowbias32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

__global__ void __launch_bounds__(kProbeThreads) gather_probe_kernel(const uint4 *__restrict__ buf, uint32_t n_blocks,
                                                                     uint32_t n_gathers, uint32_t seed,
                                                                     uint32_t *sink) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t warp = (static_cast<uint64_t>(blockIdx.x) * kProbeThreads + threadIdx.x) >> 5;
    const uint64_t n_warps = (static_cast<uint64_t>(gridDim.x) * kProbeThreads) >> 5;
    const uint32_t salt = seed * 0x9E3779B9u;
    uint32_t acc = 0;
    for (uint64_t g0 = warp * kProbeGathersPerWarpRound; g0 < n_gathers; g0 += n_warps * kProbeGathersPerWarpRound) {
        uint4 v[kProbeInFlight];
#pragma unroll
        for (int u = 0; u < kProbeInFlight; u++) {
            const uint64_t g = g0 + 8u * u + (lane >> 2);
            v[u] = make_uint4(0u, 0u, 0u, 0u);
            if (g < n_gathers) {
                const uint32_t b = __umulhi(lowbias32(static_cast<uint32_t>(g) + salt), n_blocks);
                v[u] = ld_nc(buf + 4ull * b + (lane & 3u));
            }
        }
#pragma unroll
        for (int u = 0; u < kProbeInFlight; u++) acc ^= v[u].x ^ v[u].y ^ v[u].z ^ v[u].w;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) acc ^= __shfl_xor_sync(0xFFFFFFFFu, acc, o);
    if (lane == 0 && acc) atomicXor(sink, acc);
}

bool device_pointer(const void *p, int *device) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) return false;
    *device = a.device;
    return true;
}
}  // namespace

extern "C" int aln_gather_probe(const void *buf, uint64_t buf_bytes, uint64_t n_gathers, uint32_t seed,
                                uint32_t *sink, void *stream) {
    if (!buf || !sink) return fail(ALN_EINVAL, "aln_gather_probe: null argument");
    if (reinterpret_cast<uintptr_t>(buf) % 64) return fail(ALN_EINVAL, "aln_gather_probe: buf must be 64-byte aligned");
    const uint64_t n_blocks = buf_bytes / 64;
    if (n_blocks < 1 || n_blocks > 0xFFFFFFFFull)
        return fail(ALN_EINVAL, "aln_gather_probe: buf_bytes must be in [64, 2^38)");
    if (n_gathers > 0xFFFFFFFFull) return fail(ALN_EINVAL, "aln_gather_probe: n_gathers must be < 2^32");
    int dev = 0, dev_sink = 0;
    if (!device_pointer(buf, &dev) || !device_pointer(sink, &dev_sink) || dev != dev_sink)
        return fail(ALN_EINVAL, "aln_gather_probe: buf and sink must be device memory of one device");
    if (!n_gathers) return ALN_OK;
    int prev = 0;
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
    int sms = 0, occ = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, gather_probe_kernel, kProbeThreads, 0);
    const uint64_t per_block = static_cast<uint64_t>(kProbeThreads / 32) * kProbeGathersPerWarpRound;
    const uint64_t need = (n_gathers + per_block - 1) / per_block;
    const uint64_t full = static_cast<uint64_t>(sms > 0 ? sms : 1) * static_cast<uint64_t>(occ > 0 ? occ : 1);
    const unsigned grid = static_cast<unsigned>(need < full ? need : full);
    gather_probe_kernel<<<grid, kProbeThreads, 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const uint4 *>(buf), static_cast<uint32_t>(n_blocks), static_cast<uint32_t>(n_gathers), seed, sink);
    cudaError_t e = cudaGetLastError();
    if (prev != dev) cudaSetDevice(prev);
    if (e != cudaSuccess) return cuda_fail(e, "aln_gather_probe: launch");
    return ALN_OK;
}

#ifdef ALN_STATS
namespace aln {
cudaError_t debug_stats(unsigned long long *out, int reset);
}
// Instrumented builds only (not part of the ABI): counters of the persistent kernel.
extern "C" int aln_debug_stats(unsigned long long *out16, int reset) {
    cudaError_t e = aln::debug_stats(out16, reset);
    return e == cudaSuccess ? ALN_OK : cuda_fail(e, "aln_debug_stats");
}
#endif
