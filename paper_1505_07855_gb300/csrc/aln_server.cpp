// Serving loop: continuous batching of read requests onto a resident index.
//
// A dispatcher thread keeps up to n_slots batches in flight.  Each slot is a
// fixed set of device buffers (sized at creation from the memory budget) with
// pinned host staging and its own CUDA stream.  Requests are queued on submit;
// whenever a slot is free the dispatcher fills it from the oldest requests
// (splitting a request that does not fit into several batches), packs the
// reads, and enqueues copy-in, one persistent aln_search and copy-out on the
// slot's stream.  Requests that arrive while batches run are taken into the
// next free slot, so batches overlap on the device.  When a slot's event has
// completed, its results are scattered to their requests; a request completes
// when all its reads are back.  A read's result depends only on the read and
// the index, so it is the same whatever batch it travels in.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "aln_gb300.h"
#include "aln_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t id = 0;
    uint32_t n = 0;
    std::vector<uint8_t> codes;
    std::vector<uint64_t> off;
    std::vector<uint16_t> len;
    std::vector<uint8_t> z;
    std::vector<aln_read_result> res;
    std::vector<aln_hit> hits;
    uint32_t next = 0;   // first read not yet given to a batch
    uint32_t done_reads = 0;
    bool done = false;
    Clock::time_point t_submit, t_done;
};

struct Chunk {
    std::shared_ptr<Request> req;
    uint32_t first = 0, count = 0, slot_first = 0;
};

struct Slot {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    // device
    uint32_t *d_bases = nullptr, *d_nmask = nullptr;
    uint64_t *d_off = nullptr;
    uint16_t *d_len = nullptr;
    uint8_t *d_z = nullptr;
    aln_read_result *d_res = nullptr;
    aln_hit *d_hits = nullptr;
    // pinned host
    uint32_t *h_bases = nullptr, *h_nmask = nullptr;
    uint64_t *h_off = nullptr;
    uint16_t *h_len = nullptr;
    uint8_t *h_z = nullptr;
    aln_read_result *h_res = nullptr;
    aln_hit *h_hits = nullptr;
    std::vector<Chunk> chunks;
    uint32_t n_reads = 0;
    bool busy = false;
};

}  // namespace

struct aln_server {
    const fm_dindex *idx = nullptr;
    aln_server_config cfg{};
    std::vector<Slot> slots;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Request>> pending;
    std::unordered_map<uint64_t, std::shared_ptr<Request>> live;
    std::vector<double> latencies_ms;
    uint64_t next_id = 1;
    uint64_t reads_done = 0, batches = 0;
    int error = ALN_OK;
    std::string error_msg;
    bool stop = false;
    std::thread worker;
    Clock::time_point t_start;
};

using aln::fail;

static size_t words16(uint64_t b) { return (b + 15) / 16; }
static size_t words32(uint64_t b) { return (b + 31) / 32; }

static void free_slot(Slot &s) {
    cudaFree(s.d_bases); cudaFree(s.d_nmask); cudaFree(s.d_off); cudaFree(s.d_len); cudaFree(s.d_z);
    cudaFree(s.d_res); cudaFree(s.d_hits);
    cudaFreeHost(s.h_bases); cudaFreeHost(s.h_nmask); cudaFreeHost(s.h_off); cudaFreeHost(s.h_len);
    cudaFreeHost(s.h_z); cudaFreeHost(s.h_res); cudaFreeHost(s.h_hits);
    if (s.ev) cudaEventDestroy(s.ev);
    if (s.st) cudaStreamDestroy(s.st);
}

static bool alloc_slot(Slot &s, const aln_server_config &c) {
    const uint64_t R = c.max_batch_reads, Bs = c.max_batch_bases, H = c.params.hit_cap;
    bool ok = cudaStreamCreateWithFlags(&s.st, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming) == cudaSuccess &&
              cudaMalloc(&s.d_bases, words16(Bs) * 4) == cudaSuccess &&
              cudaMalloc(&s.d_nmask, words32(Bs) * 4) == cudaSuccess &&
              cudaMalloc(&s.d_off, R * 8) == cudaSuccess && cudaMalloc(&s.d_len, R * 2) == cudaSuccess &&
              cudaMalloc(&s.d_z, R) == cudaSuccess && cudaMalloc(&s.d_res, R * sizeof(aln_read_result)) == cudaSuccess &&
              cudaMalloc(&s.d_hits, R * H * sizeof(aln_hit)) == cudaSuccess &&
              cudaMallocHost(&s.h_bases, words16(Bs) * 4) == cudaSuccess &&
              cudaMallocHost(&s.h_nmask, words32(Bs) * 4) == cudaSuccess &&
              cudaMallocHost(&s.h_off, R * 8) == cudaSuccess && cudaMallocHost(&s.h_len, R * 2) == cudaSuccess &&
              cudaMallocHost(&s.h_z, R) == cudaSuccess &&
              cudaMallocHost(&s.h_res, R * sizeof(aln_read_result)) == cudaSuccess &&
              cudaMallocHost(&s.h_hits, R * H * sizeof(aln_hit)) == cudaSuccess;
    return ok;
}

static uint64_t slot_bytes(const aln_server_config &c) {
    const uint64_t R = c.max_batch_reads, Bs = c.max_batch_bases, H = c.params.hit_cap;
    return words16(Bs) * 4 + words32(Bs) * 4 + R * (8 + 2 + 1 + sizeof(aln_read_result) + H * sizeof(aln_hit));
}

// Pack the chunk list of a slot into its pinned buffers; returns the bases used.
static uint64_t pack_slot(Slot &s, const aln_server_config &c) {
    uint64_t j = 0;
    uint32_t r = 0;
    for (Chunk &ch : s.chunks) {
        ch.slot_first = r;
        const Request &q = *ch.req;
        for (uint32_t t = ch.first; t < ch.first + ch.count; t++, r++) {
            s.h_off[r] = j;
            s.h_len[r] = q.len[t];
            s.h_z[r] = q.z.empty() ? c.params.z : q.z[t];
            const uint8_t *cd = q.codes.data() + q.off[t];
            const uint32_t L = q.len[t];
            for (uint32_t u = 0; u < L; u++, j++) {
                if ((j & 15) == 0) s.h_bases[j >> 4] = 0;
                if ((j & 31) == 0) s.h_nmask[j >> 5] = 0;
                uint32_t b = cd[u];
                if (b > 3) {
                    s.h_nmask[j >> 5] |= 1u << (j & 31);
                    b = 0;
                }
                s.h_bases[j >> 4] |= b << (2 * (j & 15));
            }
        }
    }
    s.n_reads = r;
    return j;
}

static int launch_slot(aln_server *S, Slot &s) {
    const uint64_t nb = pack_slot(s, S->cfg);
    const uint32_t n = s.n_reads;
    cudaStream_t st = s.st;
    const size_t bw = std::max<size_t>(1, words16(nb)), nw = std::max<size_t>(1, words32(nb));
    if (cudaMemcpyAsync(s.d_bases, s.h_bases, bw * 4, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(s.d_nmask, s.h_nmask, nw * 4, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(s.d_off, s.h_off, n * 8ull, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(s.d_len, s.h_len, n * 2ull, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(s.d_z, s.h_z, n, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return fail(ALN_EDEVICE, "aln_server: copy-in failed");
    aln_batch b{s.d_bases, s.d_nmask, s.d_off, s.d_len, s.d_z};
    aln_params p = S->cfg.params;
    p.mode = ALN_MODE_PERSISTENT;
    // the heavy phase holds every SM until its passes end, which stalls the
    // batches of the other slots; here those batches fill the GPU while a heavy
    // read finishes on its warp, so the phase runs only when asked for
    if (p.heavy_after == 0) p.heavy_after = 0xFFFFFFFFu;
    aln_result out{s.d_res, s.d_hits};
    int rc = aln_search(S->idx, &b, n, &p, &out, st);
    if (rc != ALN_OK) return rc;
    if (cudaMemcpyAsync(s.h_res, s.d_res, n * sizeof(aln_read_result), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(s.h_hits, s.d_hits, static_cast<size_t>(n) * p.hit_cap * sizeof(aln_hit),
                        cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaEventRecord(s.ev, st) != cudaSuccess)
        return fail(ALN_EDEVICE, "aln_server: copy-out failed");
    return ALN_OK;
}

// Fill a free slot from the pending FIFO (caller holds the lock).
static void take_chunks(aln_server *S, Slot &s) {
    s.chunks.clear();
    uint32_t reads = 0;
    uint64_t bases = 0;
    const aln_server_config &c = S->cfg;
    while (!S->pending.empty() && reads < c.max_batch_reads) {
        std::shared_ptr<Request> q = S->pending.front();
        Chunk ch;
        ch.req = q;
        ch.first = q->next;
        uint32_t t = q->next;
        while (t < q->n && reads < c.max_batch_reads && bases + q->len[t] <= c.max_batch_bases) {
            bases += q->len[t];
            reads++;
            t++;
        }
        ch.count = t - q->next;
        if (ch.count == 0) break;  // the next read does not fit: batch full
        q->next = t;
        s.chunks.push_back(ch);
        if (q->next == q->n) S->pending.pop_front();
        else break;  // request continues in the next batch
    }
}

static void scatter(aln_server *S, Slot &s) {
    const uint32_t H = S->cfg.params.hit_cap;
    const auto now = Clock::now();
    for (Chunk &ch : s.chunks) {
        Request &q = *ch.req;
        std::memcpy(q.res.data() + ch.first, s.h_res + ch.slot_first, ch.count * sizeof(aln_read_result));
        std::memcpy(q.hits.data() + static_cast<size_t>(ch.first) * H, s.h_hits + static_cast<size_t>(ch.slot_first) * H,
                    static_cast<size_t>(ch.count) * H * sizeof(aln_hit));
        q.done_reads += ch.count;
        S->reads_done += ch.count;
        if (q.done_reads == q.n) {
            q.done = true;
            q.t_done = now;
            S->latencies_ms.push_back(std::chrono::duration<double, std::milli>(q.t_done - q.t_submit).count());
        }
    }
    s.chunks.clear();
    s.busy = false;
    S->batches++;
}

static void worker_loop(aln_server *S) {
    int dev = 0;
    cudaSetDevice(S->cfg.device);
    cudaGetDevice(&dev);
    std::unique_lock<std::mutex> lk(S->mu);
    while (!S->stop) {
        bool progress = false;
        for (Slot &s : S->slots) {  // completions
            if (s.busy && cudaEventQuery(s.ev) == cudaSuccess) {
                scatter(S, s);
                progress = true;
            }
        }
        if (progress) S->cv_done.notify_all();
        int in_flight = 0;
        for (Slot &s : S->slots) in_flight += s.busy;
        for (Slot &s : S->slots) {  // admissions
            if (s.busy || S->pending.empty() || S->error != ALN_OK) continue;
            // coalesce: with work already on the device, give a young request a moment to be joined
            if (in_flight > 0 && S->cfg.coalesce_us) {
                const auto age = Clock::now() - S->pending.front()->t_submit;
                uint64_t queued = 0;
                for (auto &q : S->pending) queued += q->n - q->next;
                if (queued < S->cfg.max_batch_reads && age < std::chrono::microseconds(S->cfg.coalesce_us)) break;
            }
            take_chunks(S, s);
            if (s.chunks.empty()) continue;
            s.busy = true;
            in_flight++;
            lk.unlock();
            int rc = launch_slot(S, s);
            lk.lock();
            if (rc != ALN_OK) {
                S->error = rc;
                S->error_msg = aln_last_error();
                s.busy = false;
                S->cv_done.notify_all();
            }
            progress = true;
        }
        if (!progress) S->cv_work.wait_for(lk, std::chrono::microseconds(100));
    }
}

extern "C" int aln_server_create(const fm_dindex *idx, const aln_server_config *cfg, aln_server **out) {
    if (!idx || !cfg || !out) return fail(ALN_EINVAL, "aln_server_create: null argument");
    *out = nullptr;
    aln_server_config c = *cfg;
    if (c.max_batch_reads == 0 || c.max_batch_bases < c.max_batch_reads || c.n_slots == 0 || c.n_slots > 16 ||
        c.params.hit_cap < 1 || c.params.z > ALN_MAX_Z)
        return fail(ALN_EINVAL, "aln_server_create: bad configuration");
    fm_index_info_t info;
    if (fm_dindex_info(idx, &info) != ALN_OK) return fail(ALN_EINVAL, "aln_server_create: bad index");
    if (cudaSetDevice(c.device) != cudaSuccess) return fail(ALN_EDEVICE, "aln_server_create: cudaSetDevice");
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return fail(ALN_EDEVICE, "aln_server_create: cudaMemGetInfo");
    const uint64_t budget = c.device_mem_budget ? std::min<uint64_t>(c.device_mem_budget, free_b) : free_b / 2;
    const uint64_t per = slot_bytes(c);
    const uint32_t fit = static_cast<uint32_t>(budget / per);
    if (fit == 0) return fail(ALN_ENOMEM, "aln_server_create: not even one batch slot fits the memory budget");
    c.n_slots = std::min(c.n_slots, fit);
    aln_server *S = new aln_server();
    S->idx = idx;
    S->cfg = c;
    S->slots.resize(c.n_slots);
    for (Slot &s : S->slots) {
        if (!alloc_slot(s, c)) {
            for (Slot &t : S->slots) free_slot(t);
            delete S;
            return fail(ALN_ENOMEM, "aln_server_create: slot allocation failed");
        }
    }
    S->t_start = Clock::now();
    S->worker = std::thread(worker_loop, S);
    *out = S;
    return ALN_OK;
}

extern "C" int aln_server_submit(aln_server *S, const uint8_t *codes, const uint64_t *code_offset,
                                 const uint16_t *len, const uint8_t *z, uint32_t n_reads, uint64_t *request_id) {
    if (!S || !request_id || (n_reads && (!codes || !code_offset || !len)))
        return fail(ALN_EINVAL, "aln_server_submit: null argument");
    auto q = std::make_shared<Request>();
    q->n = n_reads;
    q->len.assign(len, len + n_reads);
    q->off.resize(n_reads);
    uint64_t total = 0;
    for (uint32_t r = 0; r < n_reads; r++) {
        if (len[r] > S->cfg.max_batch_bases) return fail(ALN_EINVAL, "aln_server_submit: read longer than a batch");
        total += len[r];
    }
    q->codes.resize(total);
    uint64_t j = 0;
    for (uint32_t r = 0; r < n_reads; r++) {
        q->off[r] = j;
        std::memcpy(q->codes.data() + j, codes + code_offset[r], len[r]);
        j += len[r];
    }
    if (z) q->z.assign(z, z + n_reads);
    q->res.resize(n_reads);
    q->hits.resize(static_cast<size_t>(n_reads) * S->cfg.params.hit_cap);
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->error != ALN_OK) return fail(S->error, "aln_server_submit: server failed: " + S->error_msg);
    q->id = S->next_id++;
    q->t_submit = Clock::now();
    if (n_reads == 0) {
        q->done = true;
        q->t_done = q->t_submit;
        S->latencies_ms.push_back(0.0);
    } else {
        S->pending.push_back(q);
    }
    S->live[q->id] = q;
    *request_id = q->id;
    S->cv_work.notify_one();
    return ALN_OK;
}

extern "C" int aln_server_poll(aln_server *S, uint64_t request_id, int wait_ms, aln_read_result *res_out,
                               aln_hit *hits_out, double *latency_ms) {
    if (!S) return fail(ALN_EINVAL, "aln_server_poll: null server");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->live.find(request_id);
    if (it == S->live.end()) return fail(ALN_EINVAL, "aln_server_poll: unknown request id");
    std::shared_ptr<Request> q = it->second;
    const auto deadline = Clock::now() + std::chrono::milliseconds(wait_ms < 0 ? 0 : wait_ms);
    while (!q->done && S->error == ALN_OK) {
        if (S->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) break;
    }
    if (!q->done) {
        if (S->error != ALN_OK) return fail(S->error, "aln_server_poll: server failed: " + S->error_msg);
        return ALN_EAGAIN;
    }
    if (res_out) std::memcpy(res_out, q->res.data(), q->n * sizeof(aln_read_result));
    if (hits_out) std::memcpy(hits_out, q->hits.data(), q->hits.size() * sizeof(aln_hit));
    if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(q->t_done - q->t_submit).count();
    S->live.erase(it);
    return ALN_OK;
}

static double pct(std::vector<double> v, double p) {
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    const double pos = p / 100.0 * (v.size() - 1);
    const size_t i = static_cast<size_t>(pos);
    const double f = pos - i;
    return i + 1 < v.size() ? v[i] * (1 - f) + v[i + 1] * f : v[i];
}

extern "C" int aln_server_stats(aln_server *S, aln_server_stats_t *out) {
    if (!S || !out) return fail(ALN_EINVAL, "aln_server_stats: null argument");
    std::lock_guard<std::mutex> lk(S->mu);
    std::memset(out, 0, sizeof *out);
    out->requests_done = S->latencies_ms.size();
    out->reads_done = S->reads_done;
    out->batches = S->batches;
    out->p50_ms = pct(S->latencies_ms, 50);
    out->p95_ms = pct(S->latencies_ms, 95);
    out->p99_ms = pct(S->latencies_ms, 99);
    out->seconds = std::chrono::duration<double>(Clock::now() - S->t_start).count();
    out->n_slots = static_cast<uint32_t>(S->slots.size());
    uint64_t q = 0;
    for (auto &r : S->pending) q += r->n - r->next;
    out->queued_reads = q;
    return ALN_OK;
}

extern "C" void aln_server_destroy(aln_server *S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->worker.joinable()) S->worker.join();
    cudaSetDevice(S->cfg.device);
    for (Slot &s : S->slots) {
        if (s.busy) cudaEventSynchronize(s.ev);
        free_slot(s);
    }
    delete S;
}
