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

template <int STACK_CAP, int SMEM, bool SCORE>
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
    FlatLane<STACK_CAP, SMEM, SCORE> L;
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
        if (!__any_sync(0xFFFFFFFFu, L.phase != PH_FREE)) break;
    }
    if (at_limit) L.stop_at_limit(lane, n_reads, p, res, queue, order);
#ifdef ALN_STATS
    STAT_ADD(0, st_it); STAT_ADD(1, st_f); STAT_ADD(2, st_occ); STAT_ADD(3, st_tab);
    STAT_ADD(4, st_wi); STAT_ADD(5, st_wl); STAT_ADD(6, L.st_reads); STAT_ADD(7, L.st_rounds);
    STAT_ADD(8, L.st_pops); STAT_ADD(9, st_wa); STAT_ADD(10, st_wal);
    STAT_ADD(11, st_cc); STAT_ADD(12, st_cf); STAT_ADD(13, st_ce);
#endif
}

// ---------------------------------------------------------------- heavy phase
//
// Reads whose owner lane passed heavy_after expansions were handed over by the
// persistent search (kFlagDemoted) and are searched here by every lane of the
// GPU, one deepening pass per launch: a pass's subtrees are tasks in a ring in
// global memory; a lane takes a task, searches it depth first (sharing it with
// the idle lanes of its warp exactly as the persistent search does), gives its
// bottom stack entries back to the ring while the ring runs low, and merges the
// candidates it found into the read's hash table (least witness per interval by
// atomicMin).  After each pass one block per read applies the iterative
// deepening rule to the table and either writes the result or starts the next
// pass.  The hit set, witnesses and counts are those of the other forms.

__device__ __forceinline__ unsigned long long global_ns() {  // the GPU's nanosecond timer
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t vload(const uint32_t *p) { return *reinterpret_cast<const volatile uint32_t *>(p); }

// Task t is published once its slot is written: ready[t % cap] = t + 1.
__device__ __forceinline__ void heavy_push(const HeavyCtx &H, const uint4 &node, uint32_t hid, uint32_t s) {
    atomicAdd(&H.hdr->outstanding, 1u);
    const uint32_t t = atomicAdd(&H.hdr->tail, 1u);
    HeavyTask task;
    task.node = node;
    task.hid = hid;
    task.s = s;
    task.pad0 = task.pad1 = 0;
    H.pool[t % kHeavyPool] = task;
    __threadfence();
    atomicExch(&H.ready[t % kHeavyPool], t + 1u);
}

__device__ __forceinline__ unsigned long long mix_id(unsigned long long x) {
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdULL;
    x ^= x >> 33;
    return x;
}

// Insert candidate (lo, hi) of strand s with witness key; returns false if the
// read's table for that strand is full.
__device__ bool heavy_insert(const HeavyCtx &H, uint32_t hid, uint32_t s, uint32_t lo, uint32_t hi, uint32_t key,
                             uint32_t score) {
    HeavySlot *T = H.slots + (static_cast<uint64_t>(hid) * 2 + s) * kHeavySlots;
    const unsigned long long id = (static_cast<unsigned long long>(lo) << 32) | hi;
    uint32_t j = static_cast<uint32_t>(mix_id(id)) & (kHeavySlots - 1);
    const unsigned long long wkey = (static_cast<unsigned long long>(score) << 32) | key;
    // Many lanes insert the same few intervals of a repeat-rich read: a plain
    // read first skips the atomics that would change nothing.  Safe with a stale
    // value: a slot's id only goes from 0 to its final value, and its key only
    // decreases, so a stale read can only cause an atomic, never skip one that
    // was needed.
    for (uint32_t probe = 0; probe < kHeavySlots; probe++, j = (j + 1) & (kHeavySlots - 1)) {
        unsigned long long cur = __ldcg(&T[j].id);
        if (cur == 0ull) {
            cur = atomicCAS(&T[j].id, 0ull, id);
            if (cur == 0ull) {
                atomicMin(&T[j].wkey, wkey);
                atomicAdd(&H.reads[hid].distinct[s], 1u);
                return true;
            }
        }
        if (cur == id) {
            if (__ldcg(&T[j].wkey) > wkey) atomicMin(&T[j].wkey, wkey);
            return true;
        }
    }
    return false;
}

// One block per handed-over read: cleared tables and the root of each strand
// the lower bound admits as a task, for the deepening pass the read was in when
// it was handed over (R->B, written by its lane).  Each pass starts from the
// root with no candidates, so the passes before it need not be searched again.
__global__ void aln_heavy_start_kernel(SearchParams p, const uint2 *dbp, uint32_t n_text) {
    const HeavyCtx H = p.heavy;
    const uint32_t hid = blockIdx.x;
    if (hid >= min(H.hdr->n_heavy, kHeavyReads)) return;
    HeavySlot *T = H.slots + static_cast<uint64_t>(hid) * 2 * kHeavySlots;
    for (uint32_t j = threadIdx.x; j < 2 * kHeavySlots; j += blockDim.x) {
        T[j].id = 0ull;
        T[j].wkey = ~0ull;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        HeavyRead *R = H.reads + hid;
        const uint2 a = dbp[2ull * R->r], b = dbp[2ull * R->r + 1];
        const uint32_t d0 = d_at(a.x, a.y, 0), d1 = d_at(b.x, b.y, 0);
        R->state = 0;
        R->flags = 0;
        R->distinct[0] = R->distinct[1] = 0;
        const uint4 root = make_uint4(0, n_text + 1, pack_info(0, 0, 0, 0, 0, 0, OP_M), 0);
        if (d0 <= R->B) heavy_push(H, root, hid, 0);
        if (d1 <= R->B) heavy_push(H, root, hid, 1);
    }
}

template <int STACK_CAP, bool SCORE>
__global__ void __launch_bounds__(kThreads, ALN_PERSISTENT_MIN_BLOCKS) aln_heavy_pass_kernel(DIndex X, ReadBatch rb,
                                                                                           SearchParams p,
                                                                                           const uint2 *dbp) {
    constexpr int SMEM = kSmemStackDefault;
    __shared__ uint32_t s_bases[kReadWords * kThreads];
    __shared__ uint32_t s_nmask[kMaskWords * kThreads];
    __shared__ uint4 s_stack[SMEM * kThreads];
    const HeavyCtx H = p.heavy;
    uint32_t *sb = s_bases + threadIdx.x, *sn = s_nmask + threadIdx.x;
    const uint32_t lane = threadIdx.x & 31u, warp_col = threadIdx.x & ~31u;
    const unsigned FULL = 0xFFFFFFFFu;
    uint4 stk[STACK_CAP - SMEM], cand[kCandCap];
    FlatLane<STACK_CAP, SMEM, SCORE> L;
    L.sstk = s_stack + threadIdx.x;
    L.stk = stk;
    L.cand = cand;
    L.has_next = false;
    L.phase = PH_IDLE;
    L.r = 0;
    L.sp = 0;
    L.base = 0;
    L.K = X.kmer_k;
    L.role = ROLE_OWN;
    L.owner = lane;
    L.outstanding = 0;
    L.heavy_seen = false;
    L.nc = 0;
    L.flags = 0;
    L.own_rv = ReadView{sb, sn};
    L.rv = L.own_rv;
    uint32_t hid = 0;
    const uint32_t n_heavy = min(vload(&H.hdr->n_heavy), kHeavyReads);
    if (n_heavy == 0) return;
    // Ring entries kept available: one per warp of the grid, so that owners
    // split their subtrees only while lanes wait for work (a mark of two per
    // lane cut them into tasks of about 128 expansions and ran longer).  The
    // ring then holds at most low_water + 32 per warp, within its capacity
    // (the launch bounds the grid).
    const uint32_t low_water = gridDim.x * (kThreads / 32u);
    // consecutive trips with no lane of the warp at work, and since when (warp-uniform)
    uint32_t idle_trips = 0;
    unsigned long long idle_since = 0;
    bool idle_expired = false;
    uint32_t trips = 0, busy = 0;  // this lane's trips, and those it spent on a task
    for (unsigned long long it = 0;; it++) {
        if (it >= p.loop_limit || idle_expired) {  // guard: unfinished tasks mark their reads, the warp stops
            if (lane == 0 && p.status) atomicOr(p.status, ALN_STATUS_LOOP_LIMIT);
            if (L.role == ROLE_OWN && L.phase != PH_IDLE && L.phase != PH_FREE)
                atomicOr(&H.reads[hid].flags, ALN_FLAG_LOOP_LIMIT);
            break;
        }
        FetchReq fr;
        fr.kind = F_NONE;
        trips++;
        busy += (L.phase != PH_IDLE && L.phase != PH_FREE) ? 1u : 0u;
        // control: advance the lane's task until it needs four extensions
        for (int round = 0; round < 32; round++) {
            if (L.phase == PH_FREE || L.phase == PH_RETURN || L.phase == PH_IDLE) break;
            if (L.phase == PH_WAIT) {
                if (L.outstanding) break;
                L.phase = PH_DFS;
            }
            if (!L.has_next && L.sp == L.base) {
                L.sp = L.base = 0;
                if (L.role == ROLE_HELP) {
                    L.phase = PH_RETURN;
                    L.ret_i = 0;
                    break;
                }
                if (L.outstanding) {
                    L.phase = PH_WAIT;
                    break;
                }
                // task done: its candidates into the read's table, then the next task
                uint32_t f = L.flags & ALN_FLAG_INCOMPLETE;
                for (uint32_t j = 0; j < L.nc; j++) {
                    const uint4 c = L.cand[j];
                    if (!heavy_insert(H, hid, c.z >> 31, c.x, c.y, c.z, c.w)) f |= ALN_FLAG_CAND_OVERFLOW;
                }
                if (f) atomicOr(&H.reads[hid].flags, f);
                atomicAdd(&H.hdr->expansions, static_cast<unsigned long long>(L.work));
                atomicSub(&H.hdr->outstanding, 1u);
                L.phase = PH_IDLE;
                break;
            }
            if (++L.work > p.work_limit) {
                L.flags |= ALN_FLAG_WORK_LIMIT;
                L.sp = L.base;
                L.has_next = false;
                continue;
            }
            if (L.expand_top(p, fr)) break;
        }
        __syncwarp();
        if (fr.kind != F_NONE) {
            uint32_t lo4[4], hi4[4];
            fetch4(X, fr, lo4, hi4);
            L.apply(X, lo4, hi4);
        }
        // the ring runs low: lanes give their bottom stack entries back to it (its
        // level read by one lane, the tickets taken once per warp); helpers too,
        // or the subtrees a warp's idle lanes take from its owners could never
        // reach other warps (L.r holds the read's list entry either way)
        const bool can_push = L.phase == PH_DFS && (L.sp - L.base >= 2 || (L.sp - L.base >= 1 && L.has_next));
        const unsigned pushers = __ballot_sync(FULL, can_push);
        if (pushers) {
            const uint32_t src = __ffs(pushers) - 1;
            uint32_t t0 = 0xFFFFFFFFu;
            if (lane == src && vload(&H.hdr->tail) - vload(&H.hdr->head) < low_water) {
                atomicAdd(&H.hdr->outstanding, static_cast<uint32_t>(__popc(pushers)));  // before publishing
                t0 = atomicAdd(&H.hdr->tail, static_cast<uint32_t>(__popc(pushers)));
            }
            t0 = __shfl_sync(FULL, t0, src);
            if (t0 != 0xFFFFFFFFu && can_push) {
                const uint32_t t = t0 + __popc(pushers & ((1u << lane) - 1u));
                const uint4 e = L.stk_get(L.base);
                L.base++;
                HeavyTask task;
                task.node = e;
                task.hid = L.r;
                task.s = L.s;
                task.pad0 = task.pad1 = 0;
                H.pool[t % kHeavyPool] = task;
                __threadfence();
                atomicExch(&H.ready[t % kHeavyPool], t + 1u);
            }
        }
        // a helper merges its candidates into the read's table itself: the
        // hand-back through the owner moves one per trip, and a subtree of a
        // repeat-rich read can hold hundreds
        if (L.phase == PH_RETURN && L.ret_i < L.nc) {
            uint32_t f = 0;
            for (uint32_t j = L.ret_i; j < L.nc; j++) {
                const uint4 c = L.cand[j];
                if (!heavy_insert(H, L.r, c.z >> 31, c.x, c.y, c.z, c.w)) f |= ALN_FLAG_CAND_OVERFLOW;
            }
            if (f) atomicOr(&H.reads[L.r].flags, f);
            L.ret_i = L.nc;
        }
        L.exchange(lane, s_bases, s_nmask, warp_col, 0u);
        // idle lanes take tasks from the ring, one claim per warp
        const unsigned idle = __ballot_sync(FULL, L.phase == PH_IDLE);
        if (idle) {
            const uint32_t leader = __ffs(idle) - 1;
            uint32_t first = 0, got = 0;
            if (lane == leader) {
                const uint32_t want = __popc(idle);
                uint32_t h = vload(&H.hdr->head);
                for (int tries = 0; tries < 64; tries++) {
                    const uint32_t t = vload(&H.hdr->tail);
                    const int avail = static_cast<int>(t - h);
                    if (avail <= 0) break;
                    const uint32_t g = min(want, static_cast<uint32_t>(avail));
                    const uint32_t old = atomicCAS(&H.hdr->head, h, h + g);
                    if (old == h) {
                        first = h;
                        got = g;
                        break;
                    }
                    h = old;
                }
            }
            first = __shfl_sync(FULL, first, leader);
            got = __shfl_sync(FULL, got, leader);
            const uint32_t rank = __popc(idle & ((1u << lane) - 1u));
            if (L.phase == PH_IDLE) {
                if (rank < got) {
                    const uint32_t t = first + rank;
                    uint32_t spins = 0;
                    while (vload(&H.ready[t % kHeavyPool]) != t + 1u && spins < (1u << 22)) spins++;
                    if (spins >= (1u << 22)) {  // a published task that never appeared: give up
                        if (p.status) atomicOr(p.status, ALN_STATUS_LOOP_LIMIT);
                        L.phase = PH_FREE;
                    } else {
                        __threadfence();  // the task's slot was written before its ready word
                        const HeavyTask *slot = H.pool + (t % kHeavyPool);
                        HeavyTask task;
                        task.node = __ldcg(&slot->node);
                        task.hid = __ldcg(&slot->hid);
                        task.s = __ldcg(&slot->s);
                        hid = task.hid;
                        const HeavyRead R = H.reads[hid];
                        L.r = hid;  // the list entry (a helper gets it with the subtree)
                        L.m = R.m;
                        L.z = R.z;
                        L.B = R.B;
                        L.s = task.s;
                        load_read(rb, rb.offset[R.r], R.m, sb, sn);
                        const uint2 bp = dbp[2ull * R.r + task.s];
                        if (task.s) {
                            L.bpb0 = bp.x;
                            L.bpb1 = bp.y;
                        } else {
                            L.bpa0 = bp.x;
                            L.bpa1 = bp.y;
                        }
                        L.rv = L.own_rv;
                        L.role = ROLE_OWN;
                        L.next = task.node;
                        L.has_next = true;
                        L.sp = L.base = 0;
                        L.nc = 0;
                        L.work = 0;
                        L.flags = 0;
                        L.outstanding = 0;
                        L.phase = PH_DFS;
                    }
                } else if (got == 0 && vload(&H.hdr->outstanding) == 0) {
                    L.phase = PH_FREE;  // the pass is over
                }
            }
            if (__ballot_sync(FULL, L.phase != PH_IDLE && L.phase != PH_FREE) == 0) {
                // back off (0.25 to 16 us) so that idle warps leave the ring's
                // counters to the lanes that publish and take tasks; 4 s without
                // work ends the warp (a task that never came)
                const unsigned long long now = global_ns();
                if (idle_trips == 0) idle_since = now;
                idle_expired = __shfl_sync(FULL, now - idle_since > 4000000000ull ? 1u : 0u, 0) != 0;
                __nanosleep(256u << min(idle_trips, 6u));
                idle_trips++;
            } else {
                idle_trips = 0;
            }
        } else {
            idle_trips = 0;
        }
        if (__ballot_sync(FULL, L.phase != PH_FREE) == 0) break;
    }
    const uint32_t wt = __reduce_add_sync(FULL, trips), wb = __reduce_add_sync(FULL, busy);
    if (lane == 0) {
        atomicAdd(&H.hdr->lane_trips, static_cast<unsigned long long>(wt));
        atomicAdd(&H.hdr->busy_trips, static_cast<unsigned long long>(wb));
    }
}

// Score-ordered result of a handed-over read from its tables (the rule of the
// persistent search's score writer: strata S1 / S2, order (score, strand, k, l)).
__device__ void heavy_write_score(const SearchParams &p, const HeavySlot *T, const HeavyRead *R, uint32_t n_used,
                                  aln_read_result *res, aln_hit *hits) {
    aln_read_result out;
    out.c0 = out.c1 = 0;
    out.n_hits = 0;
    out.d_best = 255;
    out.best_score = 255;
    uint32_t flags = R->flags & 0xFFu;
    uint32_t s1 = 0xFFFFFFFFu, s2 = 0xFFFFFFFFu;
    for (uint32_t j = 0; j < 2 * kHeavySlots; j++)
        if (T[j].id) s1 = min(s1, static_cast<uint32_t>(T[j].wkey >> 32));
    for (uint32_t j = 0; j < 2 * kHeavySlots; j++)
        if (T[j].id && static_cast<uint32_t>(T[j].wkey >> 32) > s1) s2 = min(s2, static_cast<uint32_t>(T[j].wkey >> 32));
    if (n_used) {
        unsigned long long c0 = 0, c1 = 0;
        uint32_t dbest = 255;
        for (uint32_t j = 0; j < 2 * kHeavySlots; j++) {
            if (!T[j].id) continue;
            const uint32_t sc = static_cast<uint32_t>(T[j].wkey >> 32);
            const unsigned long long w = (T[j].id & 0xFFFFFFFFull) - (T[j].id >> 32);
            if (sc == s1) {
                c0 += w;
                dbest = min(dbest, (static_cast<uint32_t>(T[j].wkey) >> 28) & 7u);
            } else if (sc == s2) {
                c1 += w;
            }
        }
        const bool many = p.max_best && c0 > p.max_best;
        uint32_t kept = 0;
        for (uint32_t j = 0; j < 2 * kHeavySlots; j++) {
            if (!T[j].id) continue;
            const uint32_t sc = static_cast<uint32_t>(T[j].wkey >> 32);
            if (sc == s1 || (!many && sc == s2)) kept++;
        }
        if (many) flags |= ALN_FLAG_MANY_BEST;
        const uint32_t nout = min(kept, p.hit_cap);
        if (kept > p.hit_cap) flags |= ALN_FLAG_HIT_OVERFLOW;
        aln_hit *Hh = hits + static_cast<uint64_t>(R->r) * p.hit_cap;
        // order (score, strand, k, l): each round takes the least entry above the previous one
        unsigned long long prev_s = 0, prev_o = 0;
        bool have_prev = false;
        for (uint32_t t = 0; t < nout; t++) {
            bool found = false;
            unsigned long long bs = 0, bo = 0;
            uint32_t bkey = 0;
            for (uint32_t j = 0; j < 2 * kHeavySlots; j++) {
                if (!T[j].id) continue;
                const uint32_t sc = static_cast<uint32_t>(T[j].wkey >> 32);
                if (!(sc == s1 || (!many && sc == s2))) continue;
                const uint32_t key = static_cast<uint32_t>(T[j].wkey);
                // (strand, k, l) as one number: strand above the 64-bit interval order
                const unsigned long long o = T[j].id;
                const unsigned long long ss = (static_cast<unsigned long long>(sc) << 1) | (key >> 31);
                if (have_prev && (ss < prev_s || (ss == prev_s && o <= prev_o))) continue;
                if (!found || ss < bs || (ss == bs && o < bo)) {
                    found = true;
                    bs = ss;
                    bo = o;
                    bkey = key;
                }
            }
            aln_hit h;
            h.k = static_cast<uint32_t>(bo >> 32);
            h.l = static_cast<uint32_t>(bo) - 1;
            h.aligned_len = static_cast<uint16_t>(bkey & 0xFFFFu);
            h.strand = static_cast<uint8_t>(bkey >> 31);
            h.n_diff = static_cast<uint8_t>((bkey >> 28) & 7u);
            h.n_gapo = static_cast<uint8_t>((bkey >> 24) & 15u);
            h.n_gape = static_cast<uint8_t>((bkey >> 20) & 15u);
            h.n_mm = static_cast<uint8_t>((bkey >> 16) & 15u);
            h.reserved = 0;
            Hh[t] = h;
            prev_s = bs;
            prev_o = bo;
            have_prev = true;
        }
        out.c0 = c0 > 0xFFFFFFFFull ? 0xFFFFFFFFu : static_cast<uint32_t>(c0);
        out.c1 = c1 > 0xFFFFFFFFull ? 0xFFFFFFFFu : static_cast<uint32_t>(c1);
        out.d_best = static_cast<uint8_t>(dbest);
        out.best_score = static_cast<uint8_t>(s1 > 254 ? 254 : s1);
        out.n_hits = static_cast<uint8_t>(nout);
    }
    out.flags = static_cast<uint8_t>(flags);
    res[R->r] = out;
}

// One block per handed-over read after a pass: the iterative deepening rule on
// its table; the result, or the next pass's budget, cleared tables and roots.
__global__ void aln_heavy_decide_kernel(SearchParams p, const uint2 *dbp, uint32_t n_text, aln_read_result *res,
                                        aln_hit *hits, int last) {
    const HeavyCtx H = p.heavy;
    const uint32_t hid = blockIdx.x;
    if (hid >= min(H.hdr->n_heavy, kHeavyReads)) return;
    HeavyRead *R = H.reads + hid;
    if (R->state != 0) return;
    HeavySlot *T = H.slots + static_cast<uint64_t>(hid) * 2 * kHeavySlots;
    __shared__ uint32_t s_dmin, s_n;
    __shared__ uint32_t s_next;  // 0 finish, else the next pass budget
    __shared__ uint32_t s_final;
    if (threadIdx.x == 0) {
        s_dmin = 255;
        s_n = 0;
    }
    __syncthreads();
    for (uint32_t j = threadIdx.x; j < 2 * kHeavySlots; j += blockDim.x)
        if (T[j].id) {
            atomicMin(&s_dmin, (static_cast<uint32_t>(T[j].wkey) >> 28) & 7u);
            atomicAdd(&s_n, 1u);
        }
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t z = R->z, B = R->B;
        uint32_t next = 0, fin = 0;
        if (s_n > static_cast<uint32_t>(kCandCap)) R->flags |= ALN_FLAG_CAND_OVERFLOW;
        if ((R->flags & ALN_FLAG_INCOMPLETE) || p.strata != ALN_STRATA_BEST1) {
            fin = z;
        } else if (s_n == 0) {
            if (B < z) next = min(z, B + 2);
            fin = 0;
        } else {
            const uint32_t F = min(z, s_dmin + 1);
            if (F <= B) fin = F;
            else next = F;
        }
        if (next && last) {  // cannot happen within kHeavyPasses passes; leave no read without a result
            R->flags |= ALN_FLAG_LOOP_LIMIT;
            next = 0;
            fin = B;
        }
        s_next = next;
        s_final = fin;
    }
    __syncthreads();
    if (s_next) {  // next pass: clear the tables, then the roots
        for (uint32_t j = threadIdx.x; j < 2 * kHeavySlots; j += blockDim.x) {
            T[j].id = 0ull;
            T[j].wkey = ~0ull;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            R->B = s_next;
            R->distinct[0] = R->distinct[1] = 0;
            const uint2 a = dbp[2ull * R->r], b = dbp[2ull * R->r + 1];
            const uint4 root = make_uint4(0, n_text + 1, pack_info(0, 0, 0, 0, 0, 0, OP_M), 0);
            if (d_at(a.x, a.y, 0) <= s_next) heavy_push(H, root, hid, 0);
            if (d_at(b.x, b.y, 0) <= s_next) heavy_push(H, root, hid, 1);
        }
        return;
    }
    if (threadIdx.x != 0) return;
    if (p.strata == ALN_STRATA_SCORE) {
        heavy_write_score(p, T, R, s_n, res, hits);
        R->state = 1;
        return;
    }
    // the result: hits with diffs <= the final budget, ordered (diffs, strand, k, l)
    const uint32_t fin = s_final;
    aln_read_result out;
    out.c0 = out.c1 = 0;
    out.n_hits = 0;
    out.d_best = 255;
    out.best_score = 0;
    uint32_t dbest = 255;
    for (uint32_t j = 0; j < 2 * kHeavySlots; j++)
        if (T[j].id && ((static_cast<uint32_t>(T[j].wkey) >> 28) & 7u) <= fin) dbest = min(dbest, (static_cast<uint32_t>(T[j].wkey) >> 28) & 7u);
    uint32_t flags = R->flags & 0xFFu;
    if (dbest != 255 && s_n) {
        unsigned long long c0 = 0, c1 = 0;
        uint32_t kept = 0;
        for (uint32_t j = 0; j < 2 * kHeavySlots; j++) {
            if (!T[j].id) continue;
            const uint32_t d = (static_cast<uint32_t>(T[j].wkey) >> 28) & 7u;
            if (d > fin) continue;
            kept++;
            const unsigned long long w = (T[j].id & 0xFFFFFFFFull) - (T[j].id >> 32);
            if (d == dbest) c0 += w;
            else if (d == dbest + 1) c1 += w;
        }
        out.c0 = c0 > 0xFFFFFFFFull ? 0xFFFFFFFFu : static_cast<uint32_t>(c0);
        out.c1 = c1 > 0xFFFFFFFFull ? 0xFFFFFFFFu : static_cast<uint32_t>(c1);
        out.d_best = static_cast<uint8_t>(dbest);
        const uint32_t nout = min(kept, p.hit_cap);
        if (kept > p.hit_cap) flags |= ALN_FLAG_HIT_OVERFLOW;
        aln_hit *Hh = hits + static_cast<uint64_t>(R->r) * p.hit_cap;
        // selection of the nout smallest by (diffs, strand, k, l): each round takes
        // the least entry above the previous one
        uint32_t pk = 0, pl = 0, pkey = 0;
        bool have_prev = false;
        for (uint32_t t = 0; t < nout; t++) {
            bool found = false;
            uint32_t bk = 0, bl = 0, bkey = 0;
            for (uint32_t j = 0; j < 2 * kHeavySlots; j++) {
                if (!T[j].id) continue;
                const uint32_t key = static_cast<uint32_t>(T[j].wkey);
                const uint32_t d = (key >> 28) & 7u;
                if (d > fin) continue;
                const uint32_t k = static_cast<uint32_t>(T[j].id >> 32), l = static_cast<uint32_t>(T[j].id);
                const uint32_t o = (d << 1) | (key >> 31);
                if (have_prev) {
                    const uint32_t po = (((pkey >> 28) & 7u) << 1) | (pkey >> 31);
                    if (o < po || (o == po && (k < pk || (k == pk && l <= pl)))) continue;
                }
                if (!found) {
                    found = true;
                    bk = k; bl = l; bkey = key;
                } else {
                    const uint32_t bo = (((bkey >> 28) & 7u) << 1) | (bkey >> 31);
                    if (o < bo || (o == bo && (k < bk || (k == bk && l < bl)))) {
                        bk = k; bl = l; bkey = key;
                    }
                }
            }
            aln_hit h;
            h.k = bk;
            h.l = bl - 1;
            h.aligned_len = static_cast<uint16_t>(bkey & 0xFFFFu);
            h.strand = static_cast<uint8_t>(bkey >> 31);
            h.n_diff = static_cast<uint8_t>((bkey >> 28) & 7u);
            h.n_gapo = static_cast<uint8_t>((bkey >> 24) & 15u);
            h.n_gape = static_cast<uint8_t>((bkey >> 20) & 15u);
            h.n_mm = static_cast<uint8_t>((bkey >> 16) & 15u);
            h.reserved = 0;
            Hh[t] = h;
            pk = bk; pl = bl; pkey = bkey;
            have_prev = true;
        }
        out.n_hits = static_cast<uint8_t>(nout);
    }
    out.flags = static_cast<uint8_t>(flags);
    res[R->r] = out;
    R->state = 1;
}

// ---------------------------------------------------------------- end of the heavy phase

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
HeavyCtx heavy_layout(void *scratch, uint32_t n);

template <int CAP, int SMEM, bool SCORE>
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
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, aln_persistent_kernel<CAP, SMEM, SCORE>, kThreads, 0);
        if (p.blocks_per_sm && static_cast<int>(p.blocks_per_sm) < per_sm) per_sm = p.blocks_per_sm;
        if (per_sm < 1) per_sm = 1;
        uint32_t blocks = static_cast<uint32_t>(sms * per_sm);
        const uint32_t need = (n + kThreads - 1) / kThreads;
        if (blocks > need) blocks = need ? need : 1;
        cudaMemsetAsync(queue, 0, sizeof(uint32_t), st);
        uint2 *dbp = nullptr;
        uint32_t *order = nullptr;
        SearchParams pp = p;
        pp.heavy.hdr = nullptr;
        if (scratch) {  // D pre-pass and visit order (layout: search_scratch_bytes)
            uint32_t *counts = static_cast<uint32_t *>(scratch), *cursor = counts + kOrderBins;
            dbp = reinterpret_cast<uint2 *>(static_cast<char *>(scratch) + 256);
            order = reinterpret_cast<uint32_t *>(static_cast<char *>(scratch) + 256 + 16ull * n);
            if (p.heavy_after != 0xFFFFFFFFu) {  // the heavy phase's state after them
                pp.heavy = heavy_layout(scratch, n);
                cudaMemsetAsync(pp.heavy.hdr, 0, sizeof(HeavyHdr), st);
                cudaMemsetAsync(pp.heavy.ready, 0, 4ull * kHeavyPool, st);
            }
            cudaMemsetAsync(scratch, 0, 2 * kOrderBins * sizeof(uint32_t), st);
            aln_dscan_kernel<<<static_cast<unsigned>((2ull * n + kThreads - 1) / kThreads), kThreads, 0, st>>>(
                X, rb, n, p, dbp);
            const uint32_t ob = min((n + 255u) / 256u, static_cast<uint32_t>(sms) * 8u);
            aln_order_count_kernel<<<ob, 256, 0, st>>>(dbp, n, counts);
            aln_order_scatter_kernel<<<ob, 256, 0, st>>>(dbp, n, counts, cursor, order);
        }
        const SearchParams &p1 = pp;
        if (p.window_base && p.window_bytes) {  // prefix-trie tables held in L2's persisting set
            cudaLaunchConfig_t cfg{};
            cfg.gridDim = dim3(blocks);
            cfg.blockDim = dim3(kThreads);
            cfg.stream = st;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeAccessPolicyWindow;
            attr[0].val.accessPolicyWindow.base_ptr = p.window_base;
            attr[0].val.accessPolicyWindow.num_bytes = p.window_bytes;
            attr[0].val.accessPolicyWindow.hitRatio = p.window_hit_ratio;
            attr[0].val.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
            attr[0].val.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            const cudaError_t e = cudaLaunchKernelEx(&cfg, aln_persistent_kernel<CAP, SMEM, SCORE>, X, rb, n, p1, res, hits,
                                                     queue, static_cast<const uint32_t *>(order),
                                                     static_cast<const uint2 *>(dbp));
            if (e != cudaSuccess) return e;
        } else {
            aln_persistent_kernel<CAP, SMEM, SCORE><<<blocks, kThreads, 0, st>>>(X, rb, n, p1, res, hits, queue, order,
                                                                                dbp);
        }
        if (pp.heavy.hdr) {  // the reads handed over, one deepening pass per launch over the whole GPU
            int hb = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&hb, aln_heavy_pass_kernel<CAP, SCORE>, kThreads, 0);
            // the ring holds at most 2 entries per thread of the grid (the pass kernel's low-water mark)
            const unsigned hgrid = min(static_cast<unsigned>(sms * (hb > 0 ? hb : 1)), kHeavyPool / (2u * kThreads));
            aln_heavy_start_kernel<<<kHeavyReads, 128, 0, st>>>(pp, dbp, X.t[0].n);
            for (uint32_t pass = 0; pass < kHeavyPasses; pass++) {
                aln_heavy_pass_kernel<CAP, SCORE><<<hgrid, kThreads, 0, st>>>(X, rb, pp, dbp);
                aln_heavy_decide_kernel<<<kHeavyReads, 128, 0, st>>>(pp, dbp, X.t[0].n, res, hits,
                                                                    pass + 1 == kHeavyPasses ? 1 : 0);
            }
        }
    }
    return cudaGetLastError();
}

// Resident blocks per SM of the persistent kernel for limit z and a shared-memory
// stack of smem entries per lane (occupancy).
template <int SMEM>
static int max_blocks_smem(uint32_t z) {
    int per_sm = 0;
    switch (stack_cap_for(z)) {
        case 19: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, aln_persistent_kernel<19, SMEM, false>, kThreads, 0); break;
        case 37: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, aln_persistent_kernel<37, SMEM, false>, kThreads, 0); break;
        default: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, aln_persistent_kernel<64, SMEM, false>, kThreads, 0); break;
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
// (256 B), D breakpoints (2 x 8 B per read), visit order (4 B per read), then
// from the next 256-byte boundary the heavy phase: its header, the handed-over
// reads, their candidate tables, the task ring and its ready words.
static uint64_t heavy_offset(uint32_t n) { return (256ull + 20ull * n + 255ull) & ~255ull; }
static constexpr uint64_t kHeavyBytes = sizeof(HeavyHdr) + kHeavyReads * sizeof(HeavyRead) +
                                        2ull * kHeavyReads * kHeavySlots * sizeof(HeavySlot) +
                                        kHeavyPool * sizeof(HeavyTask) + 4ull * kHeavyPool;
uint64_t search_scratch_bytes(uint32_t n) { return heavy_offset(n) + kHeavyBytes; }

HeavyCtx heavy_layout(void *scratch, uint32_t n) {
    char *b = static_cast<char *>(scratch) + heavy_offset(n);
    HeavyCtx H;
    H.hdr = reinterpret_cast<HeavyHdr *>(b);
    b += sizeof(HeavyHdr);
    H.reads = reinterpret_cast<HeavyRead *>(b);
    b += kHeavyReads * sizeof(HeavyRead);
    H.slots = reinterpret_cast<HeavySlot *>(b);
    b += 2ull * kHeavyReads * kHeavySlots * sizeof(HeavySlot);
    H.pool = reinterpret_cast<HeavyTask *>(b);
    b += kHeavyPool * sizeof(HeavyTask);
    H.ready = reinterpret_cast<uint32_t *>(b);
    return H;
}

template <int CAP>
static cudaError_t launch_smem(const DIndex &X, const ReadBatch &rb, uint32_t n, const SearchParams &p,
                               aln_read_result *res, aln_hit *hits, uint32_t mode, uint32_t *queue, void *scratch,
                               cudaStream_t st) {
    if (p.strata == ALN_STRATA_SCORE)  // score-ordered kernels: the default stack depth only
        return launch_cap<CAP, kSmemStackDefault, true>(X, rb, n, p, res, hits, mode, queue, scratch, st);
    switch (p.smem_stack) {
        case 4: return launch_cap<CAP, 4, false>(X, rb, n, p, res, hits, mode, queue, scratch, st);
        case 12: return launch_cap<CAP, 12, false>(X, rb, n, p, res, hits, mode, queue, scratch, st);
        default: return launch_cap<CAP, kSmemStackDefault, false>(X, rb, n, p, res, hits, mode, queue, scratch, st);
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
