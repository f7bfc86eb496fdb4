// Persistent search as one flat per-lane state machine (sm_103a).
//
// Every iteration of the kernel's single loop has three parts:
//   control  -- cheap, divergent: the lane advances its own read (take the next
//               read from the device queue, load it, step the D scan, pop the
//               stack, emit a hit, finish a strand or a pass, reduce and write
//               the result) until it needs the four extensions of one interval;
//   fetch    -- the four extensions, from one of two sources: a 32-byte group
//               of the prefix-trie table when the node's target is shorter than
//               k (the interval of a string depends on the string alone), else
//               the Occ blocks at the two rows (lf4);
//   apply    -- cheap: the D-scan step or the children pushes that use them.
// A lane that finishes a read takes the next one at once, so the lanes of a
// warp keep doing the same expensive step together, whatever reads they hold.
// Once the read queue is empty, a lane without work takes the bottom entry of
// a busy lane's stack (its shallowest, usually largest, pending subtree) with
// that read's context, searches it as a helper and hands its candidates back to
// the owner, which finishes a pass only when every handed-out subtree has come
// back (warp-level redistribution of backtracking work by ballot and shuffle).
// The search (strands, D, children, limits, iterative deepening, reduction) is
// that of aln_search.cuh; results are identical.
#pragma once

#include "aln_search.cuh"

namespace aln {

enum : uint32_t { PH_IDLE = 0, PH_DSCAN = 1, PH_DFS = 2, PH_DONE = 3, PH_FREE = 4, PH_WAIT = 5, PH_RETURN = 6 };
enum : uint32_t { ROLE_OWN = 0, ROLE_HELP = 1 };
enum : uint32_t { F_NONE = 0, F_OCC = 1, F_TABLE = 2, F_ROOT = 3, F_ZERO = 4 };
// lane-private flag bits above the ABI's (never written to a result)
constexpr uint32_t kFlagHeavyTried = 0x100;  // the read asked for a heavy-phase slot
constexpr uint32_t kFlagDemoted = 0x200;     // the read was handed to the heavy phase
constexpr uint32_t kFlagDrained = 0x400;     // a lane of the warp found the read queue empty
constexpr int kSmemStackDefault = 8;  // bottom stack entries per lane kept in shared memory

// First entry of level j (strings of length j) in the prefix-trie table.
__device__ __forceinline__ uint32_t trie_off(uint32_t j) { return ((1u << (2 * j)) - 4u) / 3u; }

struct FetchReq {
    uint32_t kind;    // F_NONE; F_OCC / F_TABLE: extensions from Occ blocks / the table;
                      // F_ROOT: extensions of the empty string; F_ZERO: none needed
    uint32_t text;    // 0 = X, 1 = X reversed
    uint32_t lo, hi;  // F_OCC: the interval
    uint32_t toff;    // F_TABLE: first of the four children entries
};

// SCORE: the score-ordered mode (candidates keyed by (score, witness)); its
// kernels are separate instantiations, so the other modes carry none of its code.
template <int STACK_CAP, int SMEM, bool SCORE = false>
struct FlatLane {
    uint4 *sstk;              // entries 0..SMEM-1: shared memory, entry j at sstk[j * kThreads]
    uint4 *stk;               // entries SMEM..STACK_CAP-1: local memory
    uint4 *cand;              // kCandCap candidates (lo, hi, key, -), local memory
    uint4 next;               // the node the next pop would return, kept in registers
    bool has_next;
    uint32_t nc, flags, work;
    uint32_t phase, r, m, z, s, K;
    int dj;
    uint32_t dcnt, dlo, dhi, dsl, dsid;  // D scan: interval, segment length and id
    uint32_t bpa0, bpa1, bpb0, bpb1;     // D breakpoints of strand 0 (a) and strand 1 (b)
    uint32_t d00, d01;                   // D(0) of strand 0 and strand 1
    uint32_t B;
    int sp;
    uint4 cur;                           // node being expanded across the fetch
    uint32_t cbits;                      // its decisions
    uint32_t role, owner;                // own read, or helper for the read of lane `owner`
    uint32_t outstanding;                // owner: subtrees handed out and not yet returned
    int base;                            // stack bottom (entries below were handed out)
    uint32_t ret_i;                      // helper: next candidate to hand back
    bool heavy_seen;                     // the last hand-over saw a heavy read with work to give
    ReadView rv;                         // bases of the read being searched
    ReadView own_rv;                     // this lane's shared-memory read columns
#ifdef ALN_STATS
    unsigned long long st_reads = 0, st_rounds = 0, st_pops = 0;
#endif

    // Record a candidate; equal (strand, lo, hi) keep the least (score, key)
    // (the score is 0 outside the score-ordered mode).
    __device__ __forceinline__ void add_cand(uint32_t lo, uint32_t hi, uint32_t key, uint32_t score) {
        for (uint32_t j = 0; j < nc; j++) {
            const uint4 c = cand[j];
            if (c.x == lo && c.y == hi && (c.z >> 31) == (key >> 31)) {
                if constexpr (SCORE) {
                    if (score < c.w || (score == c.w && key < c.z)) cand[j] = make_uint4(lo, hi, key, score);
                } else {
                    if (key < c.z) cand[j].z = key;
                }
                return;
            }
        }
        if (nc < kCandCap) cand[nc++] = make_uint4(lo, hi, key, score);
        else flags |= ALN_FLAG_CAND_OVERFLOW;
    }

    __device__ __forceinline__ void record_fail() {
        const uint32_t v = static_cast<uint32_t>(dj) + 1u;
        const uint32_t sh = 8 * (dcnt & 3u);
        if (s == 0) {
            if (dcnt < 4) bpa0 |= v << sh;
            else bpa1 |= v << sh;
        } else {
            if (dcnt < 4) bpb0 |= v << sh;
            else bpb1 |= v << sh;
        }
        dcnt++;
    }

    // Score-ordered mode: strata by penalty score (S1 and S2), order (score,
    // strand, k, l), the S1 stratum alone above max_best best places.
    __device__ void write_score_result(aln_read_result *res, aln_hit *hits, const SearchParams &p) {
        aln_read_result out;
        out.c0 = out.c1 = 0;
        out.n_hits = 0;
        out.d_best = 255;
        out.best_score = 255;
        aln_hit *H = hits + static_cast<uint64_t>(r) * p.hit_cap;
        uint32_t s1 = 0xFFFFFFFFu, s2 = 0xFFFFFFFFu;
        for (uint32_t j = 0; j < nc; j++) s1 = min(s1, cand[j].w);
        for (uint32_t j = 0; j < nc; j++)
            if (cand[j].w > s1) s2 = min(s2, cand[j].w);
        unsigned long long c0 = 0, c1 = 0;
        uint32_t dbest = 255;
        for (uint32_t j = 0; j < nc; j++) {
            const uint4 c = cand[j];
            if (c.w == s1) {
                c0 += c.y - c.x;
                dbest = min(dbest, (c.z >> 28) & 7u);
            } else if (c.w == s2) {
                c1 += c.y - c.x;
            }
        }
        const bool many = p.max_best && c0 > p.max_best;
        uint32_t kept = 0;
        for (uint32_t j = 0; j < nc; j++) {
            const uint4 c = cand[j];
            if (c.w == s1 || (!many && c.w == s2)) cand[kept++] = c;
        }
        if (many) flags |= ALN_FLAG_MANY_BEST;
        const uint32_t nout = min(kept, p.hit_cap);
        if (kept > p.hit_cap) flags |= ALN_FLAG_HIT_OVERFLOW;
        for (uint32_t t = 0; t < nout; t++) {  // order (score, strand, k, l): selection
            uint32_t best = t;
            uint4 cb = cand[t];
            for (uint32_t j = t + 1; j < kept; j++) {
                const uint4 cj = cand[j];
                if (cj.w < cb.w || (cj.w == cb.w && ((cj.z >> 31) < (cb.z >> 31) ||
                    ((cj.z >> 31) == (cb.z >> 31) && (cj.x < cb.x || (cj.x == cb.x && cj.y < cb.y)))))) {
                    best = j;
                    cb = cj;
                }
            }
            cand[best] = cand[t];
            cand[t] = cb;
            aln_hit h;
            const uint32_t key = cb.z;
            h.k = cb.x;
            h.l = cb.y - 1;
            h.aligned_len = static_cast<uint16_t>(key & 0xFFFFu);
            h.strand = static_cast<uint8_t>(key >> 31);
            h.n_diff = static_cast<uint8_t>((key >> 28) & 7u);
            h.n_gapo = static_cast<uint8_t>((key >> 24) & 15u);
            h.n_gape = static_cast<uint8_t>((key >> 20) & 15u);
            h.n_mm = static_cast<uint8_t>((key >> 16) & 15u);
            h.reserved = 0;
            H[t] = h;
        }
        if (nc) {
            out.c0 = c0 > 0xFFFFFFFFull ? 0xFFFFFFFFu : static_cast<uint32_t>(c0);
            out.c1 = c1 > 0xFFFFFFFFull ? 0xFFFFFFFFu : static_cast<uint32_t>(c1);
            out.d_best = static_cast<uint8_t>(dbest);
            out.best_score = static_cast<uint8_t>(s1 > 254 ? 254 : s1);
            out.n_hits = static_cast<uint8_t>(nout);
        }
        out.flags = static_cast<uint8_t>(flags);
        res[r] = out;
        phase = PH_IDLE;
    }

    __device__ __forceinline__ void write_result(aln_read_result *res, aln_hit *hits, const SearchParams &p,
                                                 bool any, uint32_t final_b) {
        if constexpr (SCORE) {  // the score-ordered mode has its own writer (and kernels)
            write_score_result(res, hits, p);
            return;
        }
        aln_read_result out;
        out.c0 = out.c1 = 0;
        out.n_hits = 0;
        out.d_best = 255;
        out.best_score = 0;
        aln_hit *H = hits + static_cast<uint64_t>(r) * p.hit_cap;
        if (any) {
            uint32_t kept = 0, dbest = 255;
            for (uint32_t j = 0; j < nc; j++) {
                const uint4 c = cand[j];
                const uint32_t d = (c.z >> 28) & 7u;
                if (d <= final_b) {
                    cand[kept++] = c;
                    dbest = min(dbest, d);
                }
            }
            unsigned long long c0 = 0, c1 = 0;
            for (uint32_t j = 0; j < kept; j++) {
                const uint4 c = cand[j];
                const uint32_t d = (c.z >> 28) & 7u;
                if (d == dbest) c0 += c.y - c.x;
                else if (d == dbest + 1) c1 += c.y - c.x;
            }
            out.c0 = c0 > 0xFFFFFFFFull ? 0xFFFFFFFFu : static_cast<uint32_t>(c0);
            out.c1 = c1 > 0xFFFFFFFFull ? 0xFFFFFFFFu : static_cast<uint32_t>(c1);
            out.d_best = static_cast<uint8_t>(kept ? dbest : 255);
            const uint32_t nout = min(kept, p.hit_cap);
            if (kept > p.hit_cap) flags |= ALN_FLAG_HIT_OVERFLOW;
            for (uint32_t t = 0; t < nout; t++) {  // order (diffs, strand, k, l): selection
                uint32_t best = t;
                uint4 cb = cand[t];
                for (uint32_t j = t + 1; j < kept; j++) {
                    const uint4 cj = cand[j];
                    const uint32_t kb = ((cb.z >> 28) & 7u) << 1 | (cb.z >> 31);
                    const uint32_t kj = ((cj.z >> 28) & 7u) << 1 | (cj.z >> 31);
                    if (kj < kb || (kj == kb && (cj.x < cb.x || (cj.x == cb.x && cj.y < cb.y)))) {
                        best = j;
                        cb = cj;
                    }
                }
                cand[best] = cand[t];
                cand[t] = cb;
                aln_hit h;
                const uint32_t key = cb.z;
                h.k = cb.x;
                h.l = cb.y - 1;
                h.aligned_len = static_cast<uint16_t>(key & 0xFFFFu);
                h.strand = static_cast<uint8_t>(key >> 31);
                h.n_diff = static_cast<uint8_t>((key >> 28) & 7u);
                h.n_gapo = static_cast<uint8_t>((key >> 24) & 15u);
                h.n_gape = static_cast<uint8_t>((key >> 20) & 15u);
                h.n_mm = static_cast<uint8_t>((key >> 16) & 15u);
                h.reserved = 0;
                H[t] = h;
            }
            out.n_hits = static_cast<uint8_t>(nout);
        }
        out.flags = static_cast<uint8_t>(flags);
        res[r] = out;
        phase = PH_IDLE;
#ifdef ALN_STATS
        st_reads++;
#endif
    }

    __device__ __forceinline__ void start_strand(uint32_t n, uint32_t strand) {
        s = strand;
        sp = 0;
        base = 0;
        has_next = false;
        if ((strand ? d01 : d00) <= B) {
            next = make_uint4(0, n + 1, pack_info(0, 0, 0, 0, 0, 0, OP_M), 0);
            has_next = true;
        }
    }

    __device__ __forceinline__ void start_pass(uint32_t n, uint32_t budget) {
        B = budget;
        nc = 0;
        phase = PH_DFS;
        start_strand(n, 0);
    }

    __device__ __forceinline__ uint4 stk_get(int j) const {
        return j < SMEM ? sstk[j * kThreads] : stk[j - SMEM];
    }
    __device__ __forceinline__ void stk_set(int j, const uint4 &e) {
        if (j < SMEM) sstk[j * kThreads] = e;
        else stk[j - SMEM] = e;
    }

    __device__ __forceinline__ void push_mem(const uint4 &e) {
        if (sp == STACK_CAP && base > 0) {  // slide the live entries down over handed-out ones
            for (int j = base; j < sp; j++) stk_set(j - base, stk_get(j));
            sp -= base;
            base = 0;
        }
        if (sp < STACK_CAP) stk_set(sp++, e);
        else flags |= ALN_FLAG_STACK_OVERFLOW;
    }

    // Push a child; the newest child is held in `next` (it is what the next pop
    // would return), the one it displaces goes to the stack.
    __device__ __forceinline__ void push(uint32_t lo, uint32_t hi, uint32_t info, uint32_t id) {
        if (has_next) push_mem(next);
        next = make_uint4(lo, hi, info, id);
        has_next = true;
    }

    // Children of the node in cur / cbits given its four extensions.  Push order:
    // the match child, mismatches by base, the insertion, deletions by base (the
    // match child lowest, so that the alternatives are expanded first).  Only the
    // children that exist are visited, through a bit mask in that order.
    __device__ __forceinline__ void push_children(const uint32_t lo4[4], const uint32_t hi4[4]) {
        const uint32_t info = cur.z;
        const uint32_t i = info & 0xFFu, mm = (info >> 8) & 7u, go = (info >> 11) & 7u, ge = (info >> 14) & 7u;
        const uint32_t ni = (info >> 17) & 7u, sd = (info >> 20) & 7u, last = (info >> 23) & 3u;
        const uint32_t qi = (cbits >> 4) & 3u;
        const bool isN = cbits & 64u;
        const uint32_t sd2 = sd + ((cbits >> 7) & 1u);
        const uint32_t cid = (cbits & 256u) ? cur.w << 2 : 0u;  // track child ids below depth k
        uint32_t ne = 0;
#pragma unroll
        for (uint32_t c = 0; c < 4; c++) ne |= (hi4[c] > lo4[c] ? 1u : 0u) << c;
        uint32_t mask = 0;
        if ((cbits & 1u) && ((ne >> qi) & 1u)) mask |= 1u;
        if (cbits & 2u) mask |= (ne & (isN ? 0xFu : (0xFu & ~(1u << qi)))) << 1;
        if (cbits & 4u) mask |= 1u << 5;
        if (cbits & 8u) mask |= ne << 6;
        const uint32_t infoM = pack_info(i + 1, mm, go, ge, ni, sd, OP_M);
        const uint32_t infoX = pack_info(i + 1, mm + 1, go, ge, ni, sd2, OP_M);
        const uint32_t infoI = last == OP_I ? pack_info(i + 1, mm, go, ge + 1, ni + 1, sd2, OP_I)
                                            : pack_info(i + 1, mm, go + 1, ge, ni + 1, sd2, OP_I);
        const uint32_t infoD = last == OP_D ? pack_info(i, mm, go, ge + 1, ni, sd2, OP_D)
                                            : pack_info(i, mm, go + 1, ge, ni, sd2, OP_D);
        if (!mask) return;
        // Fast form, no data-dependent loop: every existing child but the last
        // goes to its stack slot (the displaced `next` first, then the children
        // in mask order), the last becomes `next`.  This is exactly what pushing
        // them one by one does whenever no push reaches the stack capacity.
        const uint32_t nch = __popc(mask);
        const int sp0 = sp + (has_next ? 1 : 0);
        if (sp0 + static_cast<int>(nch) - 1 <= STACK_CAP) {
            const uint32_t lastb = 31u - __clz(mask);
            if (has_next) stk_set(sp, next);
            const uint32_t loM = qi == 0 ? lo4[0] : (qi == 1 ? lo4[1] : (qi == 2 ? lo4[2] : lo4[3]));
            const uint32_t hiM = qi == 0 ? hi4[0] : (qi == 1 ? hi4[1] : (qi == 2 ? hi4[2] : hi4[3]));
#pragma unroll
            for (uint32_t b = 0; b < 10; b++) {
                const uint32_t c = b == 0 ? qi : (b <= 4 ? b - 1 : (b >= 6 ? b - 6 : 0u));
                const uint4 e = b == 0   ? make_uint4(loM, hiM, infoM, cid | qi)
                                : b <= 4 ? make_uint4(lo4[(b - 1) & 3u], hi4[(b - 1) & 3u], infoX, cid | c)
                                : b == 5 ? make_uint4(cur.x, cur.y, infoI, cur.w)
                                         : make_uint4(lo4[(b - 6) & 3u], hi4[(b - 6) & 3u], infoD, cid | c);
                if (((mask >> b) & 1u) && b != lastb)
                    stk_set(sp0 + static_cast<int>(__popc(mask & ((1u << b) - 1u))), e);
                if (b == lastb) next = e;
            }
            sp = sp0 + static_cast<int>(nch) - 1;
            has_next = true;
            return;
        }
        // a push would reach the stack capacity: one by one (compaction, overflow flag)
        while (mask) {
            const uint32_t b = __ffs(mask) - 1;
            mask &= mask - 1;
            const bool kM = b == 0, kX = b >= 1 && b <= 4, kI = b == 5;
            const uint32_t c = kM ? qi : (kX ? b - 1 : (b >= 6 ? b - 6 : 0u));
            const uint32_t clo = c == 0 ? lo4[0] : (c == 1 ? lo4[1] : (c == 2 ? lo4[2] : lo4[3]));
            const uint32_t chi = c == 0 ? hi4[0] : (c == 1 ? hi4[1] : (c == 2 ? hi4[2] : hi4[3]));
            push(kI ? cur.x : clo, kI ? cur.y : chi, kM ? infoM : (kX ? infoX : (kI ? infoI : infoD)),
                 kI ? cur.w : (cid | c));
        }
    }

    // Control: advance until the lane needs the four extensions of an interval
    // (fills fr) or is done.  Each round does O(1) work; the rounds are bounded.
    __device__ __forceinline__ void control(const DIndex &X, const ReadBatch &rb, uint32_t n_reads,
                                            const SearchParams &p, aln_read_result *res, aln_hit *hits,
                                            uint32_t *queue, const uint32_t *order, const uint2 *dbp,
                                            uint32_t *sb, uint32_t *sn, FetchReq &fr) {
        const uint32_t n = X.t[0].n;  // both texts have the same length
        fr.kind = F_NONE;
        for (int round = 0; round < 32; round++) {
            if (phase == PH_DONE || phase == PH_FREE || phase == PH_RETURN) return;
            if (phase == PH_WAIT) {
                if (outstanding) return;
                phase = PH_DFS;
            }
#ifdef ALN_STATS
            st_rounds++;
#endif
            if (phase == PH_IDLE) {
                if (heavy_seen) return;  // stay idle this trip: the hand-over may give it a heavy read's subtree
                r = atomicAdd(queue, 1u);
                if (r >= n_reads) {
                    phase = PH_FREE;
                    return;
                }
                if (order) r = order[r];
                role = ROLE_OWN;
                rv = own_rv;
                m = rb.len[r];
                z = rb.z ? rb.z[r] : p.z;
                flags = 0;
                work = 0;
                nc = 0;
                if (m > ALN_MAX_READ_LEN) flags |= ALN_FLAG_READ_TOO_LONG;
                if (z > ALN_MAX_Z || z > p.z) flags |= ALN_FLAG_BAD_LIMIT;
                if (flags || m == 0) {
                    write_result(res, hits, p, false, 0);
                    continue;
                }
                load_read(rb, rb.offset[r], m, sb, sn);
                if (dbp) {  // D from the pre-pass: go straight to the first pass
                    const uint2 a = dbp[2ull * r], b = dbp[2ull * r + 1];
                    bpa0 = a.x;
                    bpa1 = a.y;
                    bpb0 = b.x;
                    bpb1 = b.y;
                    d00 = d_at(bpa0, bpa1, 0);
                    d01 = d_at(bpb0, bpb1, 0);
                    const uint32_t lb = min(d00, d01);
                    if (lb > z) {
                        write_result(res, hits, p, false, 0);
                        continue;
                    }
                    start_pass(n, p.strata != ALN_STRATA_BEST1 ? z : min(z, lb + 1));
                    continue;
                }
                phase = PH_DSCAN;
                s = 0;
                dj = static_cast<int>(m) - 1;
                dcnt = 0;
                dlo = 0;
                dhi = n + 1;
                dsl = 0;
                dsid = 0;
                bpa0 = bpa1 = bpb0 = bpb1 = 0;
                continue;
            }
            if (phase == PH_DSCAN) {
                const uint32_t zcap = min(z + 1, 8u);
                if (dj < 0 || dcnt >= zcap) {
                    if (s == 0) {
                        d00 = d_at(bpa0, bpa1, 0);
                        s = 1;
                        dj = static_cast<int>(m) - 1;
                        dcnt = 0;
                        dlo = 0;
                        dhi = n + 1;
                        dsl = 0;
                        dsid = 0;
                        continue;
                    }
                    d01 = d_at(bpb0, bpb1, 0);
                    const uint32_t lb = min(d00, d01);
                    if (lb > z) {
                        write_result(res, hits, p, false, 0);
                        continue;
                    }
                    start_pass(n, p.strata != ALN_STRATA_BEST1 ? z : min(z, lb + 1));
                    continue;
                }
                // strand 0's D comes from X, strand 1's from X reversed
                if (rv.isN(static_cast<uint32_t>(dj))) {
                    record_fail();
                    dlo = 0;
                    dhi = n + 1;
                    dsl = 0;
                    dsid = 0;
                    dj--;
                    continue;
                }
                fr.text = s;
                if (dsl == 0) {
                    fr.kind = F_ROOT;
                } else if (dsl < K) {
                    fr.kind = F_TABLE;
                    fr.toff = trie_off(dsl + 1) + (dsid << 2);
                } else {
                    fr.kind = F_OCC;
                    fr.lo = dlo;
                    fr.hi = dhi;
                }
                return;
            }
            // PH_DFS
            if (!has_next && sp == base) {
                sp = base = 0;
                if (role == ROLE_HELP) {  // subtree done: hand the candidates back
                    phase = PH_RETURN;
                    ret_i = 0;
                    return;
                }
                if (outstanding) {  // wait for handed-out subtrees before the pass ends
                    phase = PH_WAIT;
                    return;
                }
                if (s == 0) {
                    start_strand(n, 1);
                    continue;
                }
                if (flags & kFlagDemoted) {  // the heavy phase searches it and writes the result
                    phase = PH_IDLE;
                    continue;
                }
                if ((flags & ALN_FLAG_WORK_LIMIT) || p.strata != ALN_STRATA_BEST1) {
                    write_result(res, hits, p, nc > 0, z);
                    continue;
                }
                if (nc == 0) {
                    if (B >= z) {
                        write_result(res, hits, p, false, 0);
                        continue;
                    }
                    start_pass(n, min(z, B + 2));
                    continue;
                }
                uint32_t dmin = 255;
                for (uint32_t j = 0; j < nc; j++) dmin = min(dmin, (cand[j].z >> 28) & 7u);
                const uint32_t F = min(z, dmin + 1);
                if (F <= B) {
                    write_result(res, hits, p, true, F);
                    continue;
                }
                start_pass(n, F);
                continue;
            }
            if (role == ROLE_OWN && work > p.heavy_after && (flags & kFlagDrained) && p.heavy.hdr &&
                !(flags & kFlagHeavyTried)) {
                // the batch's tail: hand the read to the heavy phase if it has room
                flags |= kFlagHeavyTried;
                const uint32_t hid = atomicAdd(&p.heavy.hdr->n_heavy, 1u);
                if (hid < kHeavyReads) {
                    HeavyRead *H = p.heavy.reads + hid;
                    H->r = r;
                    H->B = B;  // the heavy phase resumes at this deepening pass
                    H->z = z;
                    H->m = m;
                    flags |= kFlagDemoted;
                    sp = base;
                    has_next = false;
                    s = 1;
                    continue;
                }
            }
            if (++work > p.work_limit) {
                flags |= ALN_FLAG_WORK_LIMIT;
                sp = base;
                has_next = false;
                if (role == ROLE_OWN) s = 1;
                continue;
            }
            if (expand_top(p, fr)) return;
        }
    }

    // Pop the top node and decide its children: false if nothing needs fetching
    // (an emitted hit, or every child pruned), true with fr filled otherwise.
    __device__ __forceinline__ bool expand_top(const SearchParams &p, FetchReq &fr) {
        uint4 e;
        if (has_next) {
            e = next;
            has_next = false;
        } else {
            e = stk_get(--sp);
        }
#ifdef ALN_STATS
        st_pops++;
#endif
        const uint32_t info = e.z;
        const uint32_t i = info & 0xFFu, mm = (info >> 8) & 7u, go = (info >> 11) & 7u, ge = (info >> 14) & 7u;
        const uint32_t ni = (info >> 17) & 7u, sd = (info >> 20) & 7u, last = (info >> 23) & 3u;
        const uint32_t diffs = mm + go + ge;
        const uint32_t rem = B - diffs;
        if (i == m) {
            const uint32_t alen = m + (go + ge - ni) - ni;
            if (alen >= 1)
                add_cand(e.x, e.y, (s << 31) | (diffs << 28) | (go << 24) | (ge << 20) | (mm << 16) | alen,
                         SCORE ? p.sc_mm * mm + p.sc_go * go + p.sc_ge * ge : 0u);
            return false;
        }
        const uint32_t bp0 = s ? bpb0 : bpa0, bp1 = s ? bpb1 : bpa1;
        const bool isN = rv.isN(i);
        const uint32_t qi = rv.base(i) ^ (s ? 3u : 0u);
        const uint32_t Dn = d_at(bp0, bp1, i + 1), Di = d_at(bp0, bp1, i);
        const uint32_t e1 = p.e < 1 ? 1 : p.e;
        const bool in_seed = p.seed_len && i < p.seed_len;
        const bool alt = rem >= 1 && (!in_seed || sd < p.seed_z);
        const bool allowM = !isN && rem >= Dn;
        const bool mm_ok = alt && rem - 1 >= Dn;
        const bool ins_ok = alt && rem - 1 >= Dn && i >= p.e && i + 1 + p.e <= m && last != OP_D &&
                            (last == OP_I ? ge < p.max_gape : go < p.max_gapo);
        const bool del_ok = alt && rem - 1 >= Di && i >= e1 && i + e1 <= m && last != OP_I &&
                            (last == OP_D ? ge < p.max_gape : go < p.max_gapo);
        const uint32_t L = i + go + ge - 2 * ni;  // target length: consumed + deleted - inserted
        cur = e;
        cbits = (allowM ? 1u : 0u) | (mm_ok ? 2u : 0u) | (ins_ok ? 4u : 0u) | (del_ok ? 8u : 0u) | (qi << 4) |
                (isN ? 64u : 0u) | (in_seed ? 128u : 0u) | (L < K ? 256u : 0u);
        if (!(allowM || mm_ok || del_ok || ins_ok)) return false;
        fr.text = s ? 0u : 1u;  // strand 0 searches X reversed, strand 1 searches X
        if (!(allowM || mm_ok || del_ok)) {
            fr.kind = F_ZERO;  // only the insertion child: no extension needed
        } else if (L == 0) {
            fr.kind = F_ROOT;
        } else if (L < K) {
            fr.kind = F_TABLE;
            fr.toff = trie_off(L + 1) + (e.w << 2);
        } else {
            fr.kind = F_OCC;
            fr.lo = e.x;
            fr.hi = e.y;
        }
        return true;
    }

    // Warp-synchronous hand-over, once per trip, all 32 lanes: returning helpers
    // send one candidate (or their completion) to the owner; then lanes without
    // work take the bottom stack entry of a lane with at least two pending
    // entries: a free lane (the read queue is empty) from any such lane, an idle
    // lane (it has finished its read and the queue may still hold reads) only
    // from a heavy one, a lane searching a read with more than help_after
    // expansions or a helper, so that a heavy read is searched by the idle lanes
    // of its warp before they take new reads.  A helper that has handed its
    // candidates back goes idle (it takes the next read, or becomes free).
    __device__ __forceinline__ void give(uint32_t lane, uint32_t rcv, uint32_t dnr, const uint32_t *sbase,
                                         const uint32_t *snbase, uint32_t warp_col) {
        const unsigned FULL = 0xFFFFFFFFu;
        const bool giver = lane == dnr;
        const uint4 e = giver ? stk_get(base) : make_uint4(0, 0, 0, 0);
        const uint32_t ex = __shfl_sync(FULL, e.x, dnr), ey = __shfl_sync(FULL, e.y, dnr);
        const uint32_t ez = __shfl_sync(FULL, e.z, dnr), ew = __shfl_sync(FULL, e.w, dnr);
        const uint32_t o = __shfl_sync(FULL, role == ROLE_OWN ? lane : owner, dnr);
        const uint32_t hm = __shfl_sync(FULL, m, dnr), hB = __shfl_sync(FULL, B, dnr);
        const uint32_t hs = __shfl_sync(FULL, s, dnr), hz = __shfl_sync(FULL, z, dnr);
        const uint32_t hr = __shfl_sync(FULL, r, dnr);  // the read (the heavy phase: its list entry)
        const uint32_t h0 = __shfl_sync(FULL, s ? bpb0 : bpa0, dnr);
        const uint32_t h1 = __shfl_sync(FULL, s ? bpb1 : bpa1, dnr);
        if (giver) base++;
        if (lane == o) outstanding++;
        if (lane == rcv) {
            role = ROLE_HELP;
            owner = o;
            r = hr;
            m = hm;
            B = hB;
            s = hs;
            z = hz;
            if (hs) { bpb0 = h0; bpb1 = h1; } else { bpa0 = h0; bpa1 = h1; }
            next = make_uint4(ex, ey, ez, ew);
            has_next = true;
            sp = 0;
            base = 0;
            nc = 0;
            work = 0;
            flags = 0;
            phase = PH_DFS;
            rv = ReadView{sbase + warp_col + o, snbase + warp_col + o};
        }
    }

    __device__ __forceinline__ void exchange(uint32_t lane, const uint32_t *sbase, const uint32_t *snbase,
                                             uint32_t warp_col, uint32_t help_after) {
        const unsigned FULL = 0xFFFFFFFFu;
        // one vote decides whether there is anything to hand over this trip: a
        // returning helper, a lane without work, a read just handed to the heavy
        // phase, or (with a finite help_after) a read heavy enough to share
        const bool want = phase == PH_RETURN || phase == PH_FREE || (phase == PH_IDLE && heavy_seen) ||
                          (flags & kFlagDemoted) || (phase == PH_DFS && work > help_after);
        if (!__any_sync(FULL, want)) return;
        unsigned ret = __ballot_sync(FULL, phase == PH_RETURN);
        while (ret) {
            const uint32_t src = __ffs(ret) - 1;
            ret &= ret - 1;
            const bool mine = lane == src;
            const uint32_t o = __shfl_sync(FULL, owner, src);
            const uint32_t has = __shfl_sync(FULL, (mine && ret_i < nc) ? 1u : 0u, src);
            const uint4 c = (mine && ret_i < nc) ? cand[ret_i] : make_uint4(0, 0, 0, 0);
            const uint32_t cx = __shfl_sync(FULL, c.x, src), cy = __shfl_sync(FULL, c.y, src),
                           cz = __shfl_sync(FULL, c.z, src), cw = SCORE ? __shfl_sync(FULL, c.w, src) : 0u;
            const uint32_t hf = __shfl_sync(FULL, flags, src);
            if (lane == o) {
                if (has) add_cand(cx, cy, cz, cw);
                else {
                    outstanding--;
                    flags |= hf & ALN_FLAG_INCOMPLETE;
                }
            }
            if (mine) {
                if (has) ret_i++;
                else {
                    phase = PH_IDLE;
                    role = ROLE_OWN;
                    rv = own_rv;
                }
            }
        }
        // helpers of a read just handed to the heavy phase drop their subtrees
        const unsigned dem = __ballot_sync(FULL, role == ROLE_OWN && (flags & kFlagDemoted));
        if (dem && role == ROLE_HELP && ((dem >> owner) & 1u) && phase == PH_DFS) {
            sp = base;
            has_next = false;
            nc = 0;
        }
        const bool can_give = phase == PH_DFS && (sp - base >= 2 || (sp - base >= 1 && has_next));
        unsigned donm = __ballot_sync(FULL, can_give);
        unsigned heavym = __ballot_sync(FULL, can_give && (role == ROLE_HELP || work > help_after));
        unsigned freem = __ballot_sync(FULL, phase == PH_FREE);
        unsigned idlem = __ballot_sync(FULL, phase == PH_IDLE && heavy_seen);
        if (freem) flags |= kFlagDrained;  // the queue is empty for good: heavy reads may be handed over
        heavy_seen = heavym != 0;
        while (freem && donm) {
            const uint32_t rcv = __ffs(freem) - 1, dnr = __ffs(donm) - 1;
            freem &= freem - 1;
            donm &= donm - 1;
            heavym &= ~(1u << dnr);
            give(lane, rcv, dnr, sbase, snbase, warp_col);
        }
        while (idlem && heavym) {
            const uint32_t rcv = __ffs(idlem) - 1, dnr = __ffs(heavym) - 1;
            idlem &= idlem - 1;
            heavym &= heavym - 1;
            give(lane, rcv, dnr, sbase, snbase, warp_col);
        }
    }

    // The launch's loop bound was reached (the warp leaves its loop together):
    // the lane's own unfinished read, and every read it can still take from the
    // queue, get an empty result flagged ALN_FLAG_LOOP_LIMIT, so that no read is
    // left without a result.  A helper's subtree belongs to an owner lane of the
    // same warp, which is flagged here.
    __device__ void stop_at_limit(uint32_t lane, uint32_t n_reads, const SearchParams &p, aln_read_result *res,
                                  uint32_t *queue, const uint32_t *order) {
        if (lane == 0 && p.status) atomicOr(p.status, ALN_STATUS_LOOP_LIMIT);
        aln_read_result out;
        out.c0 = out.c1 = 0;
        out.n_hits = 0;
        out.d_best = 255;
        out.best_score = 0;
        if (role == ROLE_OWN && (phase == PH_DSCAN || phase == PH_DFS || phase == PH_WAIT)) {
            out.flags = static_cast<uint8_t>(flags | ALN_FLAG_LOOP_LIMIT);
            res[r] = out;
        }
        out.flags = ALN_FLAG_LOOP_LIMIT;
        for (;;) {  // ends: the counter only grows, and each lane stops at n_reads
            uint32_t q = atomicAdd(queue, 1u);
            if (q >= n_reads) break;
            res[order ? order[q] : q] = out;
        }
        phase = PH_FREE;
    }


    __device__ __forceinline__ void apply(const DIndex &X, const uint32_t lo4[4], const uint32_t hi4[4]) {
        if (phase == PH_DSCAN) {
            const uint32_t c = rv.base(static_cast<uint32_t>(dj)) ^ (s ? 3u : 0u);
            dlo = c == 0 ? lo4[0] : (c == 1 ? lo4[1] : (c == 2 ? lo4[2] : lo4[3]));
            dhi = c == 0 ? hi4[0] : (c == 1 ? hi4[1] : (c == 2 ? hi4[2] : hi4[3]));
            if (dhi <= dlo) {
                record_fail();
                dlo = 0;
                dhi = X.t[0].n + 1;
                dsl = 0;
                dsid = 0;
            } else {
                dsid = dsl < K ? (dsid << 2) | c : 0u;
                dsl++;
            }
            dj--;
        } else {
            push_children(lo4, hi4);
        }
    }
};

// The four extensions for a fetch request.
__device__ __forceinline__ void fetch4(const DIndex &X, const FetchReq &fr, uint32_t lo4[4], uint32_t hi4[4]) {
    const DText T = fr.text ? X.t[1] : X.t[0];
    if (fr.kind == F_ROOT) {  // the empty string: children are the C ranges
#pragma unroll
        for (int c = 0; c < 4; c++) {
            lo4[c] = T.C1[c];
            hi4[c] = T.C1[c + 1];
        }
    } else if (fr.kind == F_ZERO) {
#pragma unroll
        for (int c = 0; c < 4; c++) lo4[c] = hi4[c] = 0;
    } else if (fr.kind == F_TABLE) {
        const uint4 *g = reinterpret_cast<const uint4 *>(T.kmer + fr.toff);
        const uint4 a = ld_nc(g), b = ld_nc(g + 1);
        lo4[0] = a.x; hi4[0] = a.y; lo4[1] = a.z; hi4[1] = a.w;
        lo4[2] = b.x; hi4[2] = b.y; lo4[3] = b.z; hi4[3] = b.w;
    } else {
        lf4(T, fr.lo, fr.hi, lo4, hi4);
    }
}

}  // namespace aln
