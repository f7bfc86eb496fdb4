// Per-read bounded backtracking search (sm_103a), shared by the plain and the
// persistent kernels.
//
// Paper Sec. 2: the search keeps a lower and an upper pointer that every read
// base updates from the index, and for non-exact matches backs up and tries
// alternatives.  The alternatives and their limits follow BWA's short-read
// method:
//   strand 0 (forward) searches q = W on the index of X reversed, strand 1
//   (reverse) searches q = complement(W) on the index of X; both consume the
//   read from its 5' end, so the seed is consumed first;
//   D (lower bound on the differences needed by q[i..m-1]) comes from a greedy
//   scan of q from its 3' end on the other strand's index: a segment is grown
//   until it no longer occurs (or meets an N), which costs one difference, and
//   the scan restarts;
//   children of a node (i, [lo, hi), counts, last op): match / mismatch to each
//   base, insertion of q[i], deletion of a target base before read index i;
//   a run of insertions or of deletions of length g = 1 gap open + g-1 gap
//   extensions = g differences; a node is kept only if budget - diffs >= D.
// An insertion directly after a deletion (or the reverse) reaches the same
// target as a single mismatch with strictly more differences, gap opens and
// seed differences, and every continuation of it is dominated too, so such
// paths are skipped: the hit set and the minimal witnesses are unchanged.
#pragma once

#include <cstdint>

#include "aln_device.cuh"
#include "aln_gb300.h"

namespace aln {

constexpr int kThreads = 128;   // threads per block of the search kernels
constexpr int kReadWords = 16;  // 2-bit words for ALN_MAX_READ_LEN bases
constexpr int kMaskWords = 8;   // N-mask words
constexpr int kCandCap = ALN_CAND_CAP;
constexpr uint32_t kDefaultWorkLimit = 1u << 24;
constexpr uint32_t kDefaultHelpAfter = 0xFFFFFFFFu;  // only once the read queue is empty
constexpr uint32_t kDefaultHeavyAfter = ALN_HEAVY_AFTER_DEFAULT;

enum : uint32_t { OP_M = 0, OP_I = 1, OP_D = 2 };

struct ReadBatch {
    const uint32_t *bases;
    const uint32_t *nmask;
    const uint64_t *offset;
    const uint16_t *len;
    const uint8_t *z;
};

// Heavy-read phase (device-wide search of the reads that passed heavy_after
// expansions in the persistent search): its state lives in the call's scratch.
constexpr uint32_t kHeavyReads = 2048;     // reads the heavy phase takes per call
constexpr uint32_t kHeavySlots = 1024;     // candidate hash slots per read and strand
constexpr uint32_t kHeavyPool = 1u << 20;  // task ring capacity
constexpr uint32_t kHeavyPasses = ALN_HEAVY_PASSES;  // deepening passes launched (enough for z <= 7)

struct HeavyHdr {   // 512 bytes: the ring's hot counters on 128-byte lines of their own
    uint32_t n_heavy;      // reads handed over (may pass kHeavyReads: those stay in the first phase)
    uint32_t pad0;
    unsigned long long expansions;  // node expansions made by the heavy phase's tasks (a statistic)
    unsigned long long lane_trips;  // lane trips of the pass kernels, and those with a task (statistics)
    unsigned long long busy_trips;
    uint32_t pad1[24];
    uint32_t head;         // task ring ticket: taken
    uint32_t pad2[31];
    uint32_t tail;         // task ring ticket: published
    uint32_t pad3[31];
    uint32_t outstanding;  // tasks of the current pass not yet finished
    uint32_t pad4[31];
};
static_assert(sizeof(HeavyHdr) == 512, "heavy header layout");
struct HeavyRead {  // 64 bytes
    uint32_t r, B, z, m;   // read index, pass budget, difference limit, length
    uint32_t state;        // 0 searching, 1 result written
    uint32_t flags;        // ALN_FLAG_* gathered from the tasks
    uint32_t distinct[2];  // distinct candidates per strand in this pass
    uint32_t pad[8];
};
struct HeavyTask {  // 32 bytes
    uint4 node;
    uint32_t hid, s, pad0, pad1;
};
struct HeavySlot {  // 16 bytes: a candidate (lo, hi) of one strand with its least witness
    unsigned long long id;    // lo << 32 | hi; 0 = empty
    unsigned long long wkey;  // score << 32 | witness key (score 0 outside the score-ordered mode)
};
struct HeavyCtx {
    HeavyHdr *hdr;
    HeavyRead *reads;
    HeavySlot *slots;      // [hid][strand][kHeavySlots]
    HeavyTask *pool;
    uint32_t *ready;       // ready[t % kHeavyPool] = t + 1 once task t is written
};

struct SearchParams {
    uint32_t z, max_gapo, max_gape, seed_len, seed_z, e, hit_cap, strata, work_limit, blocks_per_sm;
    uint32_t smem_stack;            // persistent form: stack entries per lane in shared memory
    uint32_t help_after;            // persistent form: expansions after which a read takes idle lanes
    uint32_t heavy_after;           // persistent form: owner expansions after which a read goes to the heavy phase
    uint32_t sc_mm, sc_go, sc_ge, max_best;  // score-ordered mode: penalties and the cap on best places
    HeavyCtx heavy;                 // heavy phase state (hdr == nullptr: no heavy phase)
    unsigned long long loop_limit;  // persistent form: loop trips per warp
    uint32_t *status;               // ALN_STATUS_* bits, or nullptr
    void *window_base;              // persistent form: L2 persisting window (prefix-trie tables), or nullptr
    uint64_t window_bytes;
    float window_hit_ratio;
};

// Stack-entry info word: i (8) | n_mm (3) | n_gapo (3) | n_gape (3) | n_ins (3) | seed (3) | last (2)
__device__ __forceinline__ uint32_t pack_info(uint32_t i, uint32_t mm, uint32_t go, uint32_t ge, uint32_t ni,
                                              uint32_t sd, uint32_t last) {
    return i | (mm << 8) | (go << 11) | (ge << 14) | (ni << 17) | (sd << 20) | (last << 23);
}

// D(i) from the breakpoint bytes: each byte holds j+1 for a failure at read
// index j (0 = unused), D(i) = number of failures at indices >= i.
__device__ __forceinline__ uint32_t d_at(uint32_t bp0, uint32_t bp1, uint32_t i) {
    const uint32_t ii = i * 0x01010101u;
    return (__popc(__vcmpgtu4(bp0, ii)) + __popc(__vcmpgtu4(bp1, ii))) >> 3;
}

struct ReadView {
    const uint32_t *sb;  // read bases in shared memory, word w at sb[w * kThreads]
    const uint32_t *sn;  // N mask words, same layout
    __device__ __forceinline__ uint32_t base(uint32_t i) const { return (sb[(i >> 4) * kThreads] >> (2 * (i & 15u))) & 3u; }
    __device__ __forceinline__ bool isN(uint32_t i) const { return (sn[(i >> 5) * kThreads] >> (i & 31u)) & 1u; }
};

// Copy read bits [off, off+m) of a packed stream into per-thread shared words.
__device__ __forceinline__ void load_read(const ReadBatch &rb, uint64_t off, uint32_t m, uint32_t *sb, uint32_t *sn) {
    const uint32_t nw = (m + 15) >> 4;
    const uint64_t w0 = off >> 4;
    const uint32_t sh = static_cast<uint32_t>(off & 15u) * 2;
    const uint64_t last = (off + m - 1) >> 4;
    for (uint32_t w = 0; w < nw; w++) {
        uint32_t a = __ldg(rb.bases + w0 + w);
        uint32_t b = (sh && w0 + w + 1 <= last) ? __ldg(rb.bases + w0 + w + 1) : 0u;
        sb[w * kThreads] = sh ? __funnelshift_r(a, b, sh) : a;
    }
    const uint32_t mw = (m + 31) >> 5;
    if (rb.nmask) {
        const uint64_t v0 = off >> 5;
        const uint32_t vs = static_cast<uint32_t>(off & 31u);
        const uint64_t vlast = (off + m - 1) >> 5;
        for (uint32_t w = 0; w < mw; w++) {
            uint32_t a = __ldg(rb.nmask + v0 + w);
            uint32_t b = (vs && v0 + w + 1 <= vlast) ? __ldg(rb.nmask + v0 + w + 1) : 0u;
            uint32_t v = vs ? __funnelshift_r(a, b, vs) : a;
            const uint32_t left = m - 32 * w;  // clear bits past the read end
            if (left < 32) v &= (1u << left) - 1u;
            sn[w * kThreads] = v;
        }
    } else {
        for (uint32_t w = 0; w < mw; w++) sn[w * kThreads] = 0u;
    }
}

// Greedy D scan of strand s on the other index, from the 3' end.  Stops after
// zcap failures (D >= zcap prunes everything).  Returns the number of steps.
__device__ __forceinline__ uint32_t d_scan(const DText &O, const ReadView &rv, uint32_t m, uint32_t strand,
                                           uint32_t zcap, uint32_t &bp0, uint32_t &bp1) {
    bp0 = bp1 = 0;
    uint32_t lo = 0, hi = O.n + 1, cnt = 0, steps = 0;
    for (int j = static_cast<int>(m) - 1; j >= 0; j--) {
        bool ok = false;
        if (!rv.isN(j)) {
            const uint32_t c = rv.base(j) ^ (strand ? 3u : 0u);
            lf1(O, c, lo, hi);
            ok = hi > lo;
            steps++;
        }
        if (!ok) {
            const uint32_t v = static_cast<uint32_t>(j) + 1u;
            if (cnt < 4) bp0 |= v << (8 * cnt);
            else bp1 |= v << (8 * (cnt - 4));
            cnt++;
            lo = 0;
            hi = O.n + 1;
            if (cnt >= zcap || cnt >= 8) break;
        }
    }
    return steps;
}

template <int STACK_CAP>
struct Search {
    // candidates: lo, hi, key = strand<<31 | diffs<<28 | gapo<<24 | gape<<20 | mm<<16 | aligned_len
    uint32_t clo[kCandCap], chi[kCandCap], ckey[kCandCap];
    uint32_t slo[STACK_CAP], shi[STACK_CAP], sinfo[STACK_CAP];
    uint32_t nc;
    uint32_t flags;
    uint32_t work;

    __device__ __forceinline__ void add_cand(uint32_t lo, uint32_t hi, uint32_t key) {
        for (uint32_t j = 0; j < nc; j++) {
            if (clo[j] == lo && chi[j] == hi && (ckey[j] >> 31) == (key >> 31)) {
                if (key < ckey[j]) ckey[j] = key;
                return;
            }
        }
        if (nc < kCandCap) {
            clo[nc] = lo;
            chi[nc] = hi;
            ckey[nc] = key;
            nc++;
        } else {
            flags |= ALN_FLAG_CAND_OVERFLOW;
        }
    }

    // Depth-first enumeration of strand s at budget B.
    __device__ void dfs(const DText &I, const ReadView &rv, uint32_t m, uint32_t strand, uint32_t B,
                        uint32_t bp0, uint32_t bp1, const SearchParams &p) {
        const uint32_t flip = strand ? 3u : 0u;
        const uint32_t e1 = p.e < 1 ? 1 : p.e;
        int sp = 0;
        slo[0] = 0;
        shi[0] = I.n + 1;
        sinfo[0] = pack_info(0, 0, 0, 0, 0, 0, OP_M);
        sp = 1;
        while (sp > 0) {
            if (++work > p.work_limit) {
                flags |= ALN_FLAG_WORK_LIMIT;
                return;
            }
            sp--;
            const uint32_t lo = slo[sp], hi = shi[sp], info = sinfo[sp];
            const uint32_t i = info & 0xFFu, mm = (info >> 8) & 7u, go = (info >> 11) & 7u, ge = (info >> 14) & 7u;
            const uint32_t ni = (info >> 17) & 7u, sd = (info >> 20) & 7u, last = (info >> 23) & 3u;
            const uint32_t diffs = mm + go + ge;
            const uint32_t rem = B - diffs;
            if (i == m) {
                const uint32_t alen = m + (go + ge - ni) - ni;
                if (alen >= 1)
                    add_cand(lo, hi, (strand << 31) | (diffs << 28) | (go << 24) | (ge << 20) | (mm << 16) | alen);
                continue;
            }
            const bool isN = rv.isN(i);
            const uint32_t qi = rv.base(i) ^ flip;
            const uint32_t Dn = d_at(bp0, bp1, i + 1), Di = d_at(bp0, bp1, i);
            const bool in_seed = p.seed_len && i < p.seed_len;
            const bool alt = rem >= 1 && (!in_seed || sd < p.seed_z);
            const bool allowM = !isN && rem >= Dn;
            const bool mm_ok = alt && rem - 1 >= Dn;
            const bool ins_ok = alt && rem - 1 >= Dn && i >= p.e && i + 1 + p.e <= m && last != OP_D &&
                                (last == OP_I ? ge < p.max_gape : go < p.max_gapo);
            const bool del_ok = alt && rem - 1 >= Di && i >= e1 && i + e1 <= m && last != OP_I &&
                                (last == OP_D ? ge < p.max_gape : go < p.max_gapo);
            const uint32_t sd2 = sd + (in_seed ? 1u : 0u);
            uint32_t lo4[4], hi4[4];
            if (allowM || mm_ok || del_ok) lf4(I, lo, hi, lo4, hi4);
            // match child first (deepest), then the alternatives on top
            if (allowM && hi4[qi] > lo4[qi]) {
                if (sp < STACK_CAP) {
                    slo[sp] = lo4[qi]; shi[sp] = hi4[qi];
                    sinfo[sp] = pack_info(i + 1, mm, go, ge, ni, sd, OP_M);
                    sp++;
                } else flags |= ALN_FLAG_STACK_OVERFLOW;
            }
            if (mm_ok) {
#pragma unroll
                for (uint32_t c = 0; c < 4; c++) {
                    if ((c != qi || isN) && hi4[c] > lo4[c]) {
                        if (sp < STACK_CAP) {
                            slo[sp] = lo4[c]; shi[sp] = hi4[c];
                            sinfo[sp] = pack_info(i + 1, mm + 1, go, ge, ni, sd2, OP_M);
                            sp++;
                        } else flags |= ALN_FLAG_STACK_OVERFLOW;
                    }
                }
            }
            if (ins_ok) {
                if (sp < STACK_CAP) {
                    slo[sp] = lo; shi[sp] = hi;
                    sinfo[sp] = last == OP_I ? pack_info(i + 1, mm, go, ge + 1, ni + 1, sd2, OP_I)
                                             : pack_info(i + 1, mm, go + 1, ge, ni + 1, sd2, OP_I);
                    sp++;
                } else flags |= ALN_FLAG_STACK_OVERFLOW;
            }
            if (del_ok) {
#pragma unroll
                for (uint32_t c = 0; c < 4; c++) {
                    if (hi4[c] > lo4[c]) {
                        if (sp < STACK_CAP) {
                            slo[sp] = lo4[c]; shi[sp] = hi4[c];
                            sinfo[sp] = last == OP_D ? pack_info(i, mm, go, ge + 1, ni, sd2, OP_D)
                                                     : pack_info(i, mm, go + 1, ge, ni, sd2, OP_D);
                            sp++;
                        } else flags |= ALN_FLAG_STACK_OVERFLOW;
                    }
                }
            }
        }
    }

    // Whole read: D scans, iterative deepening over budgets, reduction, output.
    __device__ void run(const DIndex &X, const ReadView &rv, uint32_t m, uint32_t z, const SearchParams &p,
                        aln_read_result *res, aln_hit *hits) {
        nc = 0;
        flags = 0;
        work = 0;
        aln_read_result out;
        out.c0 = out.c1 = 0;
        out.n_hits = 0;
        out.d_best = 255;
        out.best_score = 0;
        if (m > ALN_MAX_READ_LEN) flags |= ALN_FLAG_READ_TOO_LONG;
        if (z > ALN_MAX_Z || z > p.z) flags |= ALN_FLAG_BAD_LIMIT;
        if (flags || m == 0) {
            out.flags = static_cast<uint8_t>(flags);
            *res = out;
            return;
        }
        uint32_t bp[2][2];
        uint32_t d0[2];
        for (uint32_t s = 0; s < 2; s++) {
            // strand 0's other index is X, strand 1's is X reversed
            d_scan(X.t[s], rv, m, s, z + 1, bp[s][0], bp[s][1]);
            d0[s] = d_at(bp[s][0], bp[s][1], 0);
        }
        uint32_t lb = min(d0[0], d0[1]);
        uint32_t final_b = z;
        bool any = false;
        if (lb <= z) {
            uint32_t B = (p.strata == ALN_STRATA_FULL) ? z : min(z, lb + 1);
            for (;;) {
                nc = 0;
                for (uint32_t s = 0; s < 2; s++)
                    if (d0[s] <= B) dfs(X.t[s ? 0 : 1], rv, m, s, B, bp[s][0], bp[s][1], p);
                if (flags & ALN_FLAG_WORK_LIMIT) break;
                if (p.strata == ALN_STRATA_FULL) {
                    final_b = z;
                    any = nc > 0;
                    break;
                }
                if (nc == 0) {
                    if (B >= z) break;
                    const uint32_t b = B + 1;
                    B = min(z, b + 1);
                    continue;
                }
                uint32_t dmin = 255;
                for (uint32_t j = 0; j < nc; j++) dmin = min(dmin, (ckey[j] >> 28) & 7u);
                const uint32_t F = min(z, dmin + 1);
                if (F <= B) {
                    final_b = F;
                    any = true;
                    break;
                }
                B = F;
            }
        }
        if (any) {
            // keep diffs <= final budget; c0 / c1 over the kept hits
            uint32_t kept = 0, dbest = 255;
            for (uint32_t j = 0; j < nc; j++) {
                const uint32_t d = (ckey[j] >> 28) & 7u;
                if (d <= final_b) {
                    clo[kept] = clo[j];
                    chi[kept] = chi[j];
                    ckey[kept] = ckey[j];
                    kept++;
                    dbest = min(dbest, d);
                }
            }
            unsigned long long c0 = 0, c1 = 0;
            for (uint32_t j = 0; j < kept; j++) {
                const uint32_t d = (ckey[j] >> 28) & 7u;
                const unsigned long long w = chi[j] - clo[j];
                if (d == dbest) c0 += w;
                else if (d == dbest + 1) c1 += w;
            }
            out.c0 = c0 > 0xFFFFFFFFull ? 0xFFFFFFFFu : static_cast<uint32_t>(c0);
            out.c1 = c1 > 0xFFFFFFFFull ? 0xFFFFFFFFu : static_cast<uint32_t>(c1);
            out.d_best = static_cast<uint8_t>(dbest);
            // order (diffs, strand, k, l): selection of the hit_cap smallest
            const uint32_t nout = min(kept, p.hit_cap);
            if (kept > p.hit_cap) flags |= ALN_FLAG_HIT_OVERFLOW;
            for (uint32_t t = 0; t < nout; t++) {
                uint32_t best = t;
                for (uint32_t j = t + 1; j < kept; j++) {
                    const uint32_t kb = ((ckey[best] >> 28) & 7u) << 1 | (ckey[best] >> 31);
                    const uint32_t kj = ((ckey[j] >> 28) & 7u) << 1 | (ckey[j] >> 31);
                    if (kj < kb || (kj == kb && (clo[j] < clo[best] || (clo[j] == clo[best] && chi[j] < chi[best]))))
                        best = j;
                }
                uint32_t tl = clo[t], th = chi[t], tk = ckey[t];
                clo[t] = clo[best]; chi[t] = chi[best]; ckey[t] = ckey[best];
                clo[best] = tl; chi[best] = th; ckey[best] = tk;
                aln_hit h;
                const uint32_t key = ckey[t];
                h.k = clo[t];
                h.l = chi[t] - 1;
                h.aligned_len = static_cast<uint16_t>(key & 0xFFFFu);
                h.strand = static_cast<uint8_t>(key >> 31);
                h.n_diff = static_cast<uint8_t>((key >> 28) & 7u);
                h.n_gapo = static_cast<uint8_t>((key >> 24) & 15u);
                h.n_gape = static_cast<uint8_t>((key >> 20) & 15u);
                h.n_mm = static_cast<uint8_t>((key >> 16) & 15u);
                h.reserved = 0;
                hits[t] = h;
            }
            out.n_hits = static_cast<uint8_t>(nout);
        }
        out.flags = static_cast<uint8_t>(flags);
        *res = out;
    }
};

}  // namespace aln
