// Host construction of the FM-index of X and of X reversed (paper Sec. 2: the
// reference is encoded offline so that all suffixes with the same starting
// subsequence share one contiguous location, and extending the prefix by one
// base maps a location to a sub-location).
//
// Suffix array: prefix doubling (Manber and Myers 1993, refined per group as in
// Larsson and Sadakane 2007).  Suffixes are first radix-sorted by their first 21
// symbols (3 bits each, $ = 0), then every group of equal h-prefixes is re-sorted
// by the rank of the suffix h positions later, h doubling each round, until all
// groups are singletons.  Groups are processed in parallel.
//
// Occ layout: 64-byte blocks of 192 rows, [cnt_A cnt_C cnt_G cnt_T | 12 words of
// 2-bit symbols].  The counts are taken at the block's middle row (192 b + 96),
// with $ counted as A, so a query counts at most 96 symbols (6 words) forwards
// or backwards from there; the $ row is stored as A and a query subtracts one
// from Occ(A) past the primary row.  One LF step reads one 64-byte block per row.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <new>
#include <thread>

#include "aln_internal.h"

namespace aln {

static thread_local std::string g_error;

void set_error(const std::string &msg) { g_error = msg; }

int fail(int status, const std::string &msg) {
    g_error = msg;
    return status;
}

static int resolve_threads(int t) {
    if (t > 0) return t;
    unsigned h = std::thread::hardware_concurrency();
    return h ? static_cast<int>(h) : 1;
}

template <class F>
static void parallel_chunks(int threads, uint64_t n, F &&fn) {
    if (threads <= 1 || n < 65536) {
        fn(0, uint64_t(0), n);
        return;
    }
    std::vector<std::thread> th;
    th.reserve(threads);
    for (int t = 0; t < threads; t++) {
        uint64_t b = n * t / threads, e = n * (t + 1) / threads;
        th.emplace_back([&, t, b, e] { fn(t, b, e); });
    }
    for (auto &x : th) x.join();
}

// LSD radix sort of (key, val) pairs by the 64-bit key, 16-bit digits.
static void radix_sort_pairs(std::vector<uint64_t> &key, std::vector<uint32_t> &val, int threads) {
    const uint64_t n = key.size();
    std::vector<uint64_t> k2(n);
    std::vector<uint32_t> v2(n);
    const int T = (n < 65536) ? 1 : threads;
    std::vector<uint64_t> hist(static_cast<size_t>(T) * 65536);
    for (int pass = 0; pass < 4; pass++) {
        const int shift = 16 * pass;
        std::fill(hist.begin(), hist.end(), 0);
        parallel_chunks(T, n, [&](int t, uint64_t b, uint64_t e) {
            uint64_t *h = &hist[static_cast<size_t>(t) * 65536];
            for (uint64_t i = b; i < e; i++) h[(key[i] >> shift) & 0xFFFF]++;
        });
        // skip a pass where every key has the same digit
        bool trivial = false;
        for (uint32_t d = 0; d < 65536; d++) {
            uint64_t s = 0;
            for (int t = 0; t < T; t++) s += hist[static_cast<size_t>(t) * 65536 + d];
            if (s == n) trivial = true;
            if (s) break;
        }
        if (trivial) continue;
        uint64_t run = 0;
        for (uint32_t d = 0; d < 65536; d++)
            for (int t = 0; t < T; t++) {
                uint64_t &h = hist[static_cast<size_t>(t) * 65536 + d];
                uint64_t c = h;
                h = run;
                run += c;
            }
        parallel_chunks(T, n, [&](int t, uint64_t b, uint64_t e) {
            uint64_t *h = &hist[static_cast<size_t>(t) * 65536];
            for (uint64_t i = b; i < e; i++) {
                uint64_t o = h[(key[i] >> shift) & 0xFFFF]++;
                k2[o] = key[i];
                v2[o] = val[i];
            }
        });
        key.swap(k2);
        val.swap(v2);
    }
}

void build_suffix_array(const uint8_t *x, uint64_t n, uint32_t *sa, int threads) {
    threads = resolve_threads(threads);
    const uint64_t N = n + 1;  // suffixes 0..n, suffix n is "$"
    constexpr int K0 = 21;
    std::vector<uint64_t> key(N);
    std::vector<uint32_t> val(N);
    // key = 21 symbols, 3 bits each, real symbol c -> c+1, past the end -> 0
    parallel_chunks(threads, N, [&](int, uint64_t b, uint64_t e) {
        for (uint64_t i = b; i < e; i++) {
            uint64_t k = 0;
            for (int t = 0; t < K0; t++) {
                uint64_t p = i + t;
                uint64_t s = p < n ? uint64_t(x[p]) + 1 : 0;
                k = (k << 3) | s;
            }
            key[i] = k;
            val[i] = static_cast<uint32_t>(i);
        }
    });
    radix_sort_pairs(key, val, threads);
    std::vector<uint32_t> rank(N);
    // head rank: index of the first row of the suffix's group
    {
        uint64_t hd = 0;
        for (uint64_t j = 0; j < N; j++) {
            if (j > 0 && key[j] != key[j - 1]) hd = j;
            rank[val[j]] = static_cast<uint32_t>(hd);
        }
    }
    // unsorted groups: runs of equal keys of length >= 2
    std::vector<std::pair<uint64_t, uint64_t>> groups;
    for (uint64_t j = 0; j < N;) {
        uint64_t e = j + 1;
        while (e < N && key[e] == key[j]) e++;
        if (e - j > 1) groups.emplace_back(j, e);
        j = e;
    }
    std::vector<uint64_t>().swap(key);
    std::vector<uint32_t> key2(N);
    uint64_t h = K0;
    while (!groups.empty()) {
        const uint64_t G = groups.size();
        std::atomic<uint64_t> next(0);
        std::vector<std::vector<std::pair<uint64_t, uint64_t>>> new_groups(threads);
        auto sort_phase = [&](int t) {
            std::vector<std::pair<uint32_t, uint32_t>> buf;
            for (;;) {
                uint64_t g0 = next.fetch_add(64);
                if (g0 >= G) break;
                uint64_t g1 = std::min(G, g0 + 64);
                for (uint64_t g = g0; g < g1; g++) {
                    uint64_t a = groups[g].first, b = groups[g].second;
                    buf.resize(b - a);
                    for (uint64_t j = a; j < b; j++) {
                        // every member shares an h-prefix of real symbols, so
                        // SA + h <= n; rank[n] = 0 for the "$" suffix
                        buf[j - a] = {rank[val[j] + h], val[j]};
                    }
                    std::sort(buf.begin(), buf.end());
                    for (uint64_t j = a; j < b; j++) {
                        key2[j] = buf[j - a].first;
                        val[j] = buf[j - a].second;
                    }
                    for (uint64_t j = a; j < b;) {
                        uint64_t e = j + 1;
                        while (e < b && key2[e] == key2[j]) e++;
                        if (e - j > 1) new_groups[t].emplace_back(j, e);
                        j = e;
                    }
                }
            }
        };
        {
            std::vector<std::thread> th;
            for (int t = 0; t < threads; t++) th.emplace_back(sort_phase, t);
            for (auto &x : th) x.join();
        }
        // rank update after every group has read the old ranks
        next = 0;
        auto rank_phase = [&]() {
            for (;;) {
                uint64_t g0 = next.fetch_add(64);
                if (g0 >= G) break;
                uint64_t g1 = std::min(G, g0 + 64);
                for (uint64_t g = g0; g < g1; g++) {
                    uint64_t a = groups[g].first, b = groups[g].second;
                    uint64_t hd = a;
                    for (uint64_t j = a; j < b; j++) {
                        if (j > a && key2[j] != key2[j - 1]) hd = j;
                        rank[val[j]] = static_cast<uint32_t>(hd);
                    }
                }
            }
        };
        {
            std::vector<std::thread> th;
            for (int t = 0; t < threads; t++) th.emplace_back(rank_phase);
            for (auto &x : th) x.join();
        }
        groups.clear();
        for (auto &v : new_groups) groups.insert(groups.end(), v.begin(), v.end());
        std::sort(groups.begin(), groups.end());
        h *= 2;
    }
    std::memcpy(sa, val.data(), N * sizeof(uint32_t));
}

// SplitMix64 output function (Steele, Lea and Flood 2014) on state z + golden.
static inline uint64_t splitmix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static void pack_text(HostText &T, const uint8_t *y, uint64_t n, const uint32_t *sa,
                      uint32_t sa_sample, int threads) {
    T.n = n;
    const uint64_t rows = n + 1;
    const uint64_t nb = rows / kBlockRows + 1;  // one more block for row n+1 queries
    T.blocks.assign(nb * kBlockWords, 0);
    std::vector<uint32_t> bcount(nb * 4, 0);
    uint64_t cnt[4] = {0, 0, 0, 0};
    for (uint64_t i = 0; i < n; i++) cnt[y[i]]++;
    T.C[0] = 0;
    for (int c = 1; c < 4; c++) T.C[c] = T.C[c - 1] + cnt[c - 1];
    for (uint64_t r = 0; r < rows; r++)
        if (sa[r] == 0) T.primary = r;
    std::vector<uint32_t> hcount(nb * 4, 0);  // per block: symbols of its first half
    parallel_chunks(threads, nb, [&](int, uint64_t b0, uint64_t b1) {
        for (uint64_t b = b0; b < b1; b++) {
            uint32_t *w = &T.blocks[b * kBlockWords + 4];
            uint32_t c4[4] = {0, 0, 0, 0}, h4[4] = {0, 0, 0, 0};
            for (uint32_t t = 0; t < kBlockRows; t++) {
                uint64_t r = b * kBlockRows + t;
                if (r >= rows) break;
                uint32_t s = sa[r];
                uint32_t sym = s == 0 ? 0u : y[s - 1];  // $ stored as A
                // bit planes per half: words 0-2 low bits, 3-5 high bits of
                // the half's symbols 0-31, 32-63, 64-95
                const uint32_t half = t / (kBlockRows / 2), u = t % (kBlockRows / 2);
                w[6 * half + u / 32] |= (sym & 1u) << (u % 32);
                w[6 * half + 3 + u / 32] |= (sym >> 1) << (u % 32);
                c4[sym]++;
                if (t < kBlockRows / 2) h4[sym]++;
            }
            for (int c = 0; c < 4; c++) {
                bcount[b * 4 + c] = c4[c];
                hcount[b * 4 + c] = h4[c];
            }
        }
    });
    // counts before the middle row: prefix over earlier blocks + the block's first
    // half.  Padding past the last row is stored as A and counted here too, so a
    // backward count from the middle of the last block stays exact.
    uint32_t run[4] = {0, 0, 0, 0};
    for (uint64_t b = 0; b < nb; b++) {
        // padding rows of the first half (stored as A)
        const uint64_t mid = b * kBlockRows + kBlockRows / 2;
        const uint32_t pad = mid > rows ? static_cast<uint32_t>(std::min<uint64_t>(kBlockRows / 2, mid - rows)) : 0u;
        for (int c = 0; c < 4; c++) {
            T.blocks[b * kBlockWords + c] = run[c] + hcount[b * 4 + c] + (c == 0 ? pad : 0u);
            run[c] += bcount[b * 4 + c];
        }
    }
    const uint64_t ns = n / sa_sample + 1;
    T.sa_samp.resize(ns);
    for (uint64_t t = 0; t < ns; t++) T.sa_samp[t] = sa[t * sa_sample];
}

// Interval table of every string of length 1..k (a prefix trie of the index).
// A search extends its target one base at a time, so a node's interval is a
// function of its target string alone; indexing strings in the order the search
// processes them (first processed base in the top bits) puts the four children
// of a string s at 4 s + c, contiguous, one level down.  Level j (1..k) starts at
// entry (4^j - 4) / 3 and holds 4^j half-open (lo, hi) pairs; absent strings get
// (0, 0).  Rows sharing a j-prefix are contiguous in the SA, so one scan over
// the SA fills every level: for the suffix at s, the string processed as
// q[0..j-1] is y[s+j-1] .. y[s] and its index is sum_u y[s+u] 4^u.
static void build_kmer(HostText &T, const uint8_t *y, uint64_t n, const uint32_t *sa, uint32_t k,
                       int threads) {
    const uint64_t total = ((1ULL << (2 * (k + 1))) - 4) / 3;
    T.kmer.assign(2 * total, 0);
    const uint64_t rows = n + 1;
    for (uint32_t j = 1; j <= k; j++) {
        const uint64_t off = ((1ULL << (2 * j)) - 4) / 3;
        auto id_of = [&](uint64_t r) -> int64_t {
            uint64_t s = sa[r];
            if (s + j > n) return -1;
            uint64_t id = 0;
            for (uint32_t u = 0; u < j; u++) id |= uint64_t(y[s + u]) << (2 * u);
            return static_cast<int64_t>(id);
        };
        parallel_chunks(threads, rows, [&](int, uint64_t b, uint64_t e) {
            int64_t prev = b > 0 ? id_of(b - 1) : -2;
            int64_t cur = id_of(b);
            for (uint64_t r = b; r < e; r++) {
                int64_t nxt = r + 1 < rows ? id_of(r + 1) : -2;
                if (cur >= 0) {
                    if (cur != prev) T.kmer[2 * (off + cur)] = static_cast<uint32_t>(r);
                    if (cur != nxt) T.kmer[2 * (off + cur) + 1] = static_cast<uint32_t>(r + 1);
                }
                prev = cur;
                cur = nxt;
            }
        });
    }
}

}  // namespace aln

using namespace aln;

extern "C" int fm_index_build(const uint8_t *text, uint64_t n, const fm_build_opts *opts,
                              fm_index **out) {
    if (!text || !out) return fail(ALN_EINVAL, "fm_index_build: null argument");
    *out = nullptr;
    if (n < 1 || n >= 0xFFFFFFFFULL) return fail(ALN_EINVAL, "fm_index_build: n must be in [1, 2^32-2]");
    fm_build_opts o{};
    if (opts) o = *opts;
    if (o.sa_sample == 0) o.sa_sample = 32;
    if (o.sa_sample > 1024 || (o.sa_sample & (o.sa_sample - 1)))
        return fail(ALN_EINVAL, "fm_index_build: sa_sample must be a power of two <= 1024");
    if (o.kmer_k > ALN_MAX_KMER_K) return fail(ALN_EINVAL, "fm_index_build: kmer_k too large");
    const int threads = resolve_threads(o.n_threads);
    try {
        fm_index *ix = new fm_index();
        ix->sa_sample = o.sa_sample;
        ix->kmer_k = o.kmer_k;
        ix->n_seed = o.n_seed;
        std::vector<uint8_t> x(n), xr(n);
        for (uint64_t i = 0; i < n; i++)
            x[i] = text[i] < 4 ? text[i] : static_cast<uint8_t>(splitmix64(o.n_seed ^ i) & 3);
        for (uint64_t i = 0; i < n; i++) xr[i] = x[n - 1 - i];
        std::vector<uint32_t> sa(n + 1);
        for (int w = 0; w < 2; w++) {
            const uint8_t *y = w ? xr.data() : x.data();
            build_suffix_array(y, n, sa.data(), threads);
            pack_text(ix->t[w], y, n, sa.data(), o.sa_sample, threads);
            if (o.kmer_k) build_kmer(ix->t[w], y, n, sa.data(), o.kmer_k, threads);
        }
        *out = ix;
        return ALN_OK;
    } catch (const std::bad_alloc &) {
        return fail(ALN_ENOMEM, "fm_index_build: host allocation failed");
    } catch (const std::exception &e) {
        return fail(ALN_EINVAL, std::string("fm_index_build: ") + e.what());
    }
}

extern "C" void fm_index_free(fm_index *idx) { delete idx; }

extern "C" int fm_index_info(const fm_index *idx, fm_index_info_t *info) {
    if (!idx || !info) return fail(ALN_EINVAL, "fm_index_info: null argument");
    std::memset(info, 0, sizeof *info);
    info->n = idx->t[0].n;
    for (int w = 0; w < 2; w++) {
        info->primary[w] = idx->t[w].primary;
        for (int c = 0; c < 4; c++) info->C[w][c] = idx->t[w].C[c];
    }
    info->occ_bytes = idx->t[0].blocks.size() * 4;
    info->sa_bytes = idx->t[0].sa_samp.size() * 4;
    info->kmer_bytes = idx->t[0].kmer.size() * 4;
    info->sa_sample = idx->sa_sample;
    info->kmer_k = idx->kmer_k;
    return ALN_OK;
}

static uint64_t kmer_words(uint32_t k) { return k ? 2 * (((1ULL << (2 * (k + 1))) - 4) / 3) : 0; }

static const char kMagic[8] = {'A', 'L', 'N', 'F', 'M', 'I', 'X', '4'};

template <class V>
static bool write_vec(std::ofstream &f, const V &v) {
    uint64_t sz = v.size();
    f.write(reinterpret_cast<const char *>(&sz), 8);
    f.write(reinterpret_cast<const char *>(v.data()), sz * sizeof(v[0]));
    return bool(f);
}

template <class V>
static bool read_vec(std::ifstream &f, V &v, uint64_t max_elems) {
    uint64_t sz = 0;
    f.read(reinterpret_cast<char *>(&sz), 8);
    if (!f || sz > max_elems) return false;
    v.resize(sz);
    f.read(reinterpret_cast<char *>(v.data()), sz * sizeof(v[0]));
    return bool(f);
}

extern "C" int fm_index_save(const fm_index *idx, const char *path) {
    if (!idx || !path) return fail(ALN_EINVAL, "fm_index_save: null argument");
    std::ofstream f(path, std::ios::binary | std::ios::trunc);
    if (!f) return fail(ALN_EIO, std::string("fm_index_save: cannot open ") + path);
    f.write(kMagic, 8);
    uint64_t hdr[3] = {idx->sa_sample, idx->kmer_k, idx->n_seed};
    f.write(reinterpret_cast<const char *>(hdr), sizeof hdr);
    for (int w = 0; w < 2; w++) {
        const HostText &T = idx->t[w];
        uint64_t h2[6] = {T.n, T.primary, T.C[0], T.C[1], T.C[2], T.C[3]};
        f.write(reinterpret_cast<const char *>(h2), sizeof h2);
        write_vec(f, T.blocks);
        write_vec(f, T.sa_samp);
        write_vec(f, T.kmer);
    }
    if (!f) return fail(ALN_EIO, "fm_index_save: write failed");
    return ALN_OK;
}

extern "C" int fm_index_load(const char *path, fm_index **out) {
    if (!path || !out) return fail(ALN_EINVAL, "fm_index_load: null argument");
    *out = nullptr;
    std::ifstream f(path, std::ios::binary);
    if (!f) return fail(ALN_EIO, std::string("fm_index_load: cannot open ") + path);
    char magic[8];
    f.read(magic, 8);
    if (!f || std::memcmp(magic, kMagic, 8)) return fail(ALN_EIO, "fm_index_load: bad magic");
    try {
        fm_index *ix = new fm_index();
        uint64_t hdr[3];
        f.read(reinterpret_cast<char *>(hdr), sizeof hdr);
        ix->sa_sample = static_cast<uint32_t>(hdr[0]);
        ix->kmer_k = static_cast<uint32_t>(hdr[1]);
        ix->n_seed = hdr[2];
        bool ok = bool(f) && ix->kmer_k <= ALN_MAX_KMER_K && ix->sa_sample >= 1 && ix->sa_sample <= 1024;
        for (int w = 0; w < 2 && ok; w++) {
            HostText &T = ix->t[w];
            uint64_t h2[6];
            f.read(reinterpret_cast<char *>(h2), sizeof h2);
            ok = bool(f) && h2[0] >= 1 && h2[0] < 0xFFFFFFFFULL;
            if (!ok) break;
            T.n = h2[0];
            T.primary = h2[1];
            for (int c = 0; c < 4; c++) T.C[c] = h2[2 + c];
            const uint64_t nb = (T.n + 1) / kBlockRows + 1;
            ok = read_vec(f, T.blocks, nb * kBlockWords) && T.blocks.size() == nb * kBlockWords &&
                 read_vec(f, T.sa_samp, T.n + 1) && T.sa_samp.size() == T.n / ix->sa_sample + 1 &&
                 read_vec(f, T.kmer, kmer_words(ix->kmer_k)) && T.kmer.size() == kmer_words(ix->kmer_k) &&
                 T.primary <= T.n;
        }
        if (!ok || ix->t[0].n != ix->t[1].n) {
            delete ix;
            return fail(ALN_EIO, "fm_index_load: truncated or malformed file");
        }
        *out = ix;
        return ALN_OK;
    } catch (const std::bad_alloc &) {
        return fail(ALN_ENOMEM, "fm_index_load: host allocation failed");
    }
}

extern "C" int aln_pack_reads(const uint8_t *codes, const uint64_t *code_offset, const uint16_t *len,
                              uint32_t n_reads, uint32_t *bases_out, uint32_t *nmask_out,
                              uint64_t *offset_out) {
    if (n_reads && (!codes || !code_offset || !len || !bases_out || !nmask_out || !offset_out))
        return fail(ALN_EINVAL, "aln_pack_reads: null argument");
    uint64_t total = 0;
    for (uint32_t r = 0; r < n_reads; r++) total += len[r];
    std::memset(bases_out, 0, ((total + 15) / 16) * 4);
    std::memset(nmask_out, 0, ((total + 31) / 32) * 4);
    uint64_t j = 0;
    for (uint32_t r = 0; r < n_reads; r++) {
        offset_out[r] = j;
        const uint8_t *c = codes + code_offset[r];
        for (uint32_t t = 0; t < len[r]; t++, j++) {
            uint32_t b = c[t];
            if (b > 3) {
                nmask_out[j / 32] |= 1u << (j % 32);
                b = 0;
            }
            bases_out[j / 16] |= b << (2 * (j % 16));
        }
    }
    return ALN_OK;
}

extern "C" const char *aln_last_error(void) { return aln::g_error.c_str(); }

extern "C" int aln_version(void) { return 200; }  // 2.00: loop bound and status word, caller scratch, shared-memory stack choice
