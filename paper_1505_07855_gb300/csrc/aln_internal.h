// Internal declarations shared by the host index builder and the CUDA side of
// the library.  Not part of the public ABI (see include/aln_gb300.h).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "aln_gb300.h"

namespace aln {

// Rows per Occ block: one 64-byte block holds the Occ counts of A, C, G, T
// before its first row (4 x u32) and 192 BWT symbols at 2 bits (12 x u32).
constexpr uint32_t kBlockRows = 192;
constexpr uint32_t kBlockWords = 16;

struct HostText {
    uint64_t n = 0;        // text length, rows are 0..n
    uint64_t primary = 0;  // row of $ (stored as A in the packed symbols)
    uint64_t C[4] = {0, 0, 0, 0};
    std::vector<uint32_t> blocks;    // n_blocks * 16 words
    std::vector<uint32_t> sa_samp;   // SA[r] for r % sa_sample == 0
    std::vector<uint32_t> kmer;      // 2 * 4^k words: (lo, hi) half-open interval per k-mer
    uint64_t n_blocks() const { return blocks.size() / kBlockWords; }
};

}  // namespace aln

struct fm_index {
    aln::HostText t[2];   // t[0] = X, t[1] = X reversed
    uint32_t sa_sample = 32;
    uint32_t kmer_k = 0;
    uint64_t n_seed = 0;
};

namespace aln {
void set_error(const std::string &msg);
int fail(int status, const std::string &msg);
// Suffix array of text$ (codes 0..3, length n) by prefix doubling; sa has n+1 entries.
void build_suffix_array(const uint8_t *text, uint64_t n, uint32_t *sa, int threads);
}  // namespace aln
