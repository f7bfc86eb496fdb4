/*
 * aln_gb300.h -- C ABI of the GB300 (sm_103a) implementation of the BWA-aln
 * inexact search over an FM-index, the hot path of BarraCUDA.
 *
 * Paper: W. B. Langdon and B. Y. H. Lam, "Genetically Improved BarraCUDA",
 * UCL RN/15/03 (arXiv:1505.07855).  Sec. 2 ("NextGen DNA Sequence Alignment")
 * states the problem these calls follow:
 *   - the reference is indexed once, offline, so that all suffixes with the same
 *     starting subsequence share one contiguous location      -> fm_index_build
 *   - the whole index must be held in GPU memory             -> fm_index_to_device
 *   - each read is looked up with a lower and an upper pointer updated per
 *     base; their distance is the number of matching positions and crossed
 *     pointers mean no match; non-exact matches back up and try alternatives
 *                                                             -> aln_search
 *   - the pairing stage needs reference positions from the index (Sec. 2 and
 *     the pipeline description in Sec. 3)                     -> sa_to_pos
 * Everything finer (D lower-bound pruning, gap and seed limits, strata, counts)
 * follows BWA's short-read method; the semantics are stated below per call.
 *
 * Conventions used by every call:
 *   base codes A=0 C=1 G=2 T=3 N=4; X = the reference after N replacement,
 *   Xr = X reversed.  For a text Y, SA and the BWT B are over Y$ ($ smallest),
 *   C[c] = number of symbols < c in Y and Occ(c, r) = number of c in B[0..r].
 *   A hit is a closed interval [k, l] of suffix-array rows.  Rows run 0..n.
 *   Forward-strand hits are intervals in SA_Xr (of the reversed target),
 *   reverse-strand hits are intervals in SA_X (of the target aligned to the
 *   reverse complement of the read).  Read indices count from the read's 5' end.
 *
 * Every call returns an int status: ALN_OK (0) or a negative ALN_E* code.  No
 * call throws or aborts.  aln_last_error() returns a message for the calling
 * thread's last failure.  Device pointers are CUDA device (or managed) memory
 * on the device the index was uploaded to; "stream" is a cudaStream_t (NULL =
 * the legacy default stream).
 */
#ifndef ALN_GB300_H
#define ALN_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
#define ALN_OK 0
#define ALN_EINVAL (-1)    /* bad argument (null pointer, size, limit out of range) */
#define ALN_ENOMEM (-2)    /* host or device allocation failed / does not fit */
#define ALN_EDEVICE (-3)   /* a CUDA call failed (message has the CUDA error) */
#define ALN_ELIMIT (-4)    /* a bounded loop reached its iteration limit */
#define ALN_EOVERFLOW (-5) /* a caller-provided buffer is too small */
#define ALN_EIO (-6)       /* file could not be read or written, or is malformed */
#define ALN_EAGAIN (-7)    /* not finished yet (aln_server_poll within its wait) */

/* ---------------------------------------------------------------- limits */
#define ALN_MAX_READ_LEN 255 /* longer reads get ALN_FLAG_READ_TOO_LONG and no hits */
#define ALN_MAX_Z 7          /* largest difference limit; larger per-read z is flagged */
#define ALN_MAX_HIT_CAP 255
#define ALN_MAX_KMER_K 12
#define ALN_CAND_CAP 512     /* distinct candidate hits kept per read by the kernels */

/* ---------------------------------------------------------------- per-read flags */
#define ALN_FLAG_HIT_OVERFLOW 0x01   /* more kept hits than hit_cap: list truncated,
                                        c0/c1 still count every kept hit */
#define ALN_FLAG_STACK_OVERFLOW 0x02 /* search stack full: result incomplete */
#define ALN_FLAG_CAND_OVERFLOW 0x04  /* more than ALN_CAND_CAP distinct candidates:
                                        result incomplete */
#define ALN_FLAG_READ_TOO_LONG 0x08  /* len > ALN_MAX_READ_LEN: not searched */
#define ALN_FLAG_BAD_LIMIT 0x10      /* per-read z > ALN_MAX_Z: not searched */
#define ALN_FLAG_WORK_LIMIT 0x20     /* per-read expansion limit reached: incomplete */
#define ALN_FLAG_LOOP_LIMIT 0x40     /* the persistent launch reached its loop bound before
                                        this read was finished: no hits, incomplete */
#define ALN_FLAG_MANY_BEST 0x80      /* score-ordered mode: more than max_best places have the
                                        best score; only the best score's hits are listed */
#define ALN_FLAG_INCOMPLETE (ALN_FLAG_STACK_OVERFLOW | ALN_FLAG_CAND_OVERFLOW | ALN_FLAG_WORK_LIMIT | \
                             ALN_FLAG_LOOP_LIMIT)

/* ---------------------------------------------------------------- per-call status bits
 * written by the kernels into aln_result.status (see aln_search) */
#define ALN_STATUS_LOOP_LIMIT 0x1u   /* a warp of the persistent launch reached params.loop_limit */

/* ---------------------------------------------------------------- modes */
#define ALN_MODE_PLAIN 0      /* one launch per batch, one thread per read */
#define ALN_MODE_PERSISTENT 1 /* one persistent launch; threads pull reads from a device queue */
#define ALN_STRATA_BEST1 0    /* keep hits with diffs <= min(z, d_best + 1) */
#define ALN_STRATA_FULL 1     /* keep every hit with diffs <= z */
#define ALN_STRATA_SCORE 2    /* score-ordered (persistent form only): every hit within z with
                                 its least witness by (score, diffs, gap opens, gap extensions,
                                 mismatches, length), score = score_mm * n_mm + score_gapo *
                                 n_gapo + score_gape * n_gape; S1 = the least score, S2 = the
                                 least score above it; hits scoring S1 or S2 listed in the
                                 order (score, strand, k, l) (S1 only, flag ALN_FLAG_MANY_BEST,
                                 when c0 > max_best > 0); c0 / c1 = summed widths at S1 / S2;
                                 d_best = fewest diffs among the S1 hits; best_score = S1 */

typedef struct fm_index fm_index;   /* host-resident index (opaque) */
typedef struct fm_dindex fm_dindex; /* device-resident index image (opaque) */

typedef struct {
    uint64_t n_seed;    /* every N of the text is indexed as splitmix64(n_seed ^ pos) & 3 */
    uint32_t sa_sample; /* keep SA[r] for rows r % sa_sample == 0; power of two 1..1024; 0 -> 32 */
    uint32_t kmer_k;    /* interval table of every string of length 1..kmer_k (a prefix
                           trie), 0 = none, <= ALN_MAX_KMER_K; result-neutral, it replaces
                           Occ steps of short targets by one table read */
    int32_t n_threads;  /* host threads for construction; 0 = all online cores */
    uint32_t reserved;
} fm_build_opts;

typedef struct {
    uint64_t n;          /* text length (without $) */
    uint64_t primary[2]; /* row of $ in B_X (0) and B_Xr (1) */
    uint64_t C[2][4];    /* C arrays of X and Xr */
    uint64_t occ_bytes;  /* bytes of Occ blocks per text: 64 per 192 rows */
    uint64_t sa_bytes;   /* bytes of sampled SA per text */
    uint64_t kmer_bytes; /* bytes of the prefix-trie interval table per text */
    uint32_t sa_sample;
    uint32_t kmer_k;
} fm_index_info_t;

/* Build the index of X and of Xr on the host (Sec. 2: offline encoding).
 * text: host, n codes 0..4 (N is replaced, anything > 3 counts as N).  n must be
 * >= 1 and < 2^32 - 1 (row numbers are 32-bit), else ALN_EINVAL.  opts may be
 * NULL (defaults).  On success *out owns the index; free it with fm_index_free. */
int fm_index_build(const uint8_t *text, uint64_t n, const fm_build_opts *opts, fm_index **out);
void fm_index_free(fm_index *idx);
int fm_index_info(const fm_index *idx, fm_index_info_t *info);

/* The same index built on a GPU (Sec. 2: offline encoding; here the encoding of a
 * human-scale reference takes seconds instead of minutes).  Arguments, defaults
 * and errors are those of fm_index_build, and the result is the same host index,
 * byte for byte (the suffix array is unique; everything else is a function of
 * it).  device: CUDA ordinal that does the work; stream: the work is enqueued on
 * it and finished before return.  The call allocates about 45 * (n + 1) bytes of
 * device memory for its duration (suffix array by prefix doubling with radix
 * sorts of (u64, u32) pairs) and frees it before return; ALN_ENOMEM if that does
 * not fit, ALN_EDEVICE on a CUDA failure. */
int fm_index_build_gpu(const uint8_t *text, uint64_t n, const fm_build_opts *opts, int device, void *stream,
                       fm_index **out);

/* Write / read the index image (little-endian binary, magic "ALNFMIX4").
 * Load returns ALN_EIO on a missing, short or malformed file. */
int fm_index_save(const fm_index *idx, const char *path);
int fm_index_load(const char *path, fm_index **out);

/* Copy the index to device memory (Sec. 2: the whole index is held in GPU
 * memory).  device: CUDA ordinal.  The copy is enqueued on stream and finished
 * before return.  The library allocates the device image (Occ blocks, sampled SA
 * and k-mer table of both texts) and a stream-ordered memory pool for the
 * search's per-call scratch; ALN_ENOMEM if it does not fit.  Free with
 * fm_dindex_free. */
int fm_index_to_device(const fm_index *idx, int device, void *stream, fm_dindex **out);
void fm_dindex_free(fm_dindex *d);
int fm_dindex_info(const fm_dindex *d, fm_index_info_t *info);

/* A batch of reads in device memory.
 *   bases : 2-bit packed bases, 16 per 32-bit word, base j of the batch in word
 *           j/16 at bits 2*(j%16) (low bits first).  An N is stored as any code
 *           and marked in nmask.
 *   nmask : 1 bit per base, 32 per word, bit j%32 of word j/32; may be NULL.
 *   offset: index of the read's first base in the batch's base stream.
 *   len   : read length in bases (0 allowed: no hits).
 *   z     : per-read difference limit; NULL = params.z for every read.
 * aln_pack_reads builds this layout on the host. */
typedef struct {
    const uint32_t *bases;
    const uint32_t *nmask;
    const uint64_t *offset;
    const uint16_t *len;
    const uint8_t *z;
} aln_batch;

typedef struct {
    uint8_t z;              /* difference limit (mismatches + gap bases) when batch.z is NULL;
                               with a per-read z array, an upper bound on it (reads above it
                               get ALN_FLAG_BAD_LIMIT); sizes the search stack */
    uint8_t max_gapo;       /* gap opens */
    uint8_t max_gape;       /* gap extensions; a gap of length g = 1 open + (g-1) extensions */
    uint8_t seed_len;       /* s: first s read bases form the seed; 0 = no seed */
    uint8_t seed_z;         /* differences allowed inside the seed */
    uint8_t indel_end_skip; /* e: no insertion at read index < e or > len-1-e; a deletion
                               only between read indices with >= max(e,1) bases each side */
    uint8_t hit_cap;        /* hits written per read, 1..ALN_MAX_HIT_CAP */
    uint8_t mode;           /* ALN_MODE_* */
    uint8_t strata;         /* ALN_STRATA_* */
    uint8_t blocks_per_sm;  /* persistent form: resident 128-thread blocks per SM; 0 = as
                               many as fit.  Fewer lanes give each lane more reads, which
                               shortens the tail where a warp waits for its slowest read */
    uint8_t smem_stack;     /* persistent form: search-stack entries per lane held in shared
                               memory (the rest in local memory): 0 = 8, else one of
                               ALN_SMEM_STACK_CHOICES; result-neutral */
    uint8_t l2_window;      /* persistent form: 1 = launch the search with an L2 access-policy
                               window over the prefix-trie tables of both texts (persisting
                               hits, streaming misses), the hottest index data: every search
                               starts in them.  The first such call on a device raises this
                               process's persisting-L2 set-aside (cudaLimitPersistingL2CacheSize,
                               a limit of the CUDA context) to the window size; 0 = off;
                               result-neutral */
    uint32_t work_limit;    /* node expansions per read before ALN_FLAG_WORK_LIMIT; 0 = 2^24 */
    uint32_t loop_limit;    /* persistent form: trips of the kernel's loop per warp before the
                               warp stops (ALN_STATUS_LOOP_LIMIT, unfinished reads flagged
                               ALN_FLAG_LOOP_LIMIT); 0 = 64 * n_reads * (576 + work_limit),
                               saturating at 2^62: a guard against a livelock, far above the
                               trips of any batch measured (a trip is one fetch per lane) */
    uint32_t help_after;    /* persistent form: once the lane searching a read has made this
                               many node expansions, lanes of its warp that finish their own
                               reads take its pending subtrees before they take new reads
                               (the lanes a heavy read gets); 0 or 0xFFFFFFFF = only once
                               the read queue is empty; result-neutral.  heavy_after counts
                               the owner's own expansions, so early help delays hand-over */
    uint32_t heavy_after;   /* persistent form with a pre-pass scratch: once the read queue is
                               empty (the batch's tail), a read whose owning lane has made more
                               than this many expansions is handed to the heavy phase, which
                               searches it with every lane of the GPU (up to 2048 reads per
                               call; later ones stay with their warp);
                               0 = ALN_HEAVY_AFTER_DEFAULT, 0xFFFFFFFF = never; result-neutral */
    uint8_t score_mm;       /* score-ordered mode: mismatch penalty; 0 = 3 (with the two below: */
    uint8_t score_gapo;     /*   gap-open penalty; 0 = 11       BWA's defaults) */
    uint8_t score_gape;     /*   gap-extension penalty; 0 = 4 */
    uint8_t max_best;       /* score-ordered mode: cap on places with the best score; 0 = none */
} aln_params;

#define ALN_SMEM_STACK_CHOICES {4, 8, 12}
#define ALN_HEAVY_AFTER_DEFAULT 65536 /* heavy_after = 0 in aln_search */
#define ALN_HEAVY_PASSES 5     /* deepening passes of the heavy phase (z <= 7): one pass and one
                                  decide kernel each, after one start kernel */

/* One hit, 16 bytes.  The witness (n_diff .. aligned_len) is the minimal one,
 * ordered by (n_diff, n_gapo, n_gape, n_mm, aligned_len), over every valid
 * transcript whose target has this interval. */
typedef struct {
    uint32_t k, l;          /* closed SA interval; width l - k + 1 positions */
    uint16_t aligned_len;   /* target length */
    uint8_t strand;         /* 0 forward (interval in SA_Xr), 1 reverse (in SA_X) */
    uint8_t n_diff;         /* n_mm + n_gapo + n_gape */
    uint8_t n_mm, n_gapo, n_gape;
    uint8_t reserved;
} aln_hit;

/* Per-read result, 12 bytes. */
typedef struct {
    uint32_t c0;            /* sum of widths of kept hits with n_diff == d_best */
    uint32_t c1;            /* sum of widths of kept hits with n_diff == d_best + 1 */
    uint8_t n_hits;         /* hits written (<= hit_cap) */
    uint8_t flags;          /* ALN_FLAG_* */
    uint8_t d_best;         /* fewest differences of any hit; 255 = no hit */
    uint8_t best_score;     /* score-ordered mode: the best score S1 (at most 254; 255 = no
                               hit); 0 in the other modes */
} aln_read_result;

typedef struct {
    aln_read_result *reads; /* device, n_reads entries */
    aln_hit *hits;          /* device, n_reads * hit_cap entries; read r at r * hit_cap */
    uint32_t *status;       /* device, 1 word, may be NULL: cleared by the call on its stream,
                               then ORed with ALN_STATUS_* bits by the kernels; read it after
                               the stream has passed the call */
    void *scratch;          /* device, may be NULL: scratch for the persistent form's D
                               pre-pass and visit order, aln_search_scratch_bytes(n_reads)
                               bytes, 256-byte aligned, owned by the call (and by every replay
                               of a graph that captured it) until it completes */
    uint64_t scratch_bytes; /* size of scratch */
} aln_result;

/* Search every read on both strands (Sec. 2: pointer-pair lookup with
 * backtracking), output per read: its hits sorted by (n_diff, strand, k, l)
 * and truncated to hit_cap, d_best, c0 and c1.
 * Result definition: a transcript aligns all of the read (forward strand) or
 * of its reverse complement (reverse strand) to a non-empty substring T of X
 * with matches, mismatches (an N always mismatches), insertions (read base not
 * in T) and deletions (T base not in the read); it is valid iff diffs <= z,
 * gap opens <= max_gapo, gap extensions <= max_gape, the end window e holds,
 * and, if seed_len > 0, the differences at read indices < seed_len (a deletion
 * counts at the read index that follows it) are <= seed_z.  Hits with equal
 * (strand, k, l) merge.  BEST1 keeps hits with diffs <= min(z, d_best + 1).
 * All arrays are device memory, written asynchronously on stream; the caller
 * synchronises.  Returns ALN_EINVAL for bad params, ALN_EDEVICE on a launch
 * failure, ALN_ELIMIT if the index has no reserved queue counter left for a
 * captured search (see below).  Per-read problems are reported in flags, never
 * by the return value.  The persistent loop is bounded (params.loop_limit): a
 * warp that reaches the bound sets ALN_STATUS_LOOP_LIMIT in *out->status, flags
 * its unfinished reads ALN_FLAG_LOOP_LIMIT and flags every read it then takes
 * from the queue the same way without searching it, so every read gets a
 * result; the binding turns the status bit into ALN_ELIMIT.
 * Persistent mode first computes every read's D array in a pre-pass and visits
 * reads in decreasing order of their lower bound; in the batch's tail (the
 * read queue empty) reads past params.heavy_after expansions of their owner
 * lane are handed to the heavy phase (at most 2048 per call), which searches
 * them from the deepening pass they were in, one pass per launch, with every
 * lane of the GPU sharing their subtrees through a task ring; it adds
 * 1 + 2 * ALN_HEAVY_PASSES launches to every persistent call with scratch
 * (they return at once when no read was handed over).  Its scratch is out->scratch
 * if given, else a block from a memory pool owned by the device index,
 * allocated and freed in stream order by the call.  While stream is being
 * captured into a graph without out->scratch (or if the pool cannot serve) the
 * search scans D itself and visits reads in input order.  The results are the
 * same either way.
 * Work-queue counters: an uncaptured persistent call takes one of 1024 counters
 * of the index in turn, so at most 1024 persistent calls on one index may be in
 * flight at once.  A call made while stream is being captured takes a counter
 * reserved for that graph for the life of the index (1024 such counters;
 * ALN_ELIMIT when they are used up); replays of one graph must not overlap each
 * other, and never share a counter with uncaptured calls. */
int aln_search(const fm_dindex *idx, const aln_batch *batch, uint32_t n_reads,
               const aln_params *params, aln_result *out, void *stream);

/* Bytes of aln_result.scratch the persistent form uses for n_reads reads:
 * 256 + 20 * n_reads for the D pre-pass and visit order, rounded up to 256,
 * plus a fixed block (about 100 MB) for the heavy phase (handed-over reads,
 * their candidate tables, the task ring).  Host only; never fails. */
uint64_t aln_search_scratch_bytes(uint32_t n_reads);

/* Autotuner for the persistent form (the scheduler's knobs: how many lanes are
 * resident and how deep each lane's shared-memory stack is).  Times aln_search
 * of a sample batch (device memory, laid out as for aln_search; scratch
 * receives its results): every resident-blocks-per-SM value from 1 to what
 * fits for every shared-memory stack depth of ALN_SMEM_STACK_CHOICES (one
 * warm-up run per depth, two timed runs per candidate, a candidate counting by
 * its slower run); writes into params the fastest blocks_per_sm and smem_stack
 * if they beat the default (every block that fits, 8 stack entries) by more
 * than 5 %, else the default (its time in *best_ms, may be NULL).  The remaining fields of params
 * are used as given: help_after and heavy_after are not tuned (a sample's
 * tail says little about a batch's, and lanes that help a read early keep its
 * owner's expansions below heavy_after, so that it never reaches the heavy
 * phase).  The choice
 * is cached per (index, sample size, sample z array, limits): a repeated call
 * returns it without timing.  Blocks on stream.  ALN_EINVAL for an empty
 * sample. */
int aln_autotune(const fm_dindex *idx, const aln_batch *sample, uint32_t n_reads, aln_params *params,
                 aln_result *scratch, void *stream, float *best_ms);

#define ALN_POS_TOO_WIDE 0xFFFFFFFFu /* n_pos_out value: hit wider than max_width */
#define ALN_POS_WALK_LIMIT 0xFFFFFFFEu /* n_pos_out value: an LF walk exceeded its bound */
#define ALN_POS_BAD_HIT 0xFFFFFFFDu  /* n_pos_out value: not a hit of this index (l < k,
                                        l > n or strand > 1); nothing of the index is read */

/* Reference positions of hits (Sec. 2/3: the pairing stage needs positions
 * from the index).  For hit i of width <= max_width, n_pos_out[i] = width and
 * pos_out[i*max_width ...] = the forward-strand 0-based starts of the target,
 * sorted ascending: strand 0 -> n - SA_Xr[j] - aligned_len, strand 1 ->
 * SA_X[j], for rows j = k..l.  Each SA value comes from the sampled SA after
 * an LF walk to the nearest sampled row (expected sa_sample steps, bounded by
 * 64 * sa_sample; a hit with a walk past the bound gets ALN_POS_WALK_LIMIT).
 * Wider hits get ALN_POS_TOO_WIDE.  A record that cannot be a hit of this index
 * (l < k, l > n or strand > 1; an unused result slot, say) gets
 * ALN_POS_BAD_HIT and is checked before any index access.  hits, pos_out and
 * n_pos_out are device memory; max_width 1..64.  Asynchronous on stream. */
int sa_to_pos(const fm_dindex *idx, const aln_hit *hits, uint32_t n_hits, uint32_t max_width,
              uint64_t *pos_out, uint32_t *n_pos_out, void *stream);

/* Dense form of a search's hits, so that what a caller copies back grows with
 * the hits found rather than with n_reads * hit_cap (Sec. 2: the number of
 * places a read matches is usually one).  Reads the search's output arrays
 * (reads: n_reads results, hits: n_reads * hit_cap slots) and writes
 *   offsets[r] = hits written for reads 0 .. r-1, r = 0 .. n_reads
 *                (offsets[n_reads] = the total),
 *   dense[offsets[r] + t] = hits[r * hit_cap + t] for t < reads[r].n_hits,
 * leaving out any hit whose place is at or past dense_cap (the caller compares
 * offsets[n_reads] with dense_cap).  All pointers are device memory; scratch:
 * aln_compact_scratch_bytes(n_reads) bytes, 4-byte aligned.  Asynchronous on
 * stream.  ALN_EINVAL for null arrays, a small scratch, hit_cap outside
 * 1..ALN_MAX_HIT_CAP or n_reads * hit_cap >= 2^32. */
uint64_t aln_compact_scratch_bytes(uint32_t n_reads);
int aln_compact_hits(const aln_read_result *reads, const aln_hit *hits, uint32_t n_reads, uint32_t hit_cap,
                     uint32_t *offsets, aln_hit *dense, uint64_t dense_cap, void *scratch, uint64_t scratch_bytes,
                     void *stream);

/* ---------------------------------------------------------------- pairing
 *
 * The pairing stage after the search (Sec. 2 and the pipeline of Sec. 3: the
 * two mates' hits are combined using the fragment length; the paper gives no
 * rule, this one is the library's).  Read 2p of a searched batch is mate 1 and
 * read 2p+1 mate 2 of pair p.
 *  - Placements of a mate: every position of every hit of its best stratum
 *    (n_diff == d_best), with the hit's strand, target length and n_diff.  A mate
 *    is placed iff it has 1 <= c0 <= max_place placements and all of them are
 *    present (every best hit written and its positions known).
 *  - A combination (one placement per mate) is FR if the strands differ; its
 *    insert is (reverse placement's start + target length) - forward placement's
 *    start.
 *  - Unique pairs: both mates have c0 == 1 and their combination is FR with
 *    1 <= insert <= ALN_PAIR_ISIZE_MAX.  Their inserts, sorted as s[0..u-1], give
 *    q1 = s[u/4], q2 = s[u/2], q3 = s[3u/4] and the window
 *    [max(1, q1 - 2 (q3 - q1)), min(ALN_PAIR_ISIZE_MAX, q3 + 2 (q3 - q1))];
 *    with u < 8 the window is [1, ALN_PAIR_ISIZE_MAX] and q1 = q2 = q3 = 0.
 *  - Proper: FR with the insert inside the window.  The pair's choice is the
 *    proper combination smallest by (n_diff1 + n_diff2, |insert - q2|, insert,
 *    pos1, pos2, strand1, len1, len2); with both mates placed and no proper
 *    combination the pair is discordant (mates from unrelated loci). */
#define ALN_PAIR_ISIZE_MAX 65535
#define ALN_PAIR_MAPPED1 0x01    /* mate 1 has a hit */
#define ALN_PAIR_MAPPED2 0x02
#define ALN_PAIR_PLACED1 0x04    /* mate 1 is placed */
#define ALN_PAIR_PLACED2 0x08
#define ALN_PAIR_UNIQUE 0x10     /* a unique pair (counted in the insert-size estimate) */
#define ALN_PAIR_PROPER 0x20     /* a proper combination exists; pos, strand, insert hold the choice */
#define ALN_PAIR_DISCORDANT 0x40 /* both mates placed, no proper combination */

typedef struct {
    uint64_t pos[2];     /* chosen placement of mate 1 / mate 2 (forward-strand start); ~0 if none */
    uint32_t insert;     /* its insert size; 0 if none */
    uint16_t n_proper;   /* proper combinations (saturating at 65535) */
    uint8_t strand[2];   /* 0 forward, 1 reverse; 255 if none */
    uint8_t flags;       /* ALN_PAIR_* */
    uint8_t reserved[7];
} aln_pair_result;       /* 32 bytes */

typedef struct {
    uint32_t n_unique, q1, q2, q3, lo, hi; /* unique pairs, insert quartiles, window */
    uint32_t reserved[2];
} aln_pair_stats;

/* Pair the mates of n_pairs pairs from a search of their 2 * n_pairs reads:
 * reads (the search's results), hit_off / hits (its hits compacted by
 * aln_compact_hits: n_reads + 1 offsets, dense hits), pos / npos (sa_to_pos of
 * those dense hits with max_width).  Writes out[n_pairs] and *stats (device).
 * max_place: 1..max_width (<= 64).  scratch: aln_pair_scratch_bytes() bytes of
 * device memory.  All pointers device memory; asynchronous on stream.
 * ALN_EINVAL for null arrays or sizes out of range. */
uint64_t aln_pair_scratch_bytes(void);
int aln_pair_resolve(const aln_read_result *reads, const uint32_t *hit_off, const aln_hit *hits,
                     const uint64_t *pos, const uint32_t *npos, uint32_t max_width, uint32_t n_pairs,
                     uint32_t max_place, aln_pair_result *out, aln_pair_stats *stats, void *scratch,
                     uint64_t scratch_bytes, void *stream);

/* ---------------------------------------------------------------- serving
 *
 * Continuous batching on a resident index.  Requests (host reads, copied at
 * submit) are queued; a dispatcher thread keeps up to n_slots batches in flight,
 * each a fixed set of device buffers with pinned staging and its own stream,
 * sized at creation and admitted only within the device-memory budget.  A free
 * slot takes reads from the oldest requests (a large request is split across
 * batches) and runs copy-in, one persistent aln_search and copy-out; requests
 * arriving while batches run join the next free slot, so batches overlap on the
 * device.  A read's result depends only on the read, the limits and the index,
 * so it is identical alone and in any mix.  Latency = completion - submit. */
typedef struct aln_server aln_server;

typedef struct {
    int32_t device;             /* CUDA ordinal of the index */
    uint32_t n_slots;           /* batches in flight, 1..16 (reduced to what the budget holds) */
    uint32_t max_batch_reads;   /* reads per batch */
    uint64_t max_batch_bases;   /* bases per batch (>= max_batch_reads) */
    uint64_t device_mem_budget; /* bytes for all slots; 0 = half of the free device memory */
    uint32_t coalesce_us;       /* with batches already running, let a partly filled batch wait
                                   this long for more requests; 0 = launch at once */
    uint32_t reserved;
    aln_params params;          /* limits (mode is forced to ALN_MODE_PERSISTENT); params.z also
                                   bounds the per-read z of requests; heavy_after 0 here means
                                   no heavy phase (it would hold every SM, stalling the other
                                   slots' batches), a nonzero value asks for it */
} aln_server_config;

typedef struct {
    uint64_t requests_done, reads_done, batches, queued_reads;
    double p50_ms, p95_ms, p99_ms; /* over every completed request since creation */
    double seconds;                /* since creation */
    uint32_t n_slots, reserved;
} aln_server_stats_t;

/* Start the dispatcher; allocates the slots.  ALN_ENOMEM if no slot fits. */
int aln_server_create(const fm_dindex *idx, const aln_server_config *cfg, aln_server **out);
/* Queue a request: reads as codes 0..4 (read r at codes[code_offset[r]], len[r]
 * bases), per-read z (NULL = params.z).  The reads are copied; the caller's
 * buffers are free on return.  *request_id identifies it for aln_server_poll. */
int aln_server_submit(aln_server *s, const uint8_t *codes, const uint64_t *code_offset, const uint16_t *len,
                      const uint8_t *z, uint32_t n_reads, uint64_t *request_id);
/* Wait up to wait_ms for a request.  On completion copies n_reads results and
 * n_reads * hit_cap hits (host memory, either may be NULL), the latency, forgets
 * the request and returns ALN_OK; ALN_EAGAIN if not finished in time. */
int aln_server_poll(aln_server *s, uint64_t request_id, int wait_ms, aln_read_result *res_out,
                    aln_hit *hits_out, double *latency_ms);
int aln_server_stats(aln_server *s, aln_server_stats_t *out);
/* Stop the dispatcher (batches in flight finish first) and free everything. */
void aln_server_destroy(aln_server *s);

/* ---------------------------------------------------------------- no-allocation variant
 *
 * The paper has no counterpart to this call; it exists for callers of this
 * library that cannot call cudaMalloc: for example a process whose device
 * memory is entirely owned by another allocator (a framework's caching
 * allocator that reserves the device up front), or a serving loop that must not
 * allocate after start-up because an allocation can block, synchronise the
 * device or fail under memory pressure.
 *
 * aln_search_noalloc runs the persistent search (params.mode is ignored) exactly
 * as aln_search does and writes the same results into the caller's buffers
 * (out->scratch and params.l2_window are not used: the search scans D in its
 * own loop and sets no access-policy window).
 * Its only scratch, the device work-queue counter, lives in a fixed array of
 * ALN_NOALLOC_SCRATCH_BYTES bytes inside the library, which every GPU that loads
 * the library holds until the process exits.  The call allocates nothing.
 *  - The first call on a device looks up the array's device address on that
 *    device (cudaGetSymbolAddress) and caches it; make that first call before
 *    any stream capture on the device.
 *  - All calls share the one array and it keeps the last call's contents; each
 *    call clears the counter on its stream before its kernel starts.  Calls that
 *    overlap on the GPU (different streams, or host threads racing) race on the
 *    counter and give wrong results: serialise them.
 *  - n_reads above ALN_NOALLOC_MAX_READS (the counter's range) is rejected with
 *    ALN_EINVAL and a message; nothing is launched.
 * Other arguments, errors and the result definition are those of aln_search. */
#define ALN_NOALLOC_SCRATCH_BYTES 256
#define ALN_NOALLOC_MAX_READS 0x80000000u
int aln_search_noalloc(const fm_dindex *idx, const aln_batch *batch, uint32_t n_reads,
                       const aln_params *params, aln_result *out, void *stream);

/* ---------------------------------------------------------------- measurement
 *
 * Random 64-byte gather rate of the device memory, the bound of the LF step's
 * access pattern (Sec. 2: each processed base reads index data at a position
 * that depends on the previous one; over a large index these are scattered
 * 64-byte blocks).  aln_gather_probe reads n_gathers 64-byte blocks of buf:
 * gather g (0 <= g < n_gathers) reads block
 *     b(g) = (h(g + seed * 0x9E3779B9) * n_blocks) >> 32    (32-bit wrap-around),
 * n_blocks = buf_bytes / 64, h = the "lowbias32" integer hash (x ^= x >> 16;
 * x *= 0x7feb352d; x ^= x >> 15; x *= 0x846ca68b; x ^= x >> 16).  Four threads
 * read the four 16-byte quarters of one block; every thread keeps 8 gathers in
 * flight; the grid fills every SM.  *sink (device memory, 4 bytes) is XORed
 * (atomically) with the XOR of all 16 words of every gathered block, so the
 * loads cannot be dropped and the result is checkable.  buf is device memory,
 * 64-byte aligned, 64 <= buf_bytes < 2^38 (n_blocks < 2^32); n_gathers < 2^32.
 * Launches on the device that holds buf, asynchronous on stream (time it with
 * events on that stream).  Errors: ALN_EINVAL (null, misaligned, size out of
 * range, not device memory), ALN_EDEVICE (launch). */
int aln_gather_probe(const void *buf, uint64_t buf_bytes, uint64_t n_gathers, uint32_t seed,
                     uint32_t *sink, void *stream);

/* Host helper: pack reads (codes 0..4, read r at codes[code_offset[r]] of
 * length len[r]) back to back into the aln_batch layout.  bases_out needs
 * ceil(total/16) words, nmask_out ceil(total/32) words (total = sum of len),
 * offset_out n_reads entries.  Host memory only. */
int aln_pack_reads(const uint8_t *codes, const uint64_t *code_offset, const uint16_t *len,
                   uint32_t n_reads, uint32_t *bases_out, uint32_t *nmask_out,
                   uint64_t *offset_out);

/* Message describing the calling thread's most recent failure ("" if none). */
const char *aln_last_error(void);
/* Library ABI version (major * 100 + minor). */
int aln_version(void);

#ifdef __cplusplus
}
#endif
#endif /* ALN_GB300_H */
