/*
 * sss.h -- C ABI of the GB300 string sample sort library (libsss.so).
 *
 * What it computes (paper Sec. 2, "Preliminaries"): given n zero-terminated
 * byte strings, the permutation that sorts them in lexicographic order of
 * unsigned bytes (a proper prefix sorts first, since the terminator 0 is
 * below every character) and the LCP array lcp[r] = lcp(s_perm[r-1],
 * s_perm[r]).  Equal strings are ordered by ascending original index, which
 * makes the answer unique.  The method is super scalar string sample sort
 * (S^5, Sec. 3.1): repeated distribution rounds over 8-byte big-endian key
 * words with a sampled splitter tree and equality buckets, recursion on the
 * buckets with the common prefix depth raised per Eq. (1), and a base case
 * for small buckets.
 *
 * Conventions for every entry point:
 *   - Pointers marked "device" must point to GPU memory of the current
 *     device; "host" pointers to CPU memory.  The caller owns every buffer it
 *     passes; the library never frees them.
 *   - chars holds the string bytes; string i starts at chars[offsets[i]] and
 *     ends at its first 0 byte, which must exist inside the buffer.  The
 *     library reads the bytes of each string up to and including its
 *     terminator and, besides those, only bytes of the aligned 8-byte words
 *     that contain them, so it never touches a memory page the strings do
 *     not reach.  Strings must be shorter than 2^31 bytes.
 *   - n is limited to 2^32 - 1 strings (indices are uint32).
 *   - out_perm[r] (uint32, device) is the original index of the r-th
 *     smallest string; out_lcp[r] (uint32, device) its LCP in bytes with the
 *     previous one (terminator not counted), out_lcp[0] = 0.
 *   - stream is a cudaStream_t (NULL = the legacy default stream).  Work is
 *     enqueued on it; the calls that run distribution rounds also wait on it
 *     once per round to read the next round's sizes (a few bytes).
 *   - Every call returns an sss_status; errors are never thrown across the
 *     ABI.  sss_last_error() describes the most recent failure.
 *   - The library keeps global options, statistics and a workspace cache:
 *     calls are serialised by an internal mutex.
 */
#ifndef SSS_H
#define SSS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SSS_OK = 0,
    SSS_ERR_INVALID = -1,   /* bad argument (null pointer, bad option, ...) */
    SSS_ERR_NOMEM = -2,     /* device or host allocation failed / workspace too small */
    SSS_ERR_CUDA = -3,      /* a CUDA call failed; see sss_last_error() */
    SSS_ERR_TIMEOUT = -4,   /* a bounded device wait gave up */
    SSS_ERR_TOO_LARGE = -5, /* size beyond a documented limit */
    SSS_ERR_INTERNAL = -6   /* a device-side consistency check failed */
} sss_status;

/* Tuning knobs.  Defaults: k_max 10, base_threshold 128, medium_threshold
 * 8192, chunk 32768, seed 0x5eed, cdf_segments 4096, cdf_steps 4,
 * cdf_lr 0.005, profile 0, graph 0, key_bytes 16, classifier 0, alphabet 0,
 * radix 0. */
typedef struct sss_options {
    int32_t k_max;             /* largest splitter tree depth k: v = 2^k - 1 splitters, 1..10 */
    uint32_t base_threshold;   /* buckets of at most this many strings go to the base case, 16..128 */
    uint32_t medium_threshold; /* buckets of at most this many strings get one CTA (one warp
                                  up to 1023 strings) for their next round,
                                  base_threshold..8192 */
    uint32_t chunk;            /* largest work item (strings) of a device-wide round,
                                  multiple of 2048 */
    uint64_t seed;           /* seed of the pseudo-random sample positions */
    uint32_t cdf_segments;   /* learned CDF: number of linear pieces, 16..4096 (power of two) */
    uint32_t cdf_steps;      /* learned CDF: Adam steps per fit after a start through the
                                sample's per-piece mean points; 0 = the untrained
                                uniform model */
    float cdf_lr;            /* learned CDF: Adam step size */
    uint32_t profile;        /* 1: time every kernel launch with CUDA events on the
                                caller's stream and report per-class totals in
                                sss_stats (adds one event pair per launch; host-
                                driven rounds only) */
    uint32_t graph;          /* 1: run sss_sort / sss_sort_learned as one CUDA graph
                                whose round loop is a device-side conditional node
                                (no host round-trip per round; per-round stats not
                                recorded).  sss_sort_batched always does, unless
                                profile = 1 asks for timed host-driven rounds. */
    uint32_t key_bytes;      /* w, characters per classification key: 8 (one 64-bit
                                key word, as in Sec. 3.1) or 16 (two words compared
                                as one 128-bit key: a round steps over up to 16
                                shared characters).  The learned proposal always
                                uses 8.  The output does not depend on it. */
    uint32_t classifier;     /* 0: pS^5-Unroll, equality test against the in-order
                                splitter after the full descent; 1: pS^5-Equal,
                                equality test at every node with early exit (both
                                Sec. 3.1).  The learned proposal always uses 0.  The
                                output does not depend on it. */
    uint32_t alphabet;       /* 1: alphabet compression (App. A.2, "Practical Refinements"):
                                when only sigma' <= 15 distinct characters occur, each
                                string is first rewritten with g = floor(log_{sigma'+1}
                                256) characters per byte, as base-(sigma'+1) digits in
                                rank order (the terminator is digit 0), the rewritten
                                strings are sorted, and the LCP array is converted back
                                to characters.  DNA (sigma' = 4) gets g = 3.  Uses
                                library-managed memory: sss_sort_ws and
                                sss_sort_noalloc ignore it.  0: off.  The output does
                                not depend on it. */
    uint32_t radix;          /* classification of a device-wide round's segment by a
                                digit instead of the splitter tree (App. A.2,
                                adaptivity): the digit is the k_max bits of the key
                                after the bits every sample key shares.  0: trees
                                only; 1: a segment whose sample digits (at least
                                4 bits) have an entropy of at least k - 1 bits
                                (near uniform) is classified by its digit; 2:
                                every segment whose
                                sample keys differ.  The learned proposal always
                                uses trees.  The output does not depend on it. */
} sss_options;

#define SSS_MAX_ROUNDS_LOGGED 64

/* Kernel classes reported by the profile counters of sss_stats. */
enum {
    SSS_K_INIT = 0,     /* key gather at depth 0, roots, header reset */
    SSS_K_SAMPLE = 1,   /* sample sort + splitter tree per segment */
    SSS_K_CLASSIFY = 2, /* tree descent + bucket histogram */
    SSS_K_SCAN = 3,     /* prefix sums */
    SSS_K_SCATTER = 4,  /* stable redistribution + key refill + child segments */
    SSS_K_PLAN = 5,     /* next round layout */
    SSS_K_BASE = 6,     /* small-bucket sort with LCP */
    SSS_K_RUNS = 7,     /* large runs of equal strings */
    SSS_K_FIXUP = 8,    /* LCP at bucket boundaries, batched index rebasing */
    SSS_K_LEARNED = 9,  /* learned CDF fit and proposal */
    SSS_K_MEDIUM = 10,  /* one CTA (or warp) per medium bucket: a whole round in shared memory */
    SSS_K_ALPHABET = 11, /* alphabet compression: character scan, packing, LCP conversion */
    SSS_K_CLASSES = 12
};

/* Statistics of the last successful sort call. */
typedef struct sss_stats {
    uint32_t rounds;                 /* distribution rounds run */
    uint32_t base_tiles;             /* base-case work tiles launched */
    uint64_t round_strings;          /* sum over rounds of strings distributed */
    uint64_t medium_strings;         /* of those, strings in per-CTA or per-warp (medium) rounds */
    uint64_t base_iterations;        /* base-case sort passes summed over tiles and warp packs */
    uint32_t base_segment_hist[8];   /* base-case buckets by floor(log2(size)) (2-3, 4-7, ..., >= 128) */
    uint64_t base_strings;           /* strings finished by the base case */
    uint64_t run_strings;            /* strings finished as large runs of equal strings */
    uint64_t learned_keys;           /* keys the learned model proposed a bucket for */
    uint64_t learned_misses;         /* of those, proposals the exact check rejected */
    uint64_t refilled_strings;       /* key words gathered again from chars during rounds */
    uint64_t medium_refilled_strings; /* of those, gathered in medium rounds */
    uint32_t launches;               /* kernel launches of the call */
    uint32_t profiled;               /* 1 if the prof_* fields below were measured */
    uint32_t prof_launches[SSS_K_CLASSES]; /* launches per kernel class */
    double prof_ms[SSS_K_CLASSES];   /* summed device time per kernel class (ms) */
    uint32_t round_segments[SSS_MAX_ROUNDS_LOGGED]; /* large + medium segments per round */
    uint32_t round_active[SSS_MAX_ROUNDS_LOGGED];   /* strings distributed per round */
    uint32_t alphabet_symbols;       /* sigma': distinct non-terminator characters seen
                                        (alphabet option on), else 0 */
    uint32_t alphabet_group;         /* characters packed per byte: g >= 2 when the strings
                                        were rewritten, 1 when the alphabet was too large,
                                        0 when the option is off */
    uint32_t learned_models;         /* learned CDF models fitted (one per segment of a
                                        device-wide round that got one) */
    uint32_t radix_segments;         /* segments of device-wide rounds classified by a
                                        digit instead of a splitter tree (option radix) */
    uint64_t round_learned_keys[SSS_MAX_ROUNDS_LOGGED];   /* learned proposals per round
                                                             (host-driven rounds only) */
    uint64_t round_learned_misses[SSS_MAX_ROUNDS_LOGGED]; /* of those, rejected ones */
} sss_stats;

/* What the learned proposal did in the last sss_sort_learned call. */
typedef struct sss_learned_stats {
    uint64_t proposals;  /* keys the model proposed a bucket for */
    uint64_t misses;     /* proposals the exact splitter check rejected (the tree decided) */
    uint32_t models;     /* segment models fitted */
    uint32_t pad;
    double miss_rate;    /* misses / proposals, 0 without proposals */
} sss_learned_stats;

/* ---------------------------------------------------------------- sort */

/* Sort n strings (all pointers device).  Scratch memory comes from a
 * per-device cache grown with cudaMalloc on demand (see sss_release).
 * n = 0 is a no-op; n = 1 writes perm 0, lcp 0. */
int sss_sort(const uint8_t* chars, const uint64_t* offsets, uint32_t n,
             uint32_t* out_perm, uint32_t* out_lcp, void* stream);

/* Bytes of scratch sss_sort_ws needs for n strings under the current options. */
size_t sss_workspace_size(uint32_t n);

/* As sss_sort, with caller-provided scratch: workspace (device, 256-byte
 * aligned, at least sss_workspace_size(n) bytes; contents need not be
 * initialised and are clobbered).  Returns SSS_ERR_NOMEM if it is too small. */
int sss_sort_ws(const uint8_t* chars, const uint64_t* offsets, uint32_t n,
                uint32_t* out_perm, uint32_t* out_lcp,
                void* workspace, size_t workspace_bytes, void* stream);

/* Allocation-free variant of sss_sort, for at most 65,536 strings.  The
 * paper has no counterpart: it exists for callers that cannot call
 * cudaMalloc -- code running under a framework's caching allocator that owns
 * nearly all device memory (a stray cudaMalloc fails or fragments it),
 * latency-critical loops (cudaMalloc and cudaFree can synchronise the whole
 * device), or hosts whose policy forbids allocation after start-up.
 * Scratch is an 8 MiB static device array inside this library, held by every
 * GPU that loads the library until the process exits; the call itself
 * allocates nothing (no cudaMalloc, cudaFree or pinned host memory; the
 * per-round header is read into static host memory, and profiling is off).
 * Inputs, outputs and stream as for sss_sort.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress); make that
 * first call before any stream capture on the device.  Every call shares the
 * one array and re-initialises what it reads, so calls that overlap on the
 * GPU race on it.  The call returns only after its work on stream has
 * finished (it reads each round's sizes back, and on an error it waits for
 * the work it already queued), so two calls of this library never overlap;
 * kernels a caller enqueues elsewhere that use the array's contents would.
 * n above 65,536, or options whose scratch would exceed the array, return
 * SSS_ERR_TOO_LARGE. */
int sss_sort_noalloc(const uint8_t* chars, const uint64_t* offsets, uint32_t n,
                     uint32_t* out_perm, uint32_t* out_lcp, void* stream);

/* As sss_sort with every buffer in host memory: chars (host, chars_bytes
 * long), offsets (host), out_perm and out_lcp (host).  Copies the inputs to
 * the device, sorts (as one graph launch, unless options.profile = 1),
 * copies the results back and returns after the copy.  Copies and sort run
 * on a non-blocking stream the library owns (freed by sss_release), so they
 * neither wait for nor delay the caller's work on the legacy default
 * stream.  Pinned host buffers copy fastest; the time is bound by the host
 * link (the sort itself cannot start before every string has arrived). */
int sss_sort_host(const uint8_t* chars, uint64_t chars_bytes, const uint64_t* offsets,
                  uint32_t n, uint32_t* out_perm, uint32_t* out_lcp);

/* Sort num_sets independent sets at once, in one launch of a CUDA graph:
 * every set is a root segment and all sets advance through the same
 * distribution rounds together; the round loop is a conditional graph node
 * decided on the device, so the call makes one graph launch and one final
 * header readback (with options.profile = 1 the rounds are host-driven and
 * timed instead, as for sss_sort).  The instantiated graph is cached while the buffers,
 * sizes and options stay the same.  set_begin (host or device, num_sets + 1
 * uint64 entries, non-decreasing, set_begin[0] = 0, set_begin[num_sets] = n)
 * gives set j the strings with global index in [set_begin[j], set_begin[j+1]);
 * a device array is read back once on stream (8 (num_sets + 1) bytes) before
 * the sort.  n repeats the total so that the entries can be checked: a
 * violation returns SSS_ERR_INVALID.
 * Outputs
 * are per set: for rank r inside set j (global position set_begin[j] + r),
 * out_perm holds the index relative to set_begin[j], and out_lcp is 0 at
 * each set's first position. */
int sss_sort_batched(const uint8_t* chars, const uint64_t* offsets, uint32_t n,
                     const uint64_t* set_begin, uint32_t num_sets,
                     uint32_t* out_perm, uint32_t* out_lcp, void* stream);

/* Autotuner for the batched sort (an addition to the paper): picks the tree
 * depth (v = 2^k - 1 splitters, k = 5..10), the base-case threshold, the
 * medium threshold, the device-wide work-item size ("tile"), the key width
 * and the classifier by coordinate descent, timing graph-form sss_sort_batched runs (median of three, CUDA
 * events on stream) of the caller's tuning batch -- use a batch of the same
 * shape as the real work but different data.  Arguments as for
 * sss_sort_batched; out_perm/out_lcp (device) receive the last run's output.
 * cache_path (host string, nullable): JSON-lines file; an entry whose key
 * (device name, SM count, n and num_sets rounded to two significant digits)
 * matches is used without timing anything, otherwise the winner is appended.
 * The chosen options become the current options (sss_set_options) and are
 * written to *out_best (host); *out_ms (host, nullable) gets the winner's
 * time in milliseconds. */
int sss_autotune_batched(const uint8_t* chars, const uint64_t* offsets, uint32_t n,
                         const uint64_t* set_begin, uint32_t num_sets,
                         uint32_t* out_perm, uint32_t* out_lcp, const char* cache_path,
                         sss_options* out_best, double* out_ms, void* stream);

/* Learned bucket proposal (an addition to the paper, closest to the jump
 * tables of App. A.2): as sss_sort, but in every device-wide distribution
 * round each segment of at least 65,536 strings fits a monotone
 * piecewise-linear CDF of its key words (cdf_segments pieces, FP32) on a
 * sample of 0.1 % of its strings (2,048 to 65,536 keys) -- the pieces spread
 * over the key groups the sample's first differing byte defines, in
 * proportion to their keys; started from the line through the sample's
 * per-piece mean points, then
 * cdf_steps Adam steps of hand-written forward and backward passes on the
 * GPU -- and classification first proposes a bucket from the model and
 * checks it exactly against the bounding splitters (and the neighbouring
 * intervals); only rejected proposals descend the splitter tree.  Output is
 * identical to sss_sort.  stats (host, nullable) receives the proposals,
 * the rejected ones, their ratio and the number of models fitted (also in
 * learned_keys, learned_misses and learned_models of sss_stats); it is
 * written only on success. */
int sss_sort_learned(const uint8_t* chars, const uint64_t* offsets, uint32_t n,
                     uint32_t* out_perm, uint32_t* out_lcp, void* stream,
                     sss_learned_stats* stats);

/* ------------------------------------------------- single steps (testing) */

/* Key word of Sec. 3.1 for each string: the 8 bytes of string idx[i] at
 * depth[i], first byte most significant, bytes after the terminator 0.
 * idx (device, nullable = identity), depth (device, uint32 per i), out_keys
 * (device).  depth[i] must not exceed the length of string idx[i]. */
int sss_gather_keys(const uint8_t* chars, const uint64_t* offsets, const uint32_t* idx,
                    const uint32_t* depth, uint32_t n, uint64_t* out_keys, void* stream);

/* Splitter choice of Sec. 3.1 "Implementation Details" on a sample: sorts
 * the count keys of sample (device, 1 <= count <= 2^(k+1) - 1), picks
 * v = 2^k - 1 splitters by the recursive duplicate-skipping rule and writes
 * them in level order (out_level[0] = root) and in order (both device,
 * v entries).  1 <= k <= 10. */
int sss_build_splitters(const uint64_t* sample, uint32_t count, int32_t k,
                        uint64_t* out_level, uint64_t* out_inorder, void* stream);

/* Classification of Sec. 3.1 / Fig. 1: bucket 2j + [key = x_j] where
 * j = #{splitters < key}, by descending the level-order tree (device,
 * v = 2^k - 1 entries, as written by sss_build_splitters) and one equality
 * test against the in-order array.  out_bucket (device, uint16 per key). */
int sss_classify(const uint64_t* keys, uint32_t n, const uint64_t* level, const uint64_t* inorder,
                 int32_t k, uint16_t* out_bucket, void* stream);

/* The same classification by the pS^5-Equal descent of Sec. 3.1: an
 * equality test at each node of the level-order tree (device, v = 2^k - 1
 * entries) with early exit; a key equal to node i stops in the equality
 * bucket of that splitter, whose in-order index follows from i by bit
 * operations.  With distinct splitters the buckets equal sss_classify's; with
 * repeated splitters a key equal to them may land in the equality bucket of
 * another copy (consistently for equal keys).  out_bucket (device, uint16). */
int sss_classify_equal(const uint64_t* keys, uint32_t n, const uint64_t* level, int32_t k,
                       uint16_t* out_bucket, void* stream);

/* The learned model's loss and gradient, exposed so the fit can be checked.
 * Model with M pieces on [0,1]: increments softplus(theta_j), normalised
 * cumulative knots, F linear inside a piece.  theta (device, float32[M],
 * 1 <= M <= 4096), u (device, float32[S], clamped to [0,1]; any order),
 * y (device, float32[S] targets), 1 <= S <= 2^22.  Writes the mean of
 * (F(u_s) - y_s)^2 to *out_loss (device float32) and dLoss/dtheta to
 * out_grad (device float32[M]); computed in FP32 on one CTA by the code the
 * fit uses (the gradient from per-piece sample statistics, the loss sample
 * by sample). */
int sss_cdf_loss_grad(const float* theta, uint32_t M, const float* u, const float* y,
                      uint32_t S, float* out_loss, float* out_grad, void* stream);

/* ---------------------------------------------------------- management */

int sss_set_options(const sss_options* opt);   /* opt (host) */
int sss_get_options(sss_options* opt);         /* opt (host) */
int sss_get_last_stats(sss_stats* stats);      /* stats (host) */

/* Launch timeline of the last host-driven call made with options.profile = 1
 * (empty otherwise): for each timed launch i in launch order, its kernel class
 * cls[i] (SSS_K_*) and its start and end in milliseconds from the first
 * launch's start, measured with CUDA events on the stream it ran on (the
 * concurrent branches of a round overlap).  Writes min(count, cap) entries
 * (all arrays host, cap entries each; NULL allowed when cap = 0) and the
 * total count to *out_count. */
int sss_get_last_timeline(uint32_t cap, int32_t* cls, double* start_ms, double* end_ms, uint32_t* out_count);
const char* sss_last_error(void);              /* static storage, never NULL */
int sss_release(void);                         /* frees the workspace cache of every device */
const char* sss_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SSS_H */
