// Internal declarations of the GB300 S^5 library: device data structures,
// device helpers shared by the kernels, and the launch functions the host
// driver calls.  Nothing here is part of the public ABI (include/sss.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace sss {

// ------------------------------------------------------------ limits

constexpr int kKMax = 10;                       // deepest splitter tree
constexpr int kVMax = (1 << kKMax) - 1;         // 1023 splitters
constexpr int kNBMax = 2 * kVMax + 1;           // 2047 buckets (Sec. 3.1: k = 2v + 1)
constexpr int kSampleMax = 1 << (kKMax + 1);    // sample buffer, 2v + 1 keys padded to 2^(k+1)
constexpr uint32_t kBaseCap = 256;              // slots of one base-case tile
constexpr uint32_t kBaseMax = kBaseCap / 2;     // largest base-case bucket (128)
constexpr uint32_t kTinyMax = 32;               // base-case buckets this small get one warp each
constexpr uint32_t kRunPiece = 2048;            // strings per work item of a large run of equal strings
constexpr uint32_t kMedMax = 8192;              // largest bucket one CTA distributes alone
constexpr int kMedKMax = 9;                     // its deepest tree: choose_k(8192) = 9
constexpr int kMedNB = (2 << kMedKMax) - 1;     // 1023 buckets
// medium buckets this small take one warp each (0: all take a CTA)
#ifndef SSS_MED_WARP_MAX
#define SSS_MED_WARP_MAX 1023u
#endif
constexpr uint32_t kMedWarpMax = SSS_MED_WARP_MAX;
constexpr int kMWKMax = 5;                       // their deepest tree: choose_k(1023) = 5
constexpr int kMWNB = (2 << kMWKMax) - 1;        // 63 buckets
static_assert(kMedWarpMax < 1024u, "a per-warp medium bucket's tree has at most kMWKMax levels");
#ifndef SSS_CHUNKS_PER_SM
#define SSS_CHUNKS_PER_SM 8
#endif
constexpr int kChunksPerSM = SSS_CHUNKS_PER_SM; // device-wide rounds: target work items per SM
constexpr int kScatterThreads = 256;
constexpr int kScatterItems = 4;                // records per thread in a device-wide move
constexpr uint32_t kSubTile = 2048;             // work-chunk granularity (a multiple of every move sub-tile)
constexpr uint32_t kLcpFlag = 0x80000000u;      // out_lcp entry still to be resolved
constexpr uint32_t kNoRefill = 0xFFFFFFFFu;
constexpr uint32_t kSingle = 0xFFFFFFFEu;       // bucket of one string: finished at scatter

// ------------------------------------------------------------ structures

// One string in the working arrays: its cached characters, where it lives,
// and its index.  32 bytes, so a string moved to a scattered position is one
// whole 32-byte sector write.
struct __align__(32) Rec {
    uint64_t key;   // key word at the segment's depth (Sec. 3.1)
    uint64_t key2;  // the next 8 characters, valid when off's top bit is set
    uint64_t off;   // byte offset of the string in chars; top bit: key2 valid
    uint32_t idx;   // original index
    uint32_t pad;
};

__device__ __forceinline__ Rec load_rec(const Rec* p) {
    const ulonglong2* q = reinterpret_cast<const ulonglong2*>(p);
    const ulonglong2 a = q[0], b = q[1];
    Rec r;
    r.key = a.x; r.key2 = a.y; r.off = b.x;
    r.idx = (uint32_t)b.y; r.pad = (uint32_t)(b.y >> 32);
    return r;
}

__device__ __forceinline__ void store_rec(Rec* p, const Rec& r) {
    ulonglong2* q = reinterpret_cast<ulonglong2*>(p);
    q[0] = make_ulonglong2(r.key, r.key2);
    q[1] = make_ulonglong2(r.off, (uint64_t)r.idx);
}

// A range of positions [begin, begin + size) of the working arrays whose
// strings share their first `depth` bytes (the common prefix l of Sec. 3.1).
struct Seg {
    uint32_t begin, size, depth, aux;
};

// A large segment's layout for one device-wide distribution round.
struct SegPlan {
    uint32_t begin, size, depth, k;     // v = 2^k - 1 splitters, 2^(k+1) - 1 buckets
    uint32_t chunks, chunk_base;        // work items of this segment
    uint32_t count_base, tree_base;     // offsets into the count matrix and the trees
    uint32_t chunk;                     // strings per work item in this round
    uint32_t kp;                        // k as planned (sizes the count rows and the sample);
                                        // k_sample may lower k to the levels its splitters use
    uint32_t rbits;                     // > 0: classified by a digit of rbits bits (radix), not the tree
    uint32_t rskip;                     // leading key bits every sample key shares (radix)
    uint64_t rbase;                     // those shared bits (the rest 0) (radix)
};

// Radix classification of a segment (App. A.2, adaptivity: chosen from the
// sample's digit entropy by k_sample).  The sample keys share their first
// rskip bits; a key's next rbits bits form its digit.  Buckets: 0 holds the
// keys whose first rskip bits are below the shared ones, 1 + digit the keys
// that share them, 2^rbits + 1 the keys above.  Only the first key word
// (8 characters) is used.
__device__ __forceinline__ uint32_t radix_bucket(uint64_t h, uint32_t rskip, uint32_t rbits, uint64_t rbase) {
    if (rskip) {
        const uint64_t hp = h >> (64u - rskip), bp = rbase >> (64u - rskip);
        if (hp != bp) return hp < bp ? 0u : (1u << rbits) + 1u;
    }
    return 1u + (uint32_t)((h << rskip) >> (64u - rbits));
}
__device__ __forceinline__ uint32_t radix_buckets(uint32_t rbits) { return (1u << rbits) + 2u; }

// Device header: live append counters and the snapshot the host reads back.
struct Hdr {
    // live, appended to by the round kernels
    uint32_t n_large, n_med, n_small, n_bigrun, err, small_elems, med_elems, n_tiny, tiny_elems;
    uint32_t learned_models;  // segment models fitted by k_cdf_fit
    uint32_t radix_segments;  // segments of device-wide rounds classified by a digit
    uint32_t n_medw;          // children for the next round's one-warp-per-bucket medium round
    // snapshot for the host, written by k_plan
    uint32_t L, total_chunks, total_counts, total_tree;
    uint32_t n_med_snap, n_small_snap, n_bigrun_snap, small_elems_snap;
    uint32_t large_elems_snap, med_elems_snap, chunk, round;  // round: rounds done (buffer parity)
    uint32_t n_tiny_snap, tiny_elems_snap, n_medw_snap, pad1;
    unsigned long long refills;   // key words gathered in device-wide rounds
    unsigned long long med_refills;  // key words gathered in medium (per-CTA) rounds
    unsigned long long base_iters;  // base-case refill iterations summed over tiles
    unsigned long long learned_keys, learned_misses;  // proposals made / rejected by the exact check
    // work queues of the persistent kernels (reset by k_plan)
    uint32_t q_sample, q_fit, q_classify, q_scatter, q_med, q_base, q_bigrun, q_medw;
    uint32_t small_hist[8];         // base-case segments by floor(log2(size))
};

// err bits
constexpr uint32_t kErrLargeOverflow = 1u << 0;
constexpr uint32_t kErrSmallOverflow = 1u << 1;
constexpr uint32_t kErrRunOverflow = 1u << 2;
constexpr uint32_t kErrEqualBoundary = 1u << 3;
constexpr uint32_t kErrPlanOverflow = 1u << 4;
constexpr uint32_t kErrPosition = 1u << 5;
constexpr uint32_t kErrBaseIters = 1u << 6;
constexpr uint32_t kErrMedOverflow = 1u << 7;

// Refill steps a base-case tile may take (each moves 8 bytes deeper): a
// common prefix of 512 KiB inside one small bucket.
constexpr uint32_t kBaseMaxIters = 1u << 16;

// Tunables passed to kernels.
struct Params {
    int learned;              // classify device-wide rounds with the learned CDF proposal
    uint32_t cdf_M;           // linear pieces of the CDF model
    uint32_t cdf_steps;       // Adam steps per fit
    float cdf_lr;             // Adam step size
    int k_max;
    uint32_t base_threshold;  // <= kBaseMax: bucket goes to the warp-tile base case
    uint32_t med_threshold;   // <= kMedMax: bucket gets one CTA for its next round
    uint32_t chunk;           // largest work item of a device-wide round
    uint64_t seed;
    uint32_t num_sms;
    uint32_t key_bytes;       // w: 8 (one key word) or 16 (two words, wide keys)
    uint32_t equal_test;      // 1: equality test at every tree node (pS^5-Equal)
    uint32_t radix;           // 0: splitter trees only; 1: a digit where the sample's digits are
                              // near uniform; 2: a digit wherever the sample keys differ
    uint32_t fuse_root;       // 1: one root above the medium threshold, whose first round samples
                              // the strings directly and classifies while the records are built
};

// Views of the workspace and the caller's buffers for one sort.
struct Work {
    const uint8_t* chars;
    const uint64_t* offsets;
    uint32_t n;
    uint32_t* out_perm;
    uint32_t* out_lcp;
    // alphabet compression (sss_alphabet.cu): chars/offsets are then the
    // packed copy, alpha_g its characters per byte (0: plain strings)
    uint32_t alpha_g;
    const uint32_t* alpha_dig;  // [256] digits of each packed byte, one per nibble from the top
    const uint32_t* alpha_len;  // [n] length of each string in characters

    Rec* rec[2];             // the string at each position (ping-pong per round)
    uint32_t* counts;        // [cmax] per (segment, bucket, chunk) counts
    uint32_t* counts_scan;   // [cmax] exclusive scan of counts
    uint64_t* tree_lvl;      // [2 * tmax] level-order trees (one or two words a node)
    uint64_t* tree_ino;      // [2 * tmax] the same splitters in order
    SegPlan* plans;          // [lmax]
    uint32_t* chunk_seg;     // [chmax]
    Seg* large;              // [lmax] children for the next device-wide round
    // child lists by parity: a round with round counter r appends to parity
    // (r + 1) & 1 while the base case of the children of round r - 1 reads
    // parity r & 1 concurrently
    Seg* med[2];             // [mmax] children for the next per-CTA round
    Seg* medw[2];            // [mmax] children for the next per-warp round (at most kMedWarpMax strings)
    Seg* small[2];           // [smax] children for the base case (tile form)
    Seg* tiny[2];            // [ymax] children of at most kTinyMax strings (warp form)
    Seg* bigrun[2];          // [bmax] pieces of large runs of equal strings
    uint16_t* bids;          // [n] bucket of each string of a device-wide round (k_classify -> k_scatter)
    uint32_t* scan_tmp;      // [scan_tmp_max] scan scratch of the distribution rounds
    Hdr* hdr;
    // learned proposal (allocated for sss_sort_learned only)
    float* cdf_tab;          // [lmax * (M + 1)] CDF at the knots of each segment's model
    struct CdfNorm* cdf_norm;  // [lmax] input coordinate of each segment's model

    uint32_t cmax, tmax, lmax, chmax, smax, ymax, bmax, scan_tmp_max, mmax;
};

// ------------------------------------------------------------ device helpers

// Bit 7 set in exactly the zero bytes of x (no carries between bytes).
__device__ __forceinline__ uint64_t zero_byte_mask(uint64_t x) {
    const uint64_t lo7 = 0x7F7F7F7F7F7F7F7Full;
    return ~(((x & lo7) + lo7) | x | lo7);
}

__device__ __forceinline__ uint64_t bswap64(uint64_t x) {
    uint32_t lo = (uint32_t)x, hi = (uint32_t)(x >> 32);
    return ((uint64_t)__byte_perm(lo, 0, 0x0123) << 32) | (uint64_t)__byte_perm(hi, 0, 0x0123);
}

// The first byte at or after `valid_from` (a byte index) that is zero, as a
// mask of the bytes before it (all ones if there is none).
__device__ __forceinline__ uint64_t keep_before_zero(uint64_t x) {
    const uint64_t zm = zero_byte_mask(x);
    if (!zm) return ~0ull;
    const uint32_t nb = (uint32_t)(__ffsll((long long)zm) - 1) >> 3;  // bytes before the terminator
    return nb ? (~0ull >> (64u - 8u * nb)) : 0ull;
}

// Key words (Sec. 3.1) of the 16 bytes at chars[off ..]: k1 = bytes
// off..off+7, k2 = bytes off+8..off+15, each packed first-byte-most-
// significant, every byte after the first 0 set to 0 (k2 = 0 when k1 holds
// the terminator).  Reads only aligned 8-byte words; a word beyond the first
// is read either because no terminator came before it (so it holds a string
// byte) or, speculatively, because it lies in the same 4 KiB page as the
// first word (which holds a string byte).  So no page the string does not
// reach is ever touched.
__device__ __forceinline__ void load_key2(const uint8_t* __restrict__ chars, uint64_t off, uint64_t& k1,
                                          uint64_t& k2) {
    const uint64_t addr = reinterpret_cast<uint64_t>(chars) + off;
    const uint64_t a8 = addr & ~7ull;
    const uint64_t* w = reinterpret_cast<const uint64_t*>(a8);
    const uint32_t sh = (uint32_t)(addr & 7u) * 8u;
    uint64_t w0, w1, w2;
    if ((a8 & 4095u) <= 4096u - 24u) {  // all three words in one page
        w0 = __ldg(w);
        w1 = __ldg(w + 1);
        w2 = sh ? __ldg(w + 2) : 0ull;
    } else {
        w0 = __ldg(w);
        w1 = 0ull;
        w2 = 0ull;
        if ((zero_byte_mask(w0 >> sh) & (~0ull >> sh)) == 0) {
            w1 = __ldg(w + 1);
            if (sh && zero_byte_mask(w1) == 0) w2 = __ldg(w + 2);
        }
    }
    uint64_t r1 = sh ? (w0 >> sh) | (w1 << (64u - sh)) : w0;
    uint64_t r2 = sh ? (w1 >> sh) | (w2 << (64u - sh)) : w1;
    const uint64_t m1 = keep_before_zero(r1);
    if (m1 != ~0ull) {
        r1 &= m1;
        r2 = 0ull;
    } else {
        r2 &= keep_before_zero(r2);
    }
    k1 = bswap64(r1);
    k2 = bswap64(r2);
}

// Key word (Sec. 3.1): bytes chars[off .. off+7] packed first-byte-most-
// significant, bytes after the first 0 set to 0 (same reading rule as
// load_key2).
__device__ __forceinline__ uint64_t load_key(const uint8_t* __restrict__ chars, uint64_t off) {
    const uint64_t addr = reinterpret_cast<uint64_t>(chars) + off;
    const uint64_t a8 = addr & ~7ull;
    const uint64_t* w = reinterpret_cast<const uint64_t*>(a8);
    const uint32_t sh = (uint32_t)(addr & 7u) * 8u;
    uint64_t lo;
    if (sh && (a8 & 4095u) <= 4096u - 16u) {
        lo = (__ldg(w) >> sh) | (__ldg(w + 1) << (64u - sh));
    } else {
        lo = __ldg(w) >> sh;
        if (sh && (zero_byte_mask(lo) & (~0ull >> sh)) == 0) lo |= __ldg(w + 1) << (64u - sh);
    }
    return bswap64(lo & keep_before_zero(lo));
}

// Characters cached per string: the key word at the current depth (k1) and,
// when the top bit of the carried offset is set, the next word (k2).  A
// refill that moves delta <= 8 bytes deeper takes its word from the cache
// (and empties it); otherwise 16 bytes are gathered (caching of characters,
// Sec. 2.2, with 16 characters instead of 8).
constexpr uint64_t kK2Valid = 1ull << 63;
constexpr uint64_t kOffMask = ~kK2Valid;

__device__ __forceinline__ void refill(const uint8_t* __restrict__ chars, uint64_t& k1, uint64_t& k2,
                                       uint64_t& o, uint32_t new_depth, uint32_t delta) {
    if ((o & kK2Valid) && delta <= 8u) {
        k1 = delta == 8u ? k2 : (k1 << (8u * delta)) | (k2 >> (64u - 8u * delta));
        o &= kOffMask;
    } else {
        load_key2(chars, (o & kOffMask) + new_depth, k1, k2);
        o |= kK2Valid;
    }
}

// LCP in bytes of two different key words (XOR + count leading zeros, Sec. 3.1).
__device__ __forceinline__ uint32_t key_lcp(uint64_t a, uint64_t b) {
    return (uint32_t)__clzll((long long)(a ^ b)) >> 3;
}

// A key word holds the terminator iff its last byte is 0 (bytes after the
// terminator are 0, bytes before it are not).
__device__ __forceinline__ bool key_ends(uint64_t k) { return (k & 0xFFull) == 0; }

// Characters before the terminator in a key word that holds one.
__device__ __forceinline__ uint32_t key_chars(uint64_t k) {
    return k ? 8u - ((uint32_t)__ffsll((long long)k) - 1u) / 8u : 0u;
}

// ------------------------------------------------------------ key types

// The classification key of a round: one word of w = 8 characters (Sec. 3.1)
// or, in the wide form, two words (w = 16 characters) compared as one
// 128-bit big-endian number.  A wide key lets one round step over 16 shared
// characters, so inputs with long common prefixes need about half the rounds.
struct __align__(16) Key16 {
    uint64_t h, l;  // characters 0..7 and 8..15 at the depth
};

__device__ __forceinline__ bool kgt(uint64_t a, uint64_t b) { return a > b; }
__device__ __forceinline__ bool kgt(const Key16& a, const Key16& b) { return a.h > b.h || (a.h == b.h && a.l > b.l); }
__device__ __forceinline__ bool keq(uint64_t a, uint64_t b) { return a == b; }
__device__ __forceinline__ bool keq(const Key16& a, const Key16& b) { return a.h == b.h && a.l == b.l; }

// The key holds the terminator (bytes after it are zero).
__device__ __forceinline__ bool kends(uint64_t x) { return key_ends(x); }
__device__ __forceinline__ bool kends(const Key16& x) { return key_ends(x.l); }
// Characters before the terminator of a key that holds one.
__device__ __forceinline__ uint32_t kchars(uint64_t x) { return key_chars(x); }
__device__ __forceinline__ uint32_t kchars(const Key16& x) {
    return key_ends(x.h) ? key_chars(x.h) : 8u + key_chars(x.l);
}
// Common leading characters of two different keys.
__device__ __forceinline__ uint32_t klcp(uint64_t a, uint64_t b) { return key_lcp(a, b); }
__device__ __forceinline__ uint32_t klcp(const Key16& a, const Key16& b) {
    return a.h != b.h ? key_lcp(a.h, b.h) : 8u + key_lcp(a.l, b.l);
}

template <class KT> struct KeyTraits;
template <> struct KeyTraits<uint64_t> {
    static constexpr uint32_t kBytes = 8;
    __device__ static __forceinline__ uint64_t of(const Rec& r) { return r.key; }
    __device__ static __forceinline__ uint64_t load(const Rec* p) { return p->key; }
    __device__ static __forceinline__ uint64_t top() { return ~0ull; }
    __device__ static __forceinline__ uint64_t word(uint64_t x) { return x; }
};
template <> struct KeyTraits<Key16> {
    static constexpr uint32_t kBytes = 16;
    __device__ static __forceinline__ Key16 of(const Rec& r) { return Key16{r.key, r.key2}; }
    __device__ static __forceinline__ Key16 load(const Rec* p) {
        const ulonglong2 a = *reinterpret_cast<const ulonglong2*>(p);
        return Key16{a.x, a.y};
    }
    __device__ static __forceinline__ Key16 top() { return Key16{~0ull, ~0ull}; }
    __device__ static __forceinline__ uint64_t word(const Key16& x) { return x.h; }
};

// Byte j (first character most significant) of a key.
__device__ __forceinline__ uint32_t kbyte(uint64_t x, uint32_t j) { return (uint32_t)(x >> (56u - 8u * j)) & 0xFFu; }
__device__ __forceinline__ uint32_t kbyte(const Key16& x, uint32_t j) {
    return j < 8u ? kbyte(x.h, j) : kbyte(x.l, j - 8u);
}

// LCP entry (in characters) of two strings whose keys at `depth` differ.
// With alphabet compression a byte holds g characters as base-(sigma'+1)
// digits: depth and the common key bytes count g characters each, and the
// first differing byte adds its leading digits that still agree.
template <class KT>
__device__ __forceinline__ uint32_t lcp_of_keys(const Work& w, uint32_t depth, const KT& a, const KT& b) {
    const uint32_t j = klcp(a, b);
    if (!w.alpha_g) return depth + j;
    const uint32_t x = __ldg(&w.alpha_dig[kbyte(a, j)]) ^ __ldg(&w.alpha_dig[kbyte(b, j)]);
    return w.alpha_g * (depth + j) + ((uint32_t)__clz((int)x) >> 2);
}

// LCP entry of two equal strings: `chars` (their length counted in key
// bytes), or with alphabet compression the length of string idx.
__device__ __forceinline__ uint32_t lcp_of_equal(const Work& w, uint32_t chars, uint32_t idx) {
    return w.alpha_g ? __ldg(&w.alpha_len[idx]) : chars;
}

// Moves a record's cached characters from `depth` to `new_depth`: the
// narrow form may reuse the second cached word, the wide form needs both
// words at the new depth and gathers them.
template <class KT>
__device__ __forceinline__ void refill_rec(const uint8_t* __restrict__ chars, Rec& r, uint32_t new_depth,
                                           uint32_t depth) {
    if (KeyTraits<KT>::kBytes == 8) {
        refill(chars, r.key, r.key2, r.off, new_depth, new_depth - depth);
    } else {
        load_key2(chars, (r.off & kOffMask) + new_depth, r.key, r.key2);
        r.off |= kK2Valid;
    }
}

// Tree depth for a segment of `size` strings: about 16 strings per splitter.
__host__ __device__ __forceinline__ int choose_k(uint32_t size, int k_max) {
#ifdef __CUDA_ARCH__
    int lg = 31 - __clz(size | 1u);
#else
    int lg = 31 - __builtin_clz(size | 1u);
#endif
    int k = lg - 4;
    if (k > k_max) k = k_max;
    if (k < 1) k = 1;
    return k;
}

// Level-order splitter trees in shared memory.  A wide-key tree keeps the
// first and second words in separate arrays: a descent step reads the first
// word (8 bytes) and the second only when the first words tie, which halves
// the shared-memory traffic of the descent.
struct SplitTree {
    const uint64_t* h;
    const uint64_t* l;
};
template <class KT, int N> struct LevelTree;
template <int N> struct LevelTree<uint64_t, N> {
    uint64_t w[N];
    __device__ __forceinline__ void set(uint32_t i, uint64_t x) { w[i] = x; }
    __device__ __forceinline__ const uint64_t* view() const { return w; }
};
template <int N> struct LevelTree<Key16, N> {
    uint64_t h[N], l[N];
    __device__ __forceinline__ void set(uint32_t i, const Key16& x) { h[i] = x.h; l[i] = x.l; }
    __device__ __forceinline__ SplitTree view() const { return SplitTree{h, l}; }
};

// key > node i of a level-order tree
__device__ __forceinline__ bool node_gt(uint64_t key, const uint64_t* t, uint32_t i) { return key > t[i]; }
__device__ __forceinline__ bool node_gt(const Key16& key, const Key16* t, uint32_t i) { return kgt(key, t[i]); }
__device__ __forceinline__ bool node_gt(const Key16& key, const SplitTree& t, uint32_t i) {
    const uint64_t h = t.h[i];
    return key.h != h ? key.h > h : key.l > t.l[i];
}

// Branch-free descent of the level-order tree t[1..v] (Sec. 3.1, i := 2i + {0,1})
// then one equality test against the in-order array: bucket 2j + [key = x_j].
template <class KT, class TT>
__device__ __forceinline__ uint32_t classify_key(const KT& key, const TT& t, const KT* ino, int k) {
    uint32_t i = 1;
    for (int l = 0; l < k; l++) i = 2u * i + (node_gt(key, t, i) ? 1u : 0u);
    const uint32_t v = (1u << k) - 1u;
    const uint32_t j = i - (1u << k);
    return 2u * j + ((j < v && keq(key, ino[j])) ? 1u : 0u);
}

// classify_key for U keys at once, descending the U paths level by level so
// that each level issues U independent shared-memory loads (the interleaved
// descents of Sec. 3.1).
template <int U, class KT, class TT>
__device__ __forceinline__ void classify_keys(const KT (&key)[U], uint32_t (&b)[U], const TT& t, const KT* ino, int k) {
    uint32_t i[U];
#pragma unroll
    for (int u = 0; u < U; u++) i[u] = 1u;
    for (int l = 0; l < k; l++) {
#pragma unroll
        for (int u = 0; u < U; u++) i[u] = 2u * i[u] + (node_gt(key[u], t, i[u]) ? 1u : 0u);
    }
    const uint32_t v = (1u << k) - 1u;
#pragma unroll
    for (int u = 0; u < U; u++) {
        const uint32_t j = i[u] - (1u << k);
        b[u] = 2u * j + ((j < v && keq(key[u], ino[j])) ? 1u : 0u);
    }
}

// Three-way compare of a key with node i: -1, 0 (equal) or 1.
__device__ __forceinline__ int node_cmp(uint64_t key, const uint64_t* t, uint32_t i) {
    const uint64_t x = t[i];
    return key == x ? 0 : (key > x ? 1 : -1);
}
__device__ __forceinline__ int node_cmp(const Key16& key, const SplitTree& t, uint32_t i) {
    const uint64_t h = t.h[i];
    if (key.h != h) return key.h > h ? 1 : -1;
    const uint64_t l = t.l[i];
    return key.l == l ? 0 : (key.l > l ? 1 : -1);
}

// The pS^5-Equal classifier (Sec. 3.1, the variant that tests for equality
// at each node): a key equal to node i of level lv stops there, in the
// equality bucket of that splitter, whose in-order index comes from the
// node's position by bit operations; a key that reaches a leaf j without a
// tie gets the even bucket 2j.  U keys descend level by level.
template <int U, class KT, class TT>
__device__ __forceinline__ void classify_keys_equal(const KT (&key)[U], uint32_t (&b)[U], const TT& t, int k) {
    uint32_t i[U];
    bool done[U];
#pragma unroll
    for (int u = 0; u < U; u++) { i[u] = 1u; done[u] = false; }
    for (int lv = 0; lv < k; lv++) {
#pragma unroll
        for (int u = 0; u < U; u++) {
            if (!done[u]) {
                const int c = node_cmp(key[u], t, i[u]);
                if (c == 0) {
                    const uint32_t q = i[u] - (1u << lv);
                    b[u] = 2u * ((2u * q + 1u) * (1u << (k - 1 - lv)) - 1u) + 1u;
                    done[u] = true;
                } else {
                    i[u] = 2u * i[u] + (c > 0 ? 1u : 0u);
                }
            }
        }
    }
#pragma unroll
    for (int u = 0; u < U; u++)
        if (!done[u]) b[u] = 2u * (i[u] - (1u << k));
}

// Either classifier: equality after the full descent (pS^5-Unroll) or at
// every node (pS^5-Equal).
template <int U, class KT, class TT>
__device__ __forceinline__ void classify_keys_by(bool equal_test, const KT (&key)[U], uint32_t (&b)[U], const TT& t,
                                                 const KT* ino, int k) {
    if (equal_test) classify_keys_equal<U>(key, b, t, k);
    else classify_keys<U>(key, b, t, ino, k);
}

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Work items of a queue-driven kernel: CTA b starts with item b, then takes
// items gridDim.x, gridDim.x + 1, ... in order from the queue counter q (so a
// grid of exactly one CTA per item never touches the counter); the caller
// stops at its item count.  next_item contains barriers.
__device__ __forceinline__ uint32_t first_item() { return blockIdx.x; }
__device__ __forceinline__ uint32_t next_item(uint32_t* q, uint32_t* s_item) {
    __syncthreads();  // everyone is done with the previous item
    if (threadIdx.x == 0) *s_item = gridDim.x + atomicAdd(q, 1u);
    __syncthreads();
    return *s_item;
}

// ------------------------------------------------------------ learned proposal

// Segments smaller than this are classified by the tree alone (a model's fit
// costs more than it can save on them).
constexpr uint32_t kLearnedMinSize = 1u << 16;

// Input coordinate of a segment's model, t in [0, M] (the model's pieces
// are [m, m + 1)), in two levels.  The fit sample's smallest and largest
// keys share their first c bytes, so every key between them does too; its
// byte c (the digit) picks one of at most 256 key groups, and group d owns
// pieces [O_d, O_{d+1}), its share of the M pieces proportional to its
// share of the sample.  Inside a group, u2 = (key - gmin_d) / (gmax_d -
// gmin_d) measures the key from the group's own smallest sample key, past
// the prefix the group shares, and t = O_d + (O_{d+1} - O_d) u2.  A single
// normalisation over the whole sample (u = (key - kmin) / (kmax - kmin) in
// FP32) cannot tell keys apart that differ only after the 24 bits that
// follow the sample's common prefix, which is the rule for URL-like key
// words ("http://a..." and "http://b..." differ in their eighth byte).
// Keys below kmin get t = 0, above kmax t = M.  t is non-decreasing in
// the key.
struct CdfNorm {
    uint64_t kmin, kmax;
    uint32_t c;        // bytes kmin and kmax share (8 when they are equal)
    uint32_t pad;
    uint16_t O[260];   // first piece of digit group d, O[256] = M
    uint64_t gmin[256];
    float gscale[256]; // 1 / (gmax_d - gmin_d), 0 when the group holds one key value
};

__device__ __forceinline__ float cdf_coord(uint64_t key, const CdfNorm& n, uint32_t M) {
    if (key < n.kmin) return 0.0f;
    if (key > n.kmax) return (float)M;
    if (n.c >= 8u) return 0.0f;  // one key value in the sample
    const uint32_t d = (uint32_t)(key >> (56u - 8u * n.c)) & 0xFFu;  // kmin <= key <= kmax share c bytes
    const uint64_t g = n.gmin[d];
    const float u2 = key > g ? fminf(1.0f, __ull2float_rn(key - g) * n.gscale[d]) : 0.0f;
    return (float)n.O[d] + (float)(n.O[d + 1] - n.O[d]) * u2;
}

// Learned bucket proposal with exact verification: the model's CDF value
// F(t) (linear between the knots C[0..M]) proposes j = floor(F (v + 1));
// the key's interval (x_{j-1}, x_j] is checked against the in-order
// splitters, and failing that the neighbouring intervals j-1 and j+1.  On a
// hit returns true and the bucket 2j + [key = x_j] (identical to the tree's
// answer, since these intervals partition the keys); on a miss returns
// false and the caller descends the tree.
__device__ __forceinline__ bool propose_bucket(uint64_t key, const float* C, uint32_t M, const CdfNorm& nrm,
                                               const uint64_t* ino, uint32_t v, uint32_t& bucket) {
    const float t = cdf_coord(key, nrm, M);
    const uint32_t m = min((uint32_t)t, M - 1u);
    const float f = t - (float)m;
    const float F = C[m] + f * (C[m + 1] - C[m]);
    uint32_t j = min((uint32_t)(F * (float)(v + 1u)), v);
    const bool lo_ok = j == 0 || ino[j - 1] < key;
    const bool hi_ok = j == v || key <= ino[j];
    if (!(lo_ok && hi_ok)) {
        if (!lo_ok) {  // key <= x_{j-1}
            j = j - 1u;
            if (!(j == 0 || ino[j - 1] < key)) return false;
        } else {       // key > x_j
            j = j + 1u;
            if (!(j == v || key <= ino[j])) return false;
        }
    }
    bucket = 2u * j + ((j < v && key == ino[j]) ? 1u : 0u);
    return true;
}

// ------------------------------------------------------------ profiling

constexpr int kClasses = 12;  // matches SSS_K_CLASSES of sss.h
enum { kInit = 0, kSample, kClassify, kScan, kScatter, kPlan, kBase, kRuns, kFixup, kLearned, kMedium, kAlphabet };

// Launch counter and optional CUDA-event timing per kernel class, recorded
// on the stream each kernel is launched on.
struct Prof {
    bool enabled = false;
    uint32_t launches = 0;
    uint32_t cls_launches[kClasses] = {};
    std::vector<cudaEvent_t> pool;
    std::vector<int> used_cls;
    size_t next = 0;

    void reset(bool on) {
        enabled = on;
        launches = 0;
        for (int i = 0; i < kClasses; i++) cls_launches[i] = 0;
        used_cls.clear();
        next = 0;
    }
    void begin(int cls, cudaStream_t st) {
        launches++;
        cls_launches[cls]++;
        if (!enabled) return;
        while (pool.size() < next + 2) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) { enabled = false; return; }
            pool.push_back(e);
        }
        cudaEventRecord(pool[next], st);
        used_cls.push_back(cls);
    }
    void end(cudaStream_t st) {
        if (!enabled) return;
        cudaEventRecord(pool[next + 1], st);
        next += 2;
    }
    // after the streams are idle: each timed launch as (class, start, end) in
    // milliseconds from the first launch's start
    void timeline(std::vector<int>& cls, std::vector<double>& t0, std::vector<double>& t1) const {
        cls.clear(); t0.clear(); t1.clear();
        if (!enabled) return;
        for (size_t i = 0; i < used_cls.size(); i++) {
            float a = 0.f, b = 0.f;
            cudaEventElapsedTime(&a, pool[0], pool[2 * i]);
            cudaEventElapsedTime(&b, pool[0], pool[2 * i + 1]);
            cls.push_back(used_cls[i]);
            t0.push_back(a);
            t1.push_back(b);
        }
    }
    // after the stream is idle: summed milliseconds per class
    void collect(double* ms) const {
        for (int i = 0; i < kClasses; i++) ms[i] = 0.0;
        if (!enabled) return;
        for (size_t i = 0; i < used_cls.size(); i++) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, pool[2 * i], pool[2 * i + 1]) == cudaSuccess) ms[used_cls[i]] += t;
        }
    }
};

struct ProfScope {
    Prof* p;
    cudaStream_t st;
    ProfScope(Prof* p_, int cls, cudaStream_t st_) : p(p_), st(st_) { if (p) p->begin(cls, st); }
    ~ProfScope() { if (p) p->end(st); }
};

// ------------------------------------------------------------ launches

// records: the key words at depth 0 of every string (skipped with
// p.fuse_root: launch_fused_root builds them)
cudaError_t launch_init(const Work& w, const Params& p, Prof* pf, cudaStream_t st);
// p.fuse_root: the root's sample and splitter tree straight from the strings,
// then one pass that builds the records and classifies them for round 0
// (round 0's k_sample and k_classify then return at once).  Needs the plan.
cudaError_t launch_fused_root(const Work& w, const Params& p, const Hdr* hc, Prof* pf, cudaStream_t st);
// roots == nullptr: one root [0, n); else num_roots device segments (batched)
cudaError_t launch_roots(const Work& w, const Params& p, const Seg* roots, uint32_t num_roots, Prof* pf,
                         cudaStream_t st);
// The next round's plan; advance 1: and the round counter; 2: and the graph
// form's round-loop condition (cond)
cudaError_t launch_plan(const Work& w, const Params& p, Prof* pf, cudaStream_t st, uint32_t advance = 0u,
                        cudaGraphConditionalHandle cond = 0);
// One distribution round: device-wide kernels for the planned large segments
// and one CTA per medium segment, reading counts and the buffer parity
// (hdr->round) from device memory.  hc: host copy of the header when known
// (exact grids, empty launches skipped), nullptr for persistent grids (graph
// capture).
// Streams and events for running the base case (tile form and warp form),
// the device-wide round and the medium round of one round body concurrently
// (forked from and joined back into the caller's stream).  Stream
// priorities: the device-wide round (the chain the next round waits on)
// highest, the medium rounds next, the base case lowest; the lower branches
// fill the SMs around the higher.
struct Branches {
    cudaStream_t large = nullptr, base = nullptr, medium = nullptr, tiny = nullptr;
    cudaEvent_t fork = nullptr, join_large = nullptr, join_base = nullptr, join_medium = nullptr,
                join_tiny = nullptr;
};
// Creates / destroys the streams and events of a Branches.
cudaError_t branches_create(Branches& b);
void branches_destroy(Branches& b);

// One round body: the base case of the last round's small children (tile and
// warp forms), the device-wide round of the large segments and the per-CTA
// rounds of the medium ones.  With br, the four run as concurrent branches
// of st; without, one after the other on st.  *out_tiles: base-case tiles (host-driven only).
cudaError_t launch_body(const Work& w, const Params& p, const Hdr* hc, uint32_t* out_tiles, Prof* pf,
                        cudaStream_t st, const Branches* br);
cudaError_t launch_set_cond(const Work& w, cudaGraphConditionalHandle cond, cudaStream_t st);
cudaError_t prepare_kernels(uint32_t cdf_M);
cudaError_t prepare_cdf_kernels(uint32_t M);
// base case and large runs of the buckets listed by the last k_plan
cudaError_t launch_small(const Work& w, const Params& p, const Hdr* hc, uint32_t* out_tiles, Prof* pf,
                         cudaStream_t st);
cudaError_t launch_fixup(const Work& w, Prof* pf, cudaStream_t st);
cudaError_t launch_localize(uint32_t* perm, const Seg* roots, uint32_t num_roots, Prof* pf, cudaStream_t st);
cudaError_t launch_scan_u32(const uint32_t* in, uint32_t* out, const uint32_t* n_ptr, const uint32_t* n_host,
                            uint32_t* tmp, uint32_t* done, Prof* pf, cudaStream_t st);
size_t scan_tmp_elems(uint32_t n);
uint32_t device_sms();

cudaError_t launch_gather_keys(const uint8_t* chars, const uint64_t* offsets, const uint32_t* idx,
                               const uint32_t* depth, uint32_t n, uint64_t* out, cudaStream_t st);
cudaError_t launch_build_splitters(const uint64_t* sample, uint32_t count, int k, uint64_t* lvl,
                                   uint64_t* ino, cudaStream_t st);
cudaError_t launch_classify(const uint64_t* keys, uint32_t n, const uint64_t* lvl, const uint64_t* ino,
                            int k, uint16_t* out, int equal_test, cudaStream_t st);
// learned CDF (sss_learned.cu)
size_t cdf_fit_smem(uint32_t M);
cudaError_t launch_cdf_fit(const Work& w, const Params& p, uint32_t grid, Prof* pf, cudaStream_t st);
cudaError_t launch_cdf_loss_grad(const float* theta, uint32_t M, const float* u, const float* y, uint32_t S,
                                 float* loss, float* grad, cudaStream_t st);

}  // namespace sss
