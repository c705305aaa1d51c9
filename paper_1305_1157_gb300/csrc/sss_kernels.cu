// Kernels of super scalar string sample sort (S^5, Sec. 3.1 of Bingmann &
// Sanders) for sm_103a.
//
// Segments (ranges of the working arrays whose strings share a prefix of
// `depth` bytes) are handled by size class, after the paper's split into
// fully parallel S^5, sequential S^5 and a base case (Sec. 3.1
// "Parallelization of S^5"):
//
//   large  (> med_threshold)  device-wide round, all such segments at once:
//          k_sample (one CTA per segment: sample, sort, splitter tree),
//          k_classify (one CTA per work chunk: tree in shared memory,
//          descent, warp-aggregated histogram), exclusive scan of the
//          bucket-major count matrix, k_scatter (one CTA per chunk: stable
//          move into the shadow arrays, key refill, child segments)
//   medium (> base_threshold) k_med_round: one CTA runs a whole round for
//          its segment in shared memory (sample, tree, classify into a
//          bucket array, local scan, stable move, child segments)
//   small  (<= base_threshold) k_base: one CTA sorts a tile of packed small
//          segments, one thread per string, by ranking each element inside
//          its run (key word, then index), moving runs of equal key words 8
//          bytes deeper until all are decided; writes out_perm and the LCP
//
// Between rounds k_plan lays out the next device-wide round.  Equality
// buckets whose splitter ends the string are finished runs (k_bigrun when
// large); k_fixup resolves the LCP at bucket boundaries at the end.
#include <string.h>

#include <type_traits>

#include "sss_internal.cuh"

namespace sss {

#define FULL_MASK 0xFFFFFFFFu

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// ------------------------------------------------------------ block scans

// Exclusive sum over the block (blockDim.x a multiple of 32, <= 1024).
// wsum: shared scratch of 33 entries.  Returns the exclusive prefix; *total
// receives the block total.  Contains __syncthreads.
__device__ uint32_t block_excl_sum(uint32_t x, uint32_t* wsum, uint32_t* total) {
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint32_t nw = blockDim.x >> 5;
    uint32_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(FULL_MASK, inc, o);
        if (lane >= (uint32_t)o) inc += y;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint32_t s = lane < nw ? wsum[lane] : 0u;
        uint32_t si = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(FULL_MASK, si, o);
            if (lane >= (uint32_t)o) si += y;
        }
        if (lane < nw) wsum[lane] = si - s;
        if (lane == nw - 1) wsum[32] = si;
    }
    __syncthreads();
    const uint32_t r = wsum[warp] + inc - x;
    const uint32_t t = wsum[32];
    __syncthreads();
    if (total) *total = t;
    return r;
}

// ------------------------------------------------------------ child segments

// Where a bucket of `size` strings goes next (Sec. 3.1 "Parallelization of
// S^5": size classes).  isrun: all its strings are equal (finished).
enum : uint32_t { kChildNone = 0, kChildRuns, kChildTiny, kChildSmall, kChildMed, kChildLarge, kChildMedW };

__device__ __forceinline__ uint32_t child_kind(const Params& p, uint32_t size, bool isrun) {
    if (size <= 1) return kChildNone;
    if (isrun && size > p.base_threshold) return kChildRuns;
    if (size <= min(p.base_threshold, kTinyMax)) return kChildTiny;
    if (size <= p.base_threshold) return kChildSmall;
    if (size <= p.med_threshold) return size <= kMedWarpMax ? kChildMedW : kChildMed;
    return kChildLarge;
}

__device__ __forceinline__ void warp_add(uint32_t* counter, uint32_t x) {
    x = __reduce_add_sync(FULL_MASK, x);
    if ((threadIdx.x & 31u) == 0 && x) atomicAdd(counter, x);
}

// Exclusive prefix over the lanes of x; *total receives the warp's sum.
__device__ __forceinline__ uint32_t warp_excl(uint32_t x, uint32_t* total) {
    const uint32_t lane = threadIdx.x & 31u;
    uint32_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL_MASK, inc, o);
        if (lane >= (uint32_t)o) inc += y;
    }
    *total = __shfl_sync(FULL_MASK, inc, 31);
    return inc - x;
}

// Appends the child segments of a warp's lanes, PER buckets a lane (kind[q]
// from child_kind, kChildNone for none), to the lists of their size
// classes.  Called by all 32 lanes of a warp together.  Each list's slots
// for all PER buckets of all lanes take one atomic per warp, and lane 31
// issues the lists' atomics back to back before any of their results is
// used, so the warp waits for one round trip, not one per list.
template <int PER>
__device__ __forceinline__ void append_children_n(const Work& w, int out, const uint32_t (&kind)[PER],
                                                  const uint32_t (&start)[PER], const uint32_t (&size)[PER],
                                                  const uint32_t (&cdepth)[PER], const uint32_t (&runlcp)[PER]) {
    Hdr* h = w.hdr;
    uint32_t n_runs = 0, n_tiny = 0, n_small = 0, n_med = 0, n_large = 0, n_medw = 0;
#pragma unroll
    for (int q = 0; q < PER; q++) {
        n_runs += kind[q] == kChildRuns ? (size[q] + kRunPiece - 1u) / kRunPiece : 0u;
        n_tiny += kind[q] == kChildTiny ? 1u : 0u;
        n_small += kind[q] == kChildSmall ? 1u : 0u;
        n_med += kind[q] == kChildMed ? 1u : 0u;
        n_large += kind[q] == kChildLarge ? 1u : 0u;
        n_medw += kind[q] == kChildMedW ? 1u : 0u;
    }
    if (!__any_sync(FULL_MASK, n_runs + n_tiny + n_small + n_med + n_large + n_medw > 0u)) return;
    const uint32_t lane = threadIdx.x & 31u;
    uint32_t t_runs, t_tiny, t_small, t_med, t_large, t_medw;
    const uint32_t x_runs = warp_excl(n_runs, &t_runs), x_tiny = warp_excl(n_tiny, &t_tiny);
    const uint32_t x_small = warp_excl(n_small, &t_small), x_med = warp_excl(n_med, &t_med);
    const uint32_t x_large = warp_excl(n_large, &t_large), x_medw = warp_excl(n_medw, &t_medw);
    uint32_t b_runs = 0, b_tiny = 0, b_small = 0, b_med = 0, b_large = 0, b_medw = 0;
    if (lane == 31u) {
        if (t_runs) b_runs = atomicAdd(&h->n_bigrun, t_runs);
        if (t_tiny) b_tiny = atomicAdd(&h->n_tiny, t_tiny);
        if (t_small) b_small = atomicAdd(&h->n_small, t_small);
        if (t_med) b_med = atomicAdd(&h->n_med, t_med);
        if (t_large) b_large = atomicAdd(&h->n_large, t_large);
        if (t_medw) b_medw = atomicAdd(&h->n_medw, t_medw);
    }
    uint32_t s_runs = __shfl_sync(FULL_MASK, b_runs, 31) + x_runs;
    uint32_t s_tiny = __shfl_sync(FULL_MASK, b_tiny, 31) + x_tiny;
    uint32_t s_small = __shfl_sync(FULL_MASK, b_small, 31) + x_small;
    uint32_t s_med = __shfl_sync(FULL_MASK, b_med, 31) + x_med;
    uint32_t s_large = __shfl_sync(FULL_MASK, b_large, 31) + x_large;
    uint32_t s_medw = __shfl_sync(FULL_MASK, b_medw, 31) + x_medw;
    uint32_t e_tiny = 0, e_small = 0, e_med = 0;
    uint32_t hist[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int q = 0; q < PER; q++) {
        const uint32_t kq = kind[q];
        if (kq == kChildRuns) {
            // large runs of equal strings: pieces of at most kRunPiece
            // strings, so one large run spreads over many CTAs; depth holds
            // the run's first position
            const uint32_t np = (size[q] + kRunPiece - 1u) / kRunPiece;
            if (s_runs + np <= w.bmax) {
                for (uint32_t j = 0; j < np; j++)
                    w.bigrun[out][s_runs + j] = Seg{start[q] + j * kRunPiece,
                                                    min(kRunPiece, size[q] - j * kRunPiece), start[q], runlcp[q]};
            } else {
                atomicOr(&h->err, kErrRunOverflow);
            }
            s_runs += np;
        } else if (kq == kChildTiny) {
            if (s_tiny < w.ymax) {
                w.tiny[out][s_tiny] = Seg{start[q], size[q], cdepth[q], 0u};
                e_tiny += size[q];
            } else {
                atomicOr(&h->err, kErrSmallOverflow);
            }
            s_tiny++;
        } else if (kq == kChildSmall) {
            if (s_small < w.smax) {
                w.small[out][s_small] = Seg{start[q], size[q], cdepth[q], 0u};
                e_small += size[q];
            } else {
                atomicOr(&h->err, kErrSmallOverflow);
            }
            s_small++;
        } else if (kq == kChildMed) {
            if (s_med < w.mmax) {
                w.med[out][s_med] = Seg{start[q], size[q], cdepth[q], 0u};
                e_med += size[q];
            } else {
                atomicOr(&h->err, kErrMedOverflow);
            }
            s_med++;
        } else if (kq == kChildLarge) {
            if (s_large < w.lmax) w.large[s_large] = Seg{start[q], size[q], cdepth[q], 0u};
            else atomicOr(&h->err, kErrLargeOverflow);
            s_large++;
        } else if (kq == kChildMedW) {
            if (s_medw < w.mmax) {
                w.medw[out][s_medw] = Seg{start[q], size[q], cdepth[q], 0u};
                e_med += size[q];
            } else {
                atomicOr(&h->err, kErrMedOverflow);
            }
            s_medw++;
        }
        // base-case buckets by floor(log2(size))
        const int bin = (kq == kChildTiny || kq == kChildSmall) ? min(31 - __clz(size[q]), 7) : 0;
#pragma unroll
        for (int b = 1; b < 8; b++) hist[b] += bin == b ? 1u : 0u;
    }
    warp_add(&h->tiny_elems, e_tiny);
    warp_add(&h->small_elems, e_small);
    warp_add(&h->med_elems, e_med);
#pragma unroll
    for (int b = 1; b < 8; b++) {
        const uint32_t c = __reduce_add_sync(FULL_MASK, hist[b]);
        if (lane == 0u && c) atomicAdd(&h->small_hist[b], c);
    }
}

// One bucket a lane (valid: the lane has one).
__device__ __forceinline__ void append_children(const Work& w, const Params& p, int out, bool valid, uint32_t start,
                                                uint32_t size, uint32_t cdepth, bool isrun, uint32_t runlcp) {
    const uint32_t kind[1] = {valid ? child_kind(p, size, isrun) : kChildNone};
    const uint32_t st[1] = {start}, sz[1] = {size}, cd[1] = {cdepth}, rl[1] = {runlcp};
    append_children_n<1>(w, out, kind, st, sz, cd, rl);
}

// Child depth of bucket b of a segment at depth `depth` (Eq. (1), Sec. 3.1):
// b_0 and b_2v keep it, the equality bucket of x_i adds w (8, or 16 for wide
// keys; or is a run of equal strings when x_i holds the terminator), an inner
// even bucket adds lcp(x_{i-1}, x_i).
struct BucketInfo {
    uint32_t cdepth, runlcp;
    bool isrun;
};

template <class KT>
__device__ __forceinline__ BucketInfo bucket_info(uint32_t b, uint32_t nb, uint32_t depth, const KT* ino,
                                                  uint32_t size, uint32_t base_threshold) {
    BucketInfo bi{depth, 0u, false};
    if (b & 1u) {
        const KT x = ino[b >> 1];
        if (kends(x)) { bi.isrun = true; bi.runlcp = depth + kchars(x); }
        else bi.cdepth = depth + KeyTraits<KT>::kBytes;
    } else if (b != 0 && b != nb - 1 && size > base_threshold) {
        // an inner even bucket that goes to the base case keeps the parent's
        // depth: its cached keys at that depth still hold the characters
        // after the shared lcp(x_{i-1}, x_i), so it needs no new gather
        const uint32_t i = b >> 1;
        bi.cdepth = depth + klcp(ino[i - 1], ino[i]);
    }
    return bi;
}

// Child depth of bucket b of a radix segment: the outer buckets (keys
// outside the sample's shared leading bits) keep the depth; the strings of
// digit bucket b share the first (rskip + rbits) / 8 whole bytes of their
// key word, and when those bytes hold a zero the strings all end there and
// are equal (a finished run).  A bucket bound for the base case keeps the
// depth, as inner tree buckets do.
__device__ __forceinline__ BucketInfo bucket_info_radix(uint32_t b, uint32_t nb, const SegPlan& P, uint32_t size,
                                                        uint32_t base_threshold) {
    BucketInfo bi{P.depth, 0u, false};
    if (b == 0 || b + 1 == nb) return bi;
    const uint32_t shared = P.rskip + P.rbits;  // <= 64
    const uint64_t pw = P.rbase | ((uint64_t)(b - 1u) << (64u - shared));
    const uint32_t nbytes = shared >> 3;
    for (uint32_t j = 0; j < nbytes; j++) {
        if (((pw >> (56u - 8u * j)) & 0xFFu) == 0u) {
            bi.isrun = true;
            bi.runlcp = P.depth + j;
            return bi;
        }
    }
    if (size > base_threshold) bi.cdepth = P.depth + nbytes;
    return bi;
}

// What the scatter does with a string of the bucket: finish it (single),
// copy its key word, or gather the word at the child's depth.
__device__ __forceinline__ uint32_t refill_code(const BucketInfo& bi, uint32_t size, uint32_t depth) {
    return size == 1 ? kSingle : ((size == 0 || bi.isrun || bi.cdepth == depth) ? kNoRefill : bi.cdepth);
}

// ------------------------------------------------------------ init

__global__ void k_init(Work w) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < w.n; i += stride) {
        const uint64_t o = w.offsets[i];
        Rec r;
        load_key2(w.chars, o, r.key, r.key2);
        r.off = o | kK2Valid;
        r.idx = i;
        r.pad = 0;
        store_rec(&w.rec[0][i], r);
        w.out_lcp[i] = 0u;
    }
}

__global__ void k_hdr_reset(Work w) {
    Hdr* h = w.hdr;
    h->n_large = 0; h->n_med = 0; h->n_small = 0; h->n_bigrun = 0; h->err = 0;
    h->small_elems = 0; h->med_elems = 0; h->n_tiny = 0; h->tiny_elems = 0;
    h->refills = 0ull;
    h->med_refills = 0ull;
    h->base_iters = 0ull;
    h->learned_keys = 0ull;
    h->learned_misses = 0ull;
    h->learned_models = 0;
    h->radix_segments = 0;
    h->round = 0;
    h->q_sample = 0; h->q_fit = 0; h->q_classify = 0; h->q_scatter = 0;
    h->q_med = 0; h->q_base = 0; h->q_bigrun = 0;
    h->n_medw = 0; h->q_medw = 0;
    for (int i = 0; i < 8; i++) h->small_hist[i] = 0;
    // the scan's completion counter (the last entry of its scratch)
    w.scan_tmp[w.scan_tmp_max - 1u] = 0u;
}

// Roots: one segment per set (a single sort is one set) at depth 0.
__global__ void k_roots(Work w, Params p, const Seg* roots, uint32_t num_roots, Seg single) {
    const uint32_t stride = gridDim.x * blockDim.x;
    // the loop runs while any lane of the warp has a root (the appends are
    // made by whole warps)
    for (uint32_t j0 = (blockIdx.x * blockDim.x + threadIdx.x) & ~31u; j0 < num_roots; j0 += stride) {
        const uint32_t j = j0 + (threadIdx.x & 31u);
        const bool ok = j < num_roots;
        const Seg g = ok ? (roots ? roots[j] : single) : Seg{0u, 0u, 0u, 0u};
        if (ok && g.size == 1) w.out_perm[g.begin] = g.begin;
        append_children(w, p, 0, ok, g.begin, g.size, 0u, false, 0u);
    }
}

// ------------------------------------------------------------ plan

// One CTA: layout of the next device-wide round.  The chunk size is chosen so
// that the round has about kChunksPerSM work items per SM.
// advance: 0 plans only; 1 also advances the round counter (the host-driven
// loop); 2 also sets the graph's round-loop condition (the graph form's loop
// body), so that the round's last kernel is this one.
__global__ void __launch_bounds__(1024) k_plan(Work w, Params p, uint32_t advance, cudaGraphConditionalHandle cond) {
    __shared__ uint32_t wsum[33];
    Hdr* h = w.hdr;
    const uint32_t L_all = h->n_large;
    const uint32_t L = min(L_all, w.lmax);
    const uint32_t per = (L + blockDim.x - 1) / blockDim.x;
    const uint32_t lo = min(L, threadIdx.x * per), hi = min(L, lo + per);
    uint32_t sa = 0;
    for (uint32_t s = lo; s < hi; s++) sa += w.large[s].size;
    uint32_t ta;
    block_excl_sum(sa, wsum, &ta);
    const uint32_t target = max(1u, p.num_sms * (uint32_t)kChunksPerSM);
    uint32_t chunk = (uint32_t)(((uint64_t)ta + target - 1) / target);
    chunk = (chunk + kSubTile - 1) / kSubTile * kSubTile;
    chunk = min(max(chunk, kSubTile), p.chunk);
    uint32_t sc = 0, sn = 0, st = 0;
    for (uint32_t s = lo; s < hi; s++) {
        const Seg g = w.large[s];
        const int k = choose_k(g.size, p.k_max);
        const uint32_t ch = (g.size + chunk - 1) / chunk;
        sc += ch;
        sn += ((2u << k) - 1u) * ch;
        st += 1u << k;
    }
    uint32_t tc, tn, tt;
    uint32_t bc = block_excl_sum(sc, wsum, &tc);
    uint32_t bn = block_excl_sum(sn, wsum, &tn);
    uint32_t bt = block_excl_sum(st, wsum, &tt);
    const bool ok = tc <= w.chmax && tn <= w.cmax && tt <= w.tmax && L_all <= w.lmax;
    if (ok) {
        for (uint32_t s = lo; s < hi; s++) {
            const Seg g = w.large[s];
            const int k = choose_k(g.size, p.k_max);
            const uint32_t ch = (g.size + chunk - 1) / chunk;
            w.plans[s] = SegPlan{g.begin, g.size, g.depth, (uint32_t)k, ch, bc, bn, bt, chunk, (uint32_t)k, 0u, 0u, 0ull};
            for (uint32_t c = 0; c < ch; c++) w.chunk_seg[bc + c] = s;
            bc += ch;
            bn += ((2u << k) - 1u) * ch;
            bt += 1u << k;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (!ok) atomicOr(&h->err, kErrPlanOverflow);
        h->L = ok ? L : 0u;
        h->total_chunks = ok ? tc : 0u;
        h->total_counts = ok ? tn : 0u;
        h->total_tree = ok ? tt : 0u;
        h->chunk = chunk;
        h->large_elems_snap = ok ? ta : 0u;
        h->n_med_snap = min(h->n_med, w.mmax);
        h->n_medw_snap = min(h->n_medw, w.mmax);
        h->n_medw = 0;
        h->q_medw = 0;
        h->med_elems_snap = h->med_elems;
        h->n_small_snap = h->n_small;
        h->n_tiny_snap = h->n_tiny;
        h->tiny_elems_snap = h->tiny_elems;
        h->n_tiny = 0;
        h->tiny_elems = 0;
        h->n_bigrun_snap = h->n_bigrun;
        h->small_elems_snap = h->small_elems;
        h->n_large = 0;
        h->n_med = 0;
        h->n_small = 0;
        h->n_bigrun = 0;
        h->small_elems = 0;
        h->med_elems = 0;
        h->q_sample = 0; h->q_fit = 0; h->q_classify = 0; h->q_scatter = 0;
        h->q_med = 0; h->q_base = 0; h->q_bigrun = 0;
        if (advance) {
            h->round += 1u;
            if (advance == 2u)
                cudaGraphSetConditional(cond, (h->L > 0u || h->n_med_snap > 0u || h->n_medw_snap > 0u) ? 1u : 0u);
        }
    }
}

// ------------------------------------------------------------ sample + tree

// Ascending bitonic sort of s[0..pw) (pw a power of two) by the whole block.
template <class KT>
__device__ void bitonic_sort(KT* s, uint32_t pw) {
    for (uint32_t size = 2; size <= pw; size <<= 1) {
        for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
            for (uint32_t i = threadIdx.x; i < pw / 2; i += blockDim.x) {
                uint32_t lo = 2u * i - (i & (stride - 1u));
                uint32_t hi = lo + stride;
                bool asc = (lo & size) == 0;
                const KT a = s[lo], b = s[hi];
                if (kgt(a, b) == asc) { s[lo] = b; s[hi] = a; }
            }
            __syncthreads();
        }
    }
}

template <class KT> __device__ __forceinline__ KT shfl_xor_key(const KT& x, int m);
template <> __device__ __forceinline__ uint64_t shfl_xor_key<uint64_t>(const uint64_t& x, int m) {
    return __shfl_xor_sync(FULL_MASK, x, m);
}
template <> __device__ __forceinline__ Key16 shfl_xor_key<Key16>(const Key16& x, int m) {
    return Key16{__shfl_xor_sync(FULL_MASK, x.h, m), __shfl_xor_sync(FULL_MASK, x.l, m)};
}

// One compare-exchange of the bitonic network seen from element i holding x,
// whose partner i ^ stride holds y: the lower element of an ascending pair
// (and the upper of a descending one) keeps the smaller key.
template <class KT>
__device__ __forceinline__ KT bitonic_keep(const KT& x, const KT& y, uint32_t i, uint32_t stride, uint32_t size) {
    const bool keep_min = ((i & stride) == 0u) == ((i & size) == 0u);
    return kgt(x, y) == keep_min ? y : x;
}

// The same ascending bitonic network as bitonic_sort over n2 = max(pw, 64)
// keys, two a thread: element 2t + r is x[r] of thread t (threads with
// 2t >= n2 idle; keys past the caller's own are top).  Stride 1 is exchanged
// within the thread, strides 2..32 by warp shuffles, and only the strides
// of 64 and more through s, so that most of the network's stages need
// neither shared memory nor a barrier.  Leaves s[0..pw) sorted; called by
// the whole block, ends with __syncthreads.
template <class KT>
__device__ void bitonic_sort_regs(KT* s, KT x0, KT x1, uint32_t pw) {
    const uint32_t n2 = max(pw, 64u);
    const uint32_t i0 = 2u * threadIdx.x, i1 = i0 + 1u;
    const bool act = i0 < n2;  // whole warps: n2 is a multiple of 64
    for (uint32_t size = 2; size <= n2; size <<= 1) {
        for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
            if (stride >= 64u) {
                if (act) { s[i0] = x0; s[i1] = x1; }
                __syncthreads();
                if (act) {
                    const KT y0 = s[i0 ^ stride], y1 = s[i1 ^ stride];
                    x0 = bitonic_keep(x0, y0, i0, stride, size);
                    x1 = bitonic_keep(x1, y1, i1, stride, size);
                }
                __syncthreads();
            } else if (act) {
                if (stride >= 2u) {
                    const KT y0 = shfl_xor_key(x0, (int)(stride >> 1)), y1 = shfl_xor_key(x1, (int)(stride >> 1));
                    x0 = bitonic_keep(x0, y0, i0, stride, size);
                    x1 = bitonic_keep(x1, y1, i1, stride, size);
                } else if (kgt(x0, x1) == ((i0 & size) == 0u)) {
                    const KT y = x0;
                    x0 = x1;
                    x1 = y;
                }
            }
        }
    }
    if (i0 < pw) { s[i0] = x0; s[i1] = x1; }
    __syncthreads();
}

// Runs of equal keys in the sorted sample s[0..cnt): lo[i] is the first
// index of the run holding s[i] and hi[i] one past its last, i.e. the lower
// and upper bound of s[i] in s.  Thread t takes indices PER t .. PER t +
// PER - 1; a prefix maximum over the run heads and a suffix minimum over the
// run tails (within the thread, by warp shuffles, then over the warps'
// totals in wtmp[2 * warps]) give them for every index in one pass, where a
// binary search per tree node would read the sample at data-dependent
// indices.  Needs PER * blockDim.x >= cnt; called by the whole block, ends
// with __syncthreads.
template <int PER, class KT>
__device__ void equal_runs(const KT* s, uint32_t cnt, uint16_t* lo, uint16_t* hi, uint32_t* wtmp) {
    constexpr uint32_t kInf = 0xFFFFu;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const uint32_t base = PER * threadIdx.x;
    // a[j]: index of the latest run head at or before base + j; b[j]: one
    // past the earliest run tail at or after it (within this thread)
    uint32_t a[PER], b[PER];
    uint32_t run = 0u;
#pragma unroll
    for (int j = 0; j < PER; j++) {
        const uint32_t i = base + j;
        if (i < cnt && (i == 0u || !keq(s[i - 1u], s[i]))) run = i;
        a[j] = run;
    }
    uint32_t nxt = kInf;
#pragma unroll
    for (int j = PER - 1; j >= 0; j--) {
        const uint32_t i = base + j;
        if (i < cnt && (i + 1u >= cnt || !keq(s[i], s[i + 1u]))) nxt = i + 1u;
        b[j] = nxt;
    }
    uint32_t pa = a[PER - 1], sb = b[0];  // inclusive scans over the lanes
#pragma unroll
    for (uint32_t o = 1; o < 32u; o <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL_MASK, pa, o);
        const uint32_t z = __shfl_down_sync(FULL_MASK, sb, o);
        if (lane >= o) pa = max(pa, y);
        if (lane + o < 32u) sb = min(sb, z);
    }
    if (lane == 31u) wtmp[warp] = pa;
    if (lane == 0u) wtmp[nw + warp] = sb;
    __syncthreads();
    uint32_t cpre = __shfl_up_sync(FULL_MASK, pa, 1);
    uint32_t csuf = __shfl_down_sync(FULL_MASK, sb, 1);
    if (lane == 0u) cpre = 0u;
    if (lane == 31u) csuf = kInf;
    for (uint32_t v = 0; v < warp; v++) cpre = max(cpre, wtmp[v]);
    for (uint32_t v = warp + 1u; v < nw; v++) csuf = min(csuf, wtmp[nw + v]);
#pragma unroll
    for (int j = 0; j < PER; j++) {
        const uint32_t i = base + j;
        if (i < cnt) {
            lo[i] = (uint16_t)max(cpre, a[j]);
            hi[i] = (uint16_t)min(csuf, b[j]);
        }
    }
    __syncthreads();
}

// Splitter choice of Sec. 3.1 on the sorted sample s[0..cnt): a node owning
// the range a..b takes its middle sample x; its children own a..b' and a'..b
// where b' and a' skip every sample equal to x.  A node whose range is empty
// repeats its parent's splitter.  Level by level, one thread per node.
// lvl[1..v] receives the level-order tree; ra/rb: shared scratch [v+1].
// depth_used (shared, optional): the number of levels holding a node with a
// non-empty range.  Below them every node repeats its parent's splitter, so
// the tree cut to those levels has the same non-empty buckets (the paper's
// "inspect the sample" adaptivity, App. A.2: samples with many equal keys
// get smaller trees).  run_lo/run_hi: for every index i of s, the first
// index of the run of keys equal to s[i] and one past its last (equal_runs).
template <class KT>
__device__ void select_splitters(const KT* s, uint32_t cnt, int k, KT* lvl, int32_t* ra, int32_t* rb,
                                 const uint16_t* run_lo, const uint16_t* run_hi, int* depth_used = nullptr) {
    const uint32_t v = (1u << k) - 1u;
    if (threadIdx.x == 0) {
        ra[1] = 0;
        rb[1] = (int32_t)cnt - 1;
        if (depth_used) *depth_used = 0;
    }
    __syncthreads();
    for (int l = 0; l < k; l++) {
        const uint32_t first = 1u << l;
        for (uint32_t i = first + threadIdx.x; i < 2u * first; i += blockDim.x) {
            int32_t a = ra[i], b = rb[i];
            KT x;
            int32_t bl, ar;
            if (a <= b) {
                if (depth_used) atomicMax(depth_used, l + 1);
                int32_t m = a + (b - a) / 2;
                x = s[m];
                const int32_t first_eq = (int32_t)run_lo[m];  // the run of samples equal to x
                const int32_t past_eq = (int32_t)run_hi[m];
                bl = max(a, first_eq) - 1;
                ar = min(b + 1, past_eq);
            } else {
                x = lvl[i >> 1];
                bl = a - 1;
                ar = b + 1;
            }
            lvl[i] = x;
            if (2u * i <= v) {
                ra[2 * i] = a; rb[2 * i] = bl;
                ra[2 * i + 1] = ar; rb[2 * i + 1] = b;
            }
        }
        __syncthreads();
    }
}

// Writes the tree lvl[1..v] to out_lvl[0..v) and its in-order sequence to
// out_ino[0..v).  Ends with __syncthreads.
template <class KT>
__device__ void emit_tree(const KT* lvl, int k, KT* out_lvl, KT* out_ino) {
    const uint32_t v = (1u << k) - 1u;
    for (uint32_t i = 1 + threadIdx.x; i <= v; i += blockDim.x) {
        uint32_t l = 31u - __clz(i);
        uint32_t q = i - (1u << l);
        uint32_t pos = (2u * q + 1u) * (1u << (k - 1 - (int)l)) - 1u;
        out_lvl[i - 1] = lvl[i];
        out_ino[pos] = lvl[i];
    }
    __syncthreads();
}

// emit_tree into a shared-memory level-order tree (node i at t[i]).
template <class KT, int N>
__device__ void emit_tree_smem(const KT* lvl, int k, LevelTree<KT, N>& t, KT* out_ino) {
    const uint32_t v = (1u << k) - 1u;
    for (uint32_t i = 1 + threadIdx.x; i <= v; i += blockDim.x) {
        uint32_t l = 31u - __clz(i);
        uint32_t q = i - (1u << l);
        uint32_t pos = (2u * q + 1u) * (1u << (k - 1 - (int)l)) - 1u;
        t.set(i, lvl[i]);
        out_ino[pos] = lvl[i];
    }
    __syncthreads();
}

// Pseudo-random sample position j of a segment (Sec. 3.1: the sample is drawn
// pseudo-randomly).
__device__ __forceinline__ uint32_t sample_pos(uint64_t seed, uint32_t begin, uint32_t size, uint32_t j) {
    const uint64_t base = seed ^ ((uint64_t)begin * 0x9E3779B97F4A7C15ull) ^ ((uint64_t)size << 32);
    const uint32_t r = (uint32_t)(mix64(base + (uint64_t)j * 0xD1B54A32D192ED03ull) >> 32);
    return (uint32_t)(((uint64_t)r * size) >> 32);
}

template <class KT>
struct SampleSmem {
    KT samp[kSampleMax];
    KT lvl[kVMax + 1];
    int32_t ra[kVMax + 1], rb[kVMax + 1];
    uint16_t run_lo[kSampleMax], run_hi[kSampleMax];  // equal_runs of samp
    uint32_t wtmp[64];
};

// Radix or tree for a segment (App. A.2: "inspect the sample" and switch
// to radix-style classification where the sample shows it pays).  The
// sorted sample's keys share their first `skip` bits; the digit is the next
// `bits` = min(k, 64 - skip) bits of the first key word.  With option
// radix = 1 the segment takes a digit of at least 4 bits when the sample
// digits' entropy is at least bits - 1 (near uniform, so the digit buckets
// are about as even as the tree's), with radix = 2 whenever the sample keys
// differ.  The
// smallest and largest sample key always fall into different digit
// buckets, so a radix round always splits its segment.  Called by the whole
// block after emit_tree; hist: shared scratch of 2^k ints.
template <class KT>
__device__ void choose_radix(const Work& w, const Params& p, uint32_t seg, const KT* samp, uint32_t cnt, uint32_t k,
                             int32_t* hist, float* s_ent) {
    // the 2^bits + 2 radix buckets must fit the 2^(k+1) - 1 count rows planned
    if (k < 2u) return;
    const uint64_t lo = KeyTraits<KT>::word(samp[0]), hi = KeyTraits<KT>::word(samp[cnt - 1]);
    if (lo == hi) return;
    const uint32_t skip = (uint32_t)__clzll((long long)(lo ^ hi));
    const uint32_t bits = min(k, 64u - skip);
    bool take = p.radix == 2u;
    if (!take && bits >= 4u) {  // shorter digits split too little to choose them over a tree
        const uint32_t nd = 1u << bits;
        for (uint32_t d = threadIdx.x; d < nd; d += blockDim.x) hist[d] = 0;
        if (threadIdx.x == 0) *s_ent = 0.0f;
        __syncthreads();
        for (uint32_t j = threadIdx.x; j < cnt; j += blockDim.x)
            atomicAdd(&hist[(uint32_t)((KeyTraits<KT>::word(samp[j]) << skip) >> (64u - bits))], 1);
        __syncthreads();
        float e = 0.0f;  // sum of c log2 c over the digits
        for (uint32_t d = threadIdx.x; d < nd; d += blockDim.x) {
            const float c = (float)hist[d];
            if (c > 1.0f) e += c * log2f(c);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(FULL_MASK, e, o);
        if ((threadIdx.x & 31u) == 0) atomicAdd(s_ent, e);
        __syncthreads();
        const float H = log2f((float)cnt) - *s_ent / (float)cnt;  // entropy of the digits in bits
        take = H >= (float)bits - 1.0f;
        __syncthreads();  // hist and s_ent are reused
    }
    if (take && threadIdx.x == 0) {
        atomicAdd(&w.hdr->radix_segments, 1u);
        w.plans[seg].rbits = bits;
        w.plans[seg].rskip = skip;
        w.plans[seg].rbase = skip ? (lo >> (64u - skip)) << (64u - skip) : 0ull;
    }
}

// The key of the string at byte offset o at depth 0, read from the strings.
template <class KT> __device__ __forceinline__ KT key_at(const uint8_t* chars, uint64_t o);
template <> __device__ __forceinline__ uint64_t key_at<uint64_t>(const uint8_t* chars, uint64_t o) {
    return load_key(chars, o);
}
template <> __device__ __forceinline__ Key16 key_at<Key16>(const uint8_t* chars, uint64_t o) {
    Key16 x;
    load_key2(chars, o, x.h, x.l);
    return x;
}

// from_strings = 1: round 0 of a fused sort (p.fuse_root), launched before
// the records exist: the sample keys come from the strings themselves.  The
// round body's own launch in that round returns at once.
template <class KT>
__global__ void __launch_bounds__(1024, 2) k_sample(Work w, Params p, int from_strings) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SampleSmem<KT>& sm = *reinterpret_cast<SampleSmem<KT>*>(smem_raw);
    __shared__ uint32_t s_item;
    __shared__ int s_depth;
    __shared__ float s_ent;
    const bool fused0 = p.fuse_root && w.hdr->round == 0u;
    if (fused0 != (from_strings != 0)) return;
    const Rec* recs = w.rec[w.hdr->round & 1u];
    const uint32_t L = w.hdr->L;
    KT* tree_lvl = reinterpret_cast<KT*>(w.tree_lvl);
    KT* tree_ino = reinterpret_cast<KT*>(w.tree_ino);
    for (uint32_t seg = first_item(); seg < L; seg = next_item(&w.hdr->q_sample, &s_item)) {
        const SegPlan P = w.plans[seg];
        const int k = (int)P.kp;
        const uint32_t pw = 2u << k;
        const uint32_t cnt = pw - 1u;  // alpha (v + 1) - 1 with alpha = 2
        // sample keys 2t and 2t + 1 go to thread t (top past the sample)
        KT x[2];
#pragma unroll
        for (int r = 0; r < 2; r++) {
            const uint32_t j = 2u * threadIdx.x + r;
            x[r] = KeyTraits<KT>::top();
            if (j < cnt) {
                const uint32_t e = P.begin + sample_pos(p.seed, P.begin, P.size, j);
                x[r] = from_strings ? key_at<KT>(w.chars, w.offsets[e]) : KeyTraits<KT>::load(recs + e);
            }
        }
        bitonic_sort_regs(sm.samp, x[0], x[1], pw);
        equal_runs<2>(sm.samp, cnt, sm.run_lo, sm.run_hi, sm.wtmp);
        select_splitters(sm.samp, cnt, k, sm.lvl, sm.ra, sm.rb, sm.run_lo, sm.run_hi, &s_depth);
        const int kt = max(1, s_depth);
        if (threadIdx.x == 0 && kt != k) w.plans[seg].k = (uint32_t)kt;
        emit_tree(sm.lvl, kt, tree_lvl + P.tree_base, tree_ino + P.tree_base);
        if (p.radix && !p.learned) choose_radix<KT>(w, p, seg, sm.samp, cnt, (uint32_t)k, sm.ra, &s_ent);
    }
}

// Stand-alone splitter construction for a caller's sample (sss_build_splitters),
// by the same steps as k_sample: register bitonic sort, runs of equal keys,
// splitter choice.
__global__ void __launch_bounds__(1024) k_build_splitters(const uint64_t* sample, uint32_t count, int k,
                                                          uint64_t* out_lvl, uint64_t* out_ino) {
    __shared__ uint64_t samp[kSampleMax];
    __shared__ uint64_t lvl[kVMax + 1];
    __shared__ int32_t ra[kVMax + 1], rb[kVMax + 1];
    __shared__ uint16_t run_lo[kSampleMax], run_hi[kSampleMax];
    __shared__ uint32_t wtmp[64];
    uint32_t pw = 2;
    while (pw < count) pw <<= 1;
    const uint32_t i0 = 2u * threadIdx.x;
    const uint64_t x0 = i0 < count ? sample[i0] : ~0ull;
    const uint64_t x1 = i0 + 1u < count ? sample[i0 + 1u] : ~0ull;
    bitonic_sort_regs(samp, x0, x1, pw);
    equal_runs<2>(samp, count, run_lo, run_hi, wtmp);
    select_splitters(samp, count, k, lvl, ra, rb, run_lo, run_hi);
    emit_tree(lvl, k, out_lvl, out_ino);
}

// ------------------------------------------------------------ classify + count

constexpr int kClassifyThreads = 256;
#ifndef SSS_CLASSIFY_UNROLL
#define SSS_CLASSIFY_UNROLL 4
#endif
#ifndef SSS_CLASSIFY_MIN_BLOCKS
#define SSS_CLASSIFY_MIN_BLOCKS 5
#endif
constexpr int kClassifyUnroll = SSS_CLASSIFY_UNROLL;  // keys a thread descends at once

// Adds the buckets of the key words of recs[lo, hi) to hist (warp-aggregated shared atomics);
// bid (optional) receives each bucket at bid[e - lo].  Loop bounds are
// uniform over the block.
template <class KT, class TT>
__device__ __forceinline__ void classify_range(const Rec* __restrict__ recs, uint32_t lo, uint32_t hi, const TT& t,
                                               const KT* ino, int k, uint32_t nb, uint32_t* hist, uint16_t* bid,
                                               bool equal_test) {
    const uint32_t lane = threadIdx.x & 31u;
    for (uint32_t base = lo; base < hi; base += blockDim.x * kClassifyUnroll) {
        KT kk[kClassifyUnroll];
#pragma unroll
        for (int u = 0; u < kClassifyUnroll; u++) {
            const uint32_t e = base + u * blockDim.x + threadIdx.x;
            kk[u] = e < hi ? KeyTraits<KT>::load(recs + e) : KeyTraits<KT>::top();
        }
        uint32_t bk[kClassifyUnroll];
        classify_keys_by<kClassifyUnroll>(equal_test, kk, bk, t, ino, k);
#pragma unroll
        for (int u = 0; u < kClassifyUnroll; u++) {
            const uint32_t e = base + u * blockDim.x + threadIdx.x;
            const uint32_t b = e < hi ? bk[u] : nb;
            if (bid && e < hi) bid[e - lo] = (uint16_t)b;
            const uint32_t peers = __match_any_sync(FULL_MASK, b);
            if (lane == (uint32_t)(__ffs(peers) - 1)) atomicAdd(&hist[b], (uint32_t)__popc(peers));
        }
    }
}

// Radix form of classify_range: the bucket of a key is its digit
// (radix_bucket), no tree.
__device__ __forceinline__ void classify_range_radix(const Rec* __restrict__ recs, uint32_t lo, uint32_t hi,
                                                     uint32_t rskip, uint32_t rbits, uint64_t rbase, uint32_t nb,
                                                     uint32_t* hist, uint16_t* bid) {
    const uint32_t lane = threadIdx.x & 31u;
    for (uint32_t base = lo; base < hi; base += blockDim.x * kClassifyUnroll) {
        uint64_t kk[kClassifyUnroll];
#pragma unroll
        for (int u = 0; u < kClassifyUnroll; u++) {
            const uint32_t e = base + u * blockDim.x + threadIdx.x;
            kk[u] = e < hi ? recs[e].key : 0ull;
        }
#pragma unroll
        for (int u = 0; u < kClassifyUnroll; u++) {
            const uint32_t e = base + u * blockDim.x + threadIdx.x;
            const uint32_t b = e < hi ? radix_bucket(kk[u], rskip, rbits, rbase) : nb;
            if (e < hi) bid[e - lo] = (uint16_t)b;
            const uint32_t peers = __match_any_sync(FULL_MASK, b);
            if (lane == (uint32_t)(__ffs(peers) - 1)) atomicAdd(&hist[b], (uint32_t)__popc(peers));
        }
    }
}

// Learned form of classify_range: propose + verify, tree on a miss; counts
// proposals and misses.
__device__ __forceinline__ void classify_range_learned(const Rec* __restrict__ recs, uint32_t lo, uint32_t hi,
                                                       const uint64_t* t, const uint64_t* ino, int k, uint32_t nb,
                                                       uint32_t* hist, const float* C, uint32_t M, const CdfNorm& nrm,
                                                       uint32_t& misses, uint16_t* bid) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t v = (1u << k) - 1u;
    for (uint32_t base = lo; base < hi; base += blockDim.x * kClassifyUnroll) {
        uint64_t kk[kClassifyUnroll];
#pragma unroll
        for (int u = 0; u < kClassifyUnroll; u++) {
            const uint32_t e = base + u * blockDim.x + threadIdx.x;
            kk[u] = e < hi ? recs[e].key : 0ull;
        }
#pragma unroll
        for (int u = 0; u < kClassifyUnroll; u++) {
            const uint32_t e = base + u * blockDim.x + threadIdx.x;
            uint32_t b = nb;
            if (e < hi && !propose_bucket(kk[u], C, M, nrm, ino, v, b)) {
                b = classify_key(kk[u], t, ino, k);
                misses++;
            }
            if (e < hi) bid[e - lo] = (uint16_t)b;
            const uint32_t peers = __match_any_sync(FULL_MASK, b);
            if (lane == (uint32_t)(__ffs(peers) - 1)) atomicAdd(&hist[b], (uint32_t)__popc(peers));
        }
    }
}

constexpr uint32_t kCdfMMax = 4096;

template <class KT>
__global__ void __launch_bounds__(kClassifyThreads, SSS_CLASSIFY_MIN_BLOCKS) k_classify(Work w, Params p) {
    constexpr bool kLearned = KeyTraits<KT>::kBytes == 8;  // the learned model proposes on one word
    __shared__ LevelTree<KT, kVMax + 1> t;
    __shared__ KT ino[kVMax];
    __shared__ uint32_t hist[kNBMax + 1];
    __shared__ float C[kLearned ? kCdfMMax + 1 : 1];
    // the learned model's input coordinate (a byte where it is not used)
    __shared__ typename std::conditional<kLearned, CdfNorm, char>::type nrm_s;
    __shared__ uint32_t s_item;
    const int cur = w.hdr->round & 1u;
    if (p.fuse_root && cur == 0 && w.hdr->round == 0u) return;  // classified while the records were built
    const uint32_t total_chunks = w.hdr->total_chunks;
    const KT* tree_lvl = reinterpret_cast<const KT*>(w.tree_lvl);
    const KT* tree_ino = reinterpret_cast<const KT*>(w.tree_ino);
    for (uint32_t c = first_item(); c < total_chunks;
         c = next_item(&w.hdr->q_classify, &s_item)) {
        const uint32_t s = w.chunk_seg[c];
        const SegPlan P = w.plans[s];
        const uint32_t ci = c - P.chunk_base;
        const int k = (int)P.k;
        const uint32_t v = (1u << k) - 1u;
        const uint32_t nb = P.rbits ? radix_buckets(P.rbits) : 2u * v + 1u;
        if (!P.rbits) {
            for (uint32_t i = threadIdx.x; i < v; i += blockDim.x) {
                t.set(i + 1, tree_lvl[P.tree_base + i]);
                ino[i] = tree_ino[P.tree_base + i];
            }
        }
        for (uint32_t b = threadIdx.x; b <= nb; b += blockDim.x) hist[b] = 0;
        __syncthreads();
        const uint32_t lo = P.begin + ci * P.chunk;
        const uint32_t hi = min(lo + P.chunk, P.begin + P.size);
        if (P.rbits) {
            classify_range_radix(w.rec[cur], lo, hi, P.rskip, P.rbits, P.rbase, nb, hist, w.bids + lo);
        } else if constexpr (kLearned) {
            if (p.learned && P.size >= kLearnedMinSize) {
                const float* tab = w.cdf_tab + (size_t)s * (p.cdf_M + 1);
                for (uint32_t j = threadIdx.x; j <= p.cdf_M; j += blockDim.x) C[j] = tab[j];
                {
                    const uint32_t* src = reinterpret_cast<const uint32_t*>(w.cdf_norm + s);
                    uint32_t* dst = reinterpret_cast<uint32_t*>(&nrm_s);
                    for (uint32_t j = threadIdx.x; j < sizeof(CdfNorm) / 4; j += blockDim.x) dst[j] = src[j];
                }
                __syncthreads();
                uint32_t misses = 0;
                classify_range_learned(w.rec[cur], lo, hi, t.view(), ino, k, nb, hist, C, p.cdf_M, nrm_s, misses,
                                       w.bids + lo);
                misses = __reduce_add_sync(FULL_MASK, misses);
                if ((threadIdx.x & 31u) == 0 && misses)
                    atomicAdd(&w.hdr->learned_misses, (unsigned long long)misses);
                if (threadIdx.x == 0) atomicAdd(&w.hdr->learned_keys, (unsigned long long)(hi - lo));
            } else {
                classify_range(w.rec[cur], lo, hi, t.view(), ino, k, nb, hist, w.bids + lo, p.equal_test != 0);
            }
        } else {
            classify_range(w.rec[cur], lo, hi, t.view(), ino, k, nb, hist, w.bids + lo, p.equal_test != 0);
        }
        __syncthreads();
        // the count rows were planned for 2^(kp+1) - 1 buckets: the rows a
        // smaller tree leaves unused are zero
        const uint32_t nbp = (2u << P.kp) - 1u;
        for (uint32_t b = threadIdx.x; b < nbp; b += blockDim.x)
            w.counts[P.count_base + b * P.chunks + ci] = b < nb ? hist[b] : 0u;
        __syncthreads();
    }
}

// Round 0 of a fused sort: one pass over the root's work chunks builds each
// string's record (its key words at depth 0, as k_init does) and classifies
// the keys while they are in registers, as k_classify does (tree or digit,
// bucket ids, per-chunk histogram): the round's classification needs no
// second read of the records.
// four CTAs per SM: the phased loads of four keys need 64 registers (at
// five CTAs per SM they spill, and the kernel was slower)
#ifndef SSS_INIT_CLASSIFY_MIN_BLOCKS
#define SSS_INIT_CLASSIFY_MIN_BLOCKS 4
#endif
template <class KT>
__global__ void __launch_bounds__(kClassifyThreads, SSS_INIT_CLASSIFY_MIN_BLOCKS) k_init_classify(Work w, Params p) {
    __shared__ LevelTree<KT, kVMax + 1> t;
    __shared__ KT ino[kVMax];
    __shared__ uint32_t hist[kNBMax + 1];
    __shared__ uint32_t s_item;
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t total_chunks = w.hdr->total_chunks;
    const KT* tree_lvl = reinterpret_cast<const KT*>(w.tree_lvl);
    const KT* tree_ino = reinterpret_cast<const KT*>(w.tree_ino);
    Rec* recs = w.rec[0];
    for (uint32_t c = first_item(); c < total_chunks; c = next_item(&w.hdr->q_classify, &s_item)) {
        const uint32_t s = w.chunk_seg[c];
        const SegPlan P = w.plans[s];
        const uint32_t ci = c - P.chunk_base;
        const int k = (int)P.k;
        const uint32_t v = (1u << k) - 1u;
        const uint32_t nb = P.rbits ? radix_buckets(P.rbits) : 2u * v + 1u;
        if (!P.rbits) {
            for (uint32_t i = threadIdx.x; i < v; i += blockDim.x) {
                t.set(i + 1, tree_lvl[P.tree_base + i]);
                ino[i] = tree_ino[P.tree_base + i];
            }
        }
        for (uint32_t b = threadIdx.x; b <= nb; b += blockDim.x) hist[b] = 0;
        __syncthreads();
        const uint32_t lo = P.begin + ci * P.chunk;
        const uint32_t hi = min(lo + P.chunk, P.begin + P.size);
        for (uint32_t base = lo; base < hi; base += blockDim.x * kClassifyUnroll) {
            // three phases, so that every load of the unrolled keys is in
            // flight before the first store: offsets, key words, records
            uint64_t o[kClassifyUnroll], k1[kClassifyUnroll], k2[kClassifyUnroll];
#pragma unroll
            for (int u = 0; u < kClassifyUnroll; u++) {
                const uint32_t e = base + u * blockDim.x + threadIdx.x;
                o[u] = e < hi ? __ldg(w.offsets + e) : 0ull;
            }
#pragma unroll
            for (int u = 0; u < kClassifyUnroll; u++) {
                const uint32_t e = base + u * blockDim.x + threadIdx.x;
                k1[u] = k2[u] = 0ull;
                if (e < hi) load_key2(w.chars, o[u], k1[u], k2[u]);
            }
            KT kk[kClassifyUnroll];
#pragma unroll
            for (int u = 0; u < kClassifyUnroll; u++) {
                const uint32_t e = base + u * blockDim.x + threadIdx.x;
                kk[u] = KeyTraits<KT>::top();
                if (e < hi) {
                    Rec r;
                    r.key = k1[u];
                    r.key2 = k2[u];
                    r.off = o[u] | kK2Valid;
                    r.idx = e;
                    r.pad = 0;
                    store_rec(recs + e, r);
                    w.out_lcp[e] = 0u;
                    kk[u] = KeyTraits<KT>::of(r);
                }
            }
            uint32_t bk[kClassifyUnroll];
            if (P.rbits) {
#pragma unroll
                for (int u = 0; u < kClassifyUnroll; u++)
                    bk[u] = radix_bucket(KeyTraits<KT>::word(kk[u]), P.rskip, P.rbits, P.rbase);
            } else {
                classify_keys_by<kClassifyUnroll>(p.equal_test != 0, kk, bk, t.view(), ino, k);
            }
#pragma unroll
            for (int u = 0; u < kClassifyUnroll; u++) {
                const uint32_t e = base + u * blockDim.x + threadIdx.x;
                const uint32_t b = e < hi ? bk[u] : nb;
                if (e < hi) w.bids[e] = (uint16_t)b;
                const uint32_t peers = __match_any_sync(FULL_MASK, b);
                if (lane == (uint32_t)(__ffs(peers) - 1)) atomicAdd(&hist[b], (uint32_t)__popc(peers));
            }
        }
        __syncthreads();
        const uint32_t nbp = (2u << P.kp) - 1u;
        for (uint32_t b = threadIdx.x; b < nbp; b += blockDim.x)
            w.counts[P.count_base + b * P.chunks + ci] = b < nb ? hist[b] : 0u;
        __syncthreads();
    }
}

// ------------------------------------------------------------ stable scatter

constexpr int kScatterWarps = kScatterThreads / 32;
#ifndef SSS_SCATTER_MIN_BLOCKS
#define SSS_SCATTER_MIN_BLOCKS 4
#endif

template <int NBCAP>
struct ScatterState {
    uint32_t run_pos[NBCAP + 1];  // next output position of each bucket
    uint32_t rdep[NBCAP + 1];     // refill code of each bucket
    uint64_t wcnt[NBCAP + 1];     // strings of each bucket in this sub-tile, one byte per warp
};
static_assert(kScatterWarps == 8, "one byte per warp in ScatterState::wcnt");

// Sum of the bytes of x below byte `below` (0..8).
__device__ __forceinline__ uint32_t byte_sum_below(uint64_t x, uint32_t below) {
    if (below < 8u) x &= below ? (~0ull >> (64u - 8u * below)) : 0ull;
    return __dp4a((uint32_t)x, 0x01010101u, 0u) + __dp4a((uint32_t)(x >> 32), 0x01010101u, 0u);
}

// Stable move of the strings [lo, hi) of one segment (Sec. 3.1: out-of-place
// redistribution into the shadow arrays).  Sub-tiles of 256 * ITEMS strings
// are taken in order; warp w owns 32 * ITEMS consecutive strings of one and
// ranks equal buckets by lane (match + popc), per-warp counters give the
// offset of each warp.  Needs: ss.run_pos/rdep set, ss.wcnt zero (entries
// 0..nb), the tree in t/ino (or bucket ids in bid[e - lo]), 256 threads.
// Returns this thread's number of key words gathered again.
template <int NBCAP, bool kFromBid, class KT, int ITEMS = kScatterItems, class TT>
__device__ uint32_t scatter_range(const Work& w, int cur, uint32_t lo, uint32_t hi, uint32_t nb,
                                  ScatterState<NBCAP>& ss, const TT& t, const KT* ino, int k,
                                  const uint16_t* bid, uint32_t seg_end, uint32_t depth, bool equal_test) {
    constexpr int kBucketsPerThread = (NBCAP + kScatterThreads) / kScatterThreads;
    static_assert(32 * ITEMS <= 255, "per-warp bucket counts must fit a byte");
    uint8_t* wbytes = reinterpret_cast<uint8_t*>(ss.wcnt);
    const Rec* rec_in = w.rec[cur];
    Rec* rec_out = w.rec[cur ^ 1];
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint32_t lt = lanemask_lt();
    uint32_t nref = 0;
    for (uint32_t sub = lo; sub < hi; sub += kScatterThreads * ITEMS) {
        Rec rr[ITEMS];
        uint32_t bb[ITEMS], loc[ITEMS];
        const uint32_t wbase = sub + warp * (32u * ITEMS) + lane;
#pragma unroll
        for (int j = 0; j < ITEMS; j++) {
            const uint32_t e = wbase + j * 32u;
            const bool ok = e < hi;
            if (ok) rr[j] = load_rec(rec_in + e);
            else rr[j] = Rec{0ull, 0ull, 0ull, 0u, 0u};
            if (kFromBid) bb[j] = ok ? bid[e - lo] : nb;
        }
        if constexpr (!kFromBid) {
            KT kk[ITEMS];
#pragma unroll
            for (int j = 0; j < ITEMS; j++) kk[j] = KeyTraits<KT>::of(rr[j]);
            classify_keys_by<ITEMS>(equal_test, kk, bb, t, ino, k);
#pragma unroll
            for (int j = 0; j < ITEMS; j++)
                if (wbase + j * 32u >= hi) bb[j] = nb;
        }
        // next key words of strings whose bucket moves deeper: all gathers are
        // issued here, before any store, and complete during the ranking
#pragma unroll
        for (int j = 0; j < ITEMS; j++) {
            const uint32_t rd = bb[j] < nb ? ss.rdep[bb[j]] : kNoRefill;
            if (rd != kNoRefill && rd != kSingle) {
                refill_rec<KT>(w.chars, rr[j], rd, depth);
                nref++;
            }
        }
#pragma unroll
        for (int j = 0; j < ITEMS; j++) {
            const uint32_t b = bb[j];
            const uint32_t peers = __match_any_sync(FULL_MASK, b);
            const uint32_t leader = (uint32_t)__ffs(peers) - 1u;
            uint32_t off = 0;
            if (lane == leader) {
                off = wbytes[8u * b + warp];
                wbytes[8u * b + warp] = (uint8_t)(off + (uint32_t)__popc(peers));
            }
            off = __shfl_sync(FULL_MASK, off, leader);
            loc[j] = off + (uint32_t)__popc(peers & lt);
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < ITEMS; j++) {
            const uint32_t e = wbase + j * 32u;
            if (e < hi) {
                const uint32_t b = bb[j];
                // the strings of bucket b held by the warps before this one
                const uint32_t pos = ss.run_pos[b] + byte_sum_below(ss.wcnt[b], warp) + loc[j];
                const uint32_t rd = ss.rdep[b];
                if (pos >= seg_end) {
                    atomicOr(&w.hdr->err, kErrPosition);
                } else if (rd == kSingle) {
                    w.out_perm[pos] = rr[j].idx;
                } else {
                    store_rec(rec_out + pos, rr[j]);
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < kBucketsPerThread; q++) {
            const uint32_t b = threadIdx.x + q * kScatterThreads;
            if (b < nb) ss.run_pos[b] += byte_sum_below(ss.wcnt[b], 8u);
            if (b <= nb) ss.wcnt[b] = 0ull;
        }
        __syncthreads();
    }
    return nref;
}

__device__ __forceinline__ void add_refills(unsigned long long* counter, uint32_t nref) {
    nref = __reduce_add_sync(FULL_MASK, nref);
    if ((threadIdx.x & 31u) == 0 && nref) atomicAdd(counter, (unsigned long long)nref);
}

template <class KT>
struct ScatterSmem {
    KT ino[kVMax];
    ScatterState<kNBMax> ss;
};

template <class KT>
__global__ void __launch_bounds__(kScatterThreads, SSS_SCATTER_MIN_BLOCKS) k_scatter(Work w, Params p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ScatterSmem<KT>& sm = *reinterpret_cast<ScatterSmem<KT>*>(smem_raw);
    const KT* tree_ino = reinterpret_cast<const KT*>(w.tree_ino);
    const int cur = w.hdr->round & 1u;
    const int med_out = cur ^ 1;
    const uint32_t total_chunks = w.hdr->total_chunks;
    __shared__ uint32_t s_item;
    for (uint32_t c = first_item(); c < total_chunks;
         c = next_item(&w.hdr->q_scatter, &s_item)) {
        const uint32_t s = w.chunk_seg[c];
        const SegPlan P = w.plans[s];
        const uint32_t ci = c - P.chunk_base;
        const int k = (int)P.k;
        const uint32_t v = (1u << k) - 1u;
        const uint32_t nb = P.rbits ? radix_buckets(P.rbits) : 2u * v + 1u;
        if (!P.rbits)
            for (uint32_t i = threadIdx.x; i < v; i += blockDim.x) sm.ino[i] = tree_ino[P.tree_base + i];
        __syncthreads();
        const uint32_t* S = w.counts_scan + P.count_base;
        const uint32_t seg_end = P.begin + P.size;
        // bucket b starts at S[b * chunks] and this chunk's part of it at
        // S[b * chunks + ci] (relative to S[0]): issue every load first
        constexpr int kBPT = (kNBMax + kScatterThreads) / kScatterThreads;
        uint32_t s_first[kBPT], s_next[kBPT], s_mine[kBPT];
        const uint32_t S0 = S[0];
        const bool last_lane = (threadIdx.x & 31u) == 31u;
#pragma unroll
        for (int q = 0; q < kBPT; q++) {
            const uint32_t b = threadIdx.x + q * kScatterThreads;
            s_first[q] = b < nb ? S[b * P.chunks] : 0u;
            s_mine[q] = b < nb ? S[b * P.chunks + ci] : 0u;
            // the next bucket's start is the next lane's s_first; lane 31 reads it
            s_next[q] = last_lane && b + 1 < nb ? S[(b + 1) * P.chunks] : 0u;
        }
#pragma unroll
        for (int q = 0; q < kBPT; q++) {
            const uint32_t nx = __shfl_down_sync(FULL_MASK, s_first[q], 1);
            if (!last_lane) s_next[q] = nx;
        }
        // child segments of this thread's buckets (chunk 0 appends them):
        // start and size replace s_first and s_next in place
        uint32_t ckind[kBPT], cdep[kBPT], crun[kBPT];
#pragma unroll
        for (int q = 0; q < kBPT; q++) {
            const uint32_t b = threadIdx.x + q * kScatterThreads;
            if (b <= nb) sm.ss.wcnt[b] = 0ull;
            uint32_t start = 0, size = 0;
            BucketInfo bi{0u, 0u, false};
            if (b < nb) {
                start = P.begin + (s_first[q] - S0);
                const uint32_t end = (b + 1 < nb) ? P.begin + (s_next[q] - S0) : seg_end;
                size = end - start;
                sm.ss.run_pos[b] = P.begin + (s_mine[q] - S0);
                bi = P.rbits ? bucket_info_radix(b, nb, P, size, p.base_threshold)
                             : bucket_info(b, nb, P.depth, sm.ino, size, p.base_threshold);
                sm.ss.rdep[b] = refill_code(bi, size, P.depth);
                if (ci == 0 && size > 0 && start > P.begin) w.out_lcp[start] = kLcpFlag | P.depth;
            }
            s_first[q] = start;
            s_next[q] = size;
            ckind[q] = b < nb && size > 0 ? child_kind(p, size, bi.isrun) : kChildNone;
            cdep[q] = bi.cdepth;
            crun[q] = bi.runlcp;
        }
        if (ci == 0) append_children_n<kBPT>(w, med_out, ckind, s_first, s_next, cdep, crun);
        __syncthreads();
        const uint32_t lo = P.begin + ci * P.chunk;
        const uint32_t hi = min(lo + P.chunk, seg_end);
        // buckets as k_classify found them (tree or learned proposal)
        const uint32_t nref = scatter_range<kNBMax, true, KT>(w, cur, lo, hi, nb, sm.ss, (const KT*)sm.ino, sm.ino, k,
                                                          w.bids + lo, seg_end, P.depth, p.equal_test != 0);
        add_refills(&w.hdr->refills, nref);
        __syncthreads();
    }
}

// ------------------------------------------------------------ medium round

template <class KT>
struct MedSmem {
    LevelTree<KT, 1 << kMedKMax> t;
    KT ino[1 << kMedKMax];
    uint32_t hist[kMedNB + 1];
    uint32_t wsum[33];
    uint32_t full;  // a bucket holding the whole segment, or kNoRefill
    union {
        struct {  // splitter choice
            KT samp[1 << (kMedKMax + 1)];
            KT lvl[1 << kMedKMax];
            int32_t ra[1 << kMedKMax], rb[1 << kMedKMax];
            uint16_t run_lo[1 << (kMedKMax + 1)], run_hi[1 << (kMedKMax + 1)];  // equal_runs of samp
        } sel;
        struct {  // classification and move
            uint16_t bid[kMedMax];
            ScatterState<kMedNB> ss;
        } mv;
    };
};

constexpr int kMedItems = 4;  // records per thread in a medium round's move

// One CTA runs one whole distribution round for one medium segment (the
// sequential S^5 of the paper, here on one SM): sample, tree, classify into a
// shared bucket array, local prefix sum, stable move, child segments.  When
// every string lands in the equality bucket of one splitter without the
// terminator (they all share the next w characters), the CTA steps over
// those characters in place (gathers the keys w deeper, same positions) and
// classifies again, instead of moving the whole segment into one child.
#ifndef SSS_MED_MIN_BLOCKS
#define SSS_MED_MIN_BLOCKS 4
#endif
template <class KT>
__global__ void __launch_bounds__(kScatterThreads, SSS_MED_MIN_BLOCKS) k_med_round(Work w, Params p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    MedSmem<KT>& sm = *reinterpret_cast<MedSmem<KT>*>(smem_raw);
    const int cur = w.hdr->round & 1u;
    const int med_in = cur, med_out = cur ^ 1;
    const uint32_t n_med = w.hdr->n_med_snap;
    __shared__ uint32_t s_item;
    __shared__ int s_depth;  // levels the splitters use (select_splitters)
    for (uint32_t mi = first_item(); mi < n_med; mi = next_item(&w.hdr->q_med, &s_item)) {
        Seg g = w.med[med_in][mi];
        const uint32_t m = g.size;
        const int kp = choose_k(m, min(p.k_max, kMedKMax));
        const uint32_t nbp = (2u << kp) - 1u;
        const uint32_t pw = 2u << kp, cnt = pw - 1u;
        int k = kp;          // the tree's levels this pass (cut to the levels its splitters use)
        uint32_t nb = nbp;
        Rec* recs = w.rec[cur];
        for (uint32_t level = 0;; level++) {
            for (uint32_t j = threadIdx.x; j < pw; j += blockDim.x)
                sm.sel.samp[j] = j < cnt ? KeyTraits<KT>::load(recs + g.begin + sample_pos(p.seed, g.begin, m, j))
                                         : KeyTraits<KT>::top();
            for (uint32_t b = threadIdx.x; b <= nbp; b += blockDim.x) sm.hist[b] = 0;
            if (threadIdx.x == 0) sm.full = kNoRefill;
            __syncthreads();
            bitonic_sort(sm.sel.samp, pw);
            equal_runs<(1 << (kMedKMax + 1)) / kScatterThreads>(sm.sel.samp, cnt, sm.sel.run_lo, sm.sel.run_hi,
                                                                sm.wsum);
            select_splitters(sm.sel.samp, cnt, kp, sm.sel.lvl, sm.sel.ra, sm.sel.rb, sm.sel.run_lo, sm.sel.run_hi,
                             &s_depth);
            k = max(1, s_depth);
            nb = (2u << k) - 1u;
            emit_tree_smem(sm.sel.lvl, k, sm.t, sm.ino);
            // the splitter-choice scratch is dead: the move state takes its place
            for (uint32_t b = threadIdx.x; b <= nb; b += blockDim.x) sm.mv.ss.wcnt[b] = 0ull;
            classify_range(recs, g.begin, g.begin + m, sm.t.view(), sm.ino, k, nb, sm.hist, sm.mv.bid,
                           p.equal_test != 0);
            __syncthreads();
            for (uint32_t b = 1u + 2u * threadIdx.x; b < nb; b += 2u * blockDim.x)
                if (sm.hist[b] == m && !kends(sm.ino[b >> 1])) sm.full = b;
            __syncthreads();
            if (sm.full == kNoRefill || level >= kBaseMaxIters) break;
            // all strings share the next w characters: gather their keys w
            // deeper in place and classify again
            uint32_t nref = 0;
            for (uint32_t e = g.begin + threadIdx.x; e < g.begin + m; e += blockDim.x) {
                Rec r = load_rec(recs + e);
                refill_rec<KT>(w.chars, r, g.depth + KeyTraits<KT>::kBytes, g.depth);
                store_rec(recs + e, r);
                nref++;
            }
            add_refills(&w.hdr->med_refills, nref);
            g.depth += KeyTraits<KT>::kBytes;
            __syncthreads();
        }
        // bucket starts: consecutive buckets per thread
        constexpr int kPer = (kMedNB + 1) / kScatterThreads;
        uint32_t cnts[kPer], sum = 0;
#pragma unroll
        for (int q = 0; q < kPer; q++) {
            const uint32_t b = threadIdx.x * kPer + q;
            cnts[q] = b < nb ? sm.hist[b] : 0u;
            sum += cnts[q];
        }
        uint32_t start = g.begin + block_excl_sum(sum, sm.wsum, nullptr);
        uint32_t ckind[kPer], cstart[kPer], cdep[kPer], crun[kPer];
#pragma unroll
        for (int q = 0; q < kPer; q++) {
            const uint32_t b = threadIdx.x * kPer + q;
            const uint32_t size = cnts[q];
            BucketInfo bi{0u, 0u, false};
            if (b < nb) {
                bi = bucket_info(b, nb, g.depth, sm.ino, size, p.base_threshold);
                sm.mv.ss.run_pos[b] = start;
                sm.mv.ss.rdep[b] = refill_code(bi, size, g.depth);
                if (size > 0 && start > g.begin) w.out_lcp[start] = kLcpFlag | g.depth;
            }
            ckind[q] = b < nb && size > 0 ? child_kind(p, size, bi.isrun) : kChildNone;
            cstart[q] = start;
            cdep[q] = bi.cdepth;
            crun[q] = bi.runlcp;
            start += cnts[q];
        }
        append_children_n<kPer>(w, med_out, ckind, cstart, cnts, cdep, crun);
        __syncthreads();
        const uint32_t nref =
            scatter_range<kMedNB, true, KT, kMedItems>(w, cur, g.begin, g.begin + m, nb, sm.mv.ss, sm.t.view(), sm.ino, k,
                                                       sm.mv.bid, g.begin + m, g.depth, p.equal_test != 0);
        add_refills(&w.hdr->med_refills, nref);
        __syncthreads();
    }
}

// ------------------------------------------------------------ medium round, one warp per bucket

// The medium buckets of at most kMedWarpMax strings: one warp runs the
// whole distribution round of a bucket (sample of at most 63 keys, tree of
// at most 31 splitters, classification, bucket starts, child segments,
// stable move), with warp shuffles and __syncwarp instead of block-wide
// barriers, so that the many small buckets of a round overlap their phases
// instead of leaving most of a CTA idle between barriers.
#ifndef SSS_MW_WARPS
#define SSS_MW_WARPS 4
#endif
constexpr int kMWWarps = SSS_MW_WARPS;  // buckets a CTA holds at once

template <class KT>
struct MedWarpSmem {
    KT samp[2 << kMWKMax];                       // the sorted sample (64 keys)
    KT lvl[1 << kMWKMax];                        // splitter choice, level order 1..v
    int32_t ra[1 << kMWKMax], rb[1 << kMWKMax];  // its sample ranges
    uint16_t run_lo[2 << kMWKMax], run_hi[2 << kMWKMax];
    LevelTree<KT, 1 << kMWKMax> t;               // the tree of the descent, level order 1..v
    KT ino[1 << kMWKMax];                        // in-order splitters 0..v-1
    uint32_t hist[kMWNB + 1];                    // bucket sizes (entry kMWNB: no string)
    uint32_t run_pos[kMWNB + 1];                 // next output position of each bucket
    uint32_t rdep[kMWNB + 1];                    // refill code of each bucket
    uint8_t bid[kMedWarpMax + 1];                // bucket of each string of the segment
};

// bitonic_sort_regs for one warp and 64 keys: element 2 lane + r is x[r];
// every stride lies within the warp.  Leaves s[0..64) sorted.
template <class KT>
__device__ __forceinline__ void warp_bitonic64(KT* s, KT x0, KT x1) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t i0 = 2u * lane, i1 = i0 + 1u;
#pragma unroll
    for (uint32_t size = 2; size <= 64u; size <<= 1) {
#pragma unroll
        for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
            if (stride >= 2u) {
                const KT y0 = shfl_xor_key(x0, (int)(stride >> 1)), y1 = shfl_xor_key(x1, (int)(stride >> 1));
                x0 = bitonic_keep(x0, y0, i0, stride, size);
                x1 = bitonic_keep(x1, y1, i1, stride, size);
            } else if (kgt(x0, x1) == ((i0 & size) == 0u)) {
                const KT y = x0;
                x0 = x1;
                x1 = y;
            }
        }
    }
    s[i0] = x0;
    s[i1] = x1;
    __syncwarp();
}

// equal_runs for one warp and at most 64 keys (indices 2 lane, 2 lane + 1).
template <class KT>
__device__ __forceinline__ void warp_equal_runs(const KT* s, uint32_t cnt, uint16_t* lo, uint16_t* hi) {
    constexpr uint32_t kInf = 0xFFFFu;
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t i0 = 2u * lane, i1 = i0 + 1u;
    uint32_t a0 = 0u, a1 = 0u, b0 = kInf, b1 = kInf;
    if (i0 < cnt) a0 = (i0 == 0u || !keq(s[i0 - 1u], s[i0])) ? i0 : 0u;
    a1 = (i1 < cnt && !keq(s[i0], s[i1])) ? i1 : a0;
    if (i1 < cnt) b1 = (i1 + 1u >= cnt || !keq(s[i1], s[i1 + 1u])) ? i1 + 1u : kInf;
    if (i0 < cnt) b0 = (i1 >= cnt || !keq(s[i0], s[i1])) ? i0 + 1u : b1;
    uint32_t pa = a1, sb = b0;
#pragma unroll
    for (uint32_t o = 1; o < 32u; o <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL_MASK, pa, o);
        const uint32_t z = __shfl_down_sync(FULL_MASK, sb, o);
        if (lane >= o) pa = max(pa, y);
        if (lane + o < 32u) sb = min(sb, z);
    }
    uint32_t cpre = __shfl_up_sync(FULL_MASK, pa, 1);
    uint32_t csuf = __shfl_down_sync(FULL_MASK, sb, 1);
    if (lane == 0u) cpre = 0u;
    if (lane == 31u) csuf = kInf;
    if (i0 < cnt) {
        lo[i0] = (uint16_t)max(cpre, a0);
        hi[i0] = (uint16_t)min(csuf, b0);
    }
    if (i1 < cnt) {
        lo[i1] = (uint16_t)max(cpre, a1);
        hi[i1] = (uint16_t)min(csuf, b1);
    }
    __syncwarp();
}

// select_splitters for one warp and a tree of at most kMWKMax levels (a
// level's nodes, at most 16, one per lane); returns the levels that hold a
// node with a non-empty sample range.
template <class KT>
__device__ __forceinline__ int warp_select_splitters(const KT* s, uint32_t cnt, int k, KT* lvl, int32_t* ra,
                                                     int32_t* rb, const uint16_t* run_lo, const uint16_t* run_hi) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t v = (1u << k) - 1u;
    if (lane == 0) {
        ra[1] = 0;
        rb[1] = (int32_t)cnt - 1;
    }
    __syncwarp();
    int used = 0;
    for (int l = 0; l < k; l++) {
        const uint32_t first = 1u << l;
        const uint32_t i = first + lane;
        bool nonempty = false;
        if (lane < first) {
            const int32_t a = ra[i], b = rb[i];
            KT x;
            int32_t bl, ar;
            if (a <= b) {
                nonempty = true;
                const int32_t m = a + (b - a) / 2;
                x = s[m];
                bl = max(a, (int32_t)run_lo[m]) - 1;
                ar = min(b + 1, (int32_t)run_hi[m]);
            } else {
                x = lvl[i >> 1];
                bl = a - 1;
                ar = b + 1;
            }
            lvl[i] = x;
            if (2u * i <= v) {
                ra[2 * i] = a; rb[2 * i] = bl;
                ra[2 * i + 1] = ar; rb[2 * i + 1] = b;
            }
        }
        if (__any_sync(FULL_MASK, nonempty)) used = l + 1;
        __syncwarp();
    }
    return used;
}

// emit_tree_smem for one warp (v <= 31 nodes, one per lane).
template <class KT, int N>
__device__ __forceinline__ void warp_emit_tree(const KT* lvl, int k, LevelTree<KT, N>& t, KT* ino) {
    const uint32_t v = (1u << k) - 1u;
    const uint32_t i = 1u + (threadIdx.x & 31u);
    if (i <= v) {
        const uint32_t l = 31u - __clz(i);
        const uint32_t q = i - (1u << l);
        const uint32_t pos = (2u * q + 1u) * (1u << (k - 1 - (int)l)) - 1u;
        t.set(i, lvl[i]);
        ino[pos] = lvl[i];
    }
    __syncwarp();
}

template <class KT>
__global__ void __launch_bounds__(32 * kMWWarps, 32 / kMWWarps) k_med_warp(Work w, Params p) {
    constexpr int kU = 4;  // strings a lane takes at once
    __shared__ MedWarpSmem<KT> smw[kMWWarps];
    const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
    MedWarpSmem<KT>& sm = smw[wid];
    const int cur = w.hdr->round & 1u;
    const int med_in = cur, med_out = cur ^ 1;
    const uint32_t n = w.hdr->n_medw_snap;
    const uint32_t lt = lanemask_lt();
    const Rec* rec_in = w.rec[cur];
    Rec* rec_out = w.rec[cur ^ 1];
    const uint32_t nwarps = gridDim.x * kMWWarps;
    uint32_t nref = 0;
    for (uint32_t mi = blockIdx.x * kMWWarps + wid; mi < n;) {
        Seg g = w.medw[med_in][mi];
        const uint32_t m = g.size, end = g.begin + g.size;
        const int kp = choose_k(m, min(p.k_max, kMWKMax));
        const uint32_t pw = 2u << kp, cnt = pw - 1u;
        int k = kp;
        uint32_t nb = pw - 1u;
        Rec* recs = w.rec[cur];
        for (uint32_t level = 0;; level++) {
            // sample, sorted two keys a lane (top past the sample)
            KT x[2];
#pragma unroll
            for (int r = 0; r < 2; r++) {
                const uint32_t j = 2u * lane + r;
                x[r] = j < cnt ? KeyTraits<KT>::load(recs + g.begin + sample_pos(p.seed, g.begin, m, j))
                               : KeyTraits<KT>::top();
            }
            sm.hist[lane] = 0u;
            sm.hist[lane + 32u] = 0u;
            warp_bitonic64(sm.samp, x[0], x[1]);
            warp_equal_runs(sm.samp, cnt, sm.run_lo, sm.run_hi);
            k = max(1, warp_select_splitters(sm.samp, cnt, kp, sm.lvl, sm.ra, sm.rb, sm.run_lo, sm.run_hi));
            nb = (2u << k) - 1u;
            warp_emit_tree(sm.lvl, k, sm.t, sm.ino);
            // classify: bucket of every string, sizes
            for (uint32_t base = g.begin; base < end; base += 32u * kU) {
                KT kk[kU];
#pragma unroll
                for (int u = 0; u < kU; u++) {
                    const uint32_t e = base + 32u * u + lane;
                    kk[u] = e < end ? KeyTraits<KT>::load(recs + e) : KeyTraits<KT>::top();
                }
                uint32_t bk[kU];
                classify_keys_by<kU>(p.equal_test != 0, kk, bk, sm.t.view(), sm.ino, k);
#pragma unroll
                for (int u = 0; u < kU; u++) {
                    const uint32_t e = base + 32u * u + lane;
                    const uint32_t b = e < end ? bk[u] : (uint32_t)kMWNB;
                    if (e < end) sm.bid[e - g.begin] = (uint8_t)b;
                    const uint32_t peers = __match_any_sync(FULL_MASK, b);
                    if (lane == (uint32_t)(__ffs(peers) - 1)) atomicAdd(&sm.hist[b], (uint32_t)__popc(peers));
                }
            }
            __syncwarp();
            // every string in the equality bucket of one splitter without the
            // terminator: they share the next w characters; gather their keys
            // w deeper in place and classify again
            bool full = false;
            for (uint32_t b = 1u + 2u * lane; b < nb; b += 64u)
                if (sm.hist[b] == m && !kends(sm.ino[b >> 1])) full = true;
            if (!__any_sync(FULL_MASK, full) || level >= kBaseMaxIters) break;
            for (uint32_t e = g.begin + lane; e < end; e += 32u) {
                Rec r = load_rec(recs + e);
                refill_rec<KT>(w.chars, r, g.depth + KeyTraits<KT>::kBytes, g.depth);
                store_rec(recs + e, r);
                nref++;
            }
            g.depth += KeyTraits<KT>::kBytes;
            __syncwarp();
        }
        // bucket starts, two buckets a lane, and the child segments
        uint32_t cnts[2], ckind[2], cstart[2], cdep[2], crun[2];
#pragma unroll
        for (int q = 0; q < 2; q++) cnts[q] = 2u * lane + q < nb ? sm.hist[2u * lane + q] : 0u;
        uint32_t tot;
        uint32_t start = g.begin + warp_excl(cnts[0] + cnts[1], &tot);
#pragma unroll
        for (int q = 0; q < 2; q++) {
            const uint32_t b = 2u * lane + q;
            BucketInfo bi{0u, 0u, false};
            if (b < nb) {
                bi = bucket_info(b, nb, g.depth, sm.ino, cnts[q], p.base_threshold);
                sm.run_pos[b] = start;
                sm.rdep[b] = refill_code(bi, cnts[q], g.depth);
                if (cnts[q] > 0 && start > g.begin) w.out_lcp[start] = kLcpFlag | g.depth;
            }
            ckind[q] = b < nb && cnts[q] > 0 ? child_kind(p, cnts[q], bi.isrun) : kChildNone;
            cstart[q] = start;
            cdep[q] = bi.cdepth;
            crun[q] = bi.runlcp;
            start += cnts[q];
        }
        append_children_n<2>(w, med_out, ckind, cstart, cnts, cdep, crun);
        __syncwarp();
        // stable move, strings in index order
        for (uint32_t base = g.begin; base < end; base += 32u * kU) {
            Rec rr[kU];
            uint32_t bb[kU];
#pragma unroll
            for (int u = 0; u < kU; u++) {
                const uint32_t e = base + 32u * u + lane;
                const bool ok = e < end;
                rr[u] = ok ? load_rec(rec_in + e) : Rec{0ull, 0ull, 0ull, 0u, 0u};
                bb[u] = ok ? (uint32_t)sm.bid[e - g.begin] : (uint32_t)kMWNB;
            }
            // next key words of strings whose bucket moves deeper, issued
            // before any store
#pragma unroll
            for (int u = 0; u < kU; u++) {
                const uint32_t rd = bb[u] < nb ? sm.rdep[bb[u]] : kNoRefill;
                if (rd != kNoRefill && rd != kSingle) {
                    refill_rec<KT>(w.chars, rr[u], rd, g.depth);
                    nref++;
                }
            }
#pragma unroll
            for (int u = 0; u < kU; u++) {
                const uint32_t b = bb[u];
                const uint32_t peers = __match_any_sync(FULL_MASK, b);
                const uint32_t leader = (uint32_t)__ffs(peers) - 1u;
                const uint32_t pos = sm.run_pos[b] + (uint32_t)__popc(peers & lt);
                __syncwarp();
                if (lane == leader && b < nb) sm.run_pos[b] += (uint32_t)__popc(peers);
                __syncwarp();
                if (b < nb) {
                    if (pos >= end) atomicOr(&w.hdr->err, kErrPosition);
                    else if (sm.rdep[b] == kSingle) w.out_perm[pos] = rr[u].idx;
                    else store_rec(rec_out + pos, rr[u]);
                }
            }
        }
        __syncwarp();
        // the next bucket
        uint32_t nx = 0;
        if (lane == 0) nx = nwarps + atomicAdd(&w.hdr->q_medw, 1u);
        mi = __shfl_sync(FULL_MASK, nx, 0);
    }
    add_refills(&w.hdr->med_refills, nref);
}

// ------------------------------------------------------------ base case

constexpr int kBaseThreads = kBaseCap;  // one thread per slot of a tile
// small-list buckets a CTA takes at a time (<= 32: one warp packs them).
// Four keep the work items fine enough for the persistent grid of the graph
// form (8 and 16 measured up to 2.7 % slower on url-16m, no faster on dna-20m)
#ifndef SSS_BASE_CHUNK
#define SSS_BASE_CHUNK 4
#endif
constexpr uint32_t kBaseChunk = SSS_BASE_CHUNK;
static_assert(kBaseChunk >= 1 && kBaseChunk <= 32, "one warp packs a chunk");

struct BaseSmem {
    uint64_t K[kBaseCap];             // key word of the element in a slot
    uint64_t K2[kBaseCap];            // the next 8 characters (valid per O's top bit)
    uint64_t O[kBaseCap];             // its string's byte offset
    uint32_t I[kBaseCap];             // its string index
    uint32_t drun[kBaseCap];          // depth of the run that starts at a slot
    uint32_t RL[kBaseCap];            // length of the run that starts at a slot
    uint32_t SR[kBaseCap];            // group of equal keys a slot belongs to
    uint32_t sbase[kBaseMax + 2];     // first slot of each segment of the tile
    uint32_t sbegin[kBaseMax + 2];    // its first position in the working arrays
    uint16_t R[kBaseCap];             // first slot of the run a slot belongs to
    uint32_t wmax[kBaseThreads / 32];
};

template <class KT> __device__ __forceinline__ KT base_key(uint64_t a, uint64_t b);
template <> __device__ __forceinline__ uint64_t base_key<uint64_t>(uint64_t a, uint64_t) { return a; }
template <> __device__ __forceinline__ Key16 base_key<Key16>(uint64_t a, uint64_t b) { return Key16{a, b}; }

// Buckets of the small list (kTinyMax < size <= base_threshold <= kBaseMax),
// kBaseChunk at a time per CTA (the work queue hands out chunks), packed into
// tiles of at most kBaseCap slots: as many consecutive buckets as fit, on
// consecutive slots; thread s owns slot s.  A run is a contiguous slot range
// whose strings share a prefix of drun[run] bytes, held in index order.
// Each pass ranks every element of every active run among the run's
// elements by (key word, slot) and moves it there (a stable sort of the
// run); then a key change between neighbours fixes their LCP, equal key
// words holding the terminator are equal strings, and groups of equal key
// words without it become runs w bytes deeper (new words gathered) for the
// next pass.  KT: the key of a pass, one word (w = 8) or both cached words
// (w = 16).
template <class KT>
__global__ void __launch_bounds__(kBaseThreads, 8) k_base(Work w, Params p) {
    constexpr bool kWide = KeyTraits<KT>::kBytes == 16;
    __shared__ BaseSmem sm;
    const uint32_t s = threadIdx.x;
    const uint32_t lane = s & 31u, warp = s >> 5;
    const int buf = w.hdr->round & 1u;
    const uint32_t ns = w.hdr->n_small_snap;
    const uint32_t nchunks = (ns + kBaseChunk - 1u) / kBaseChunk;
    __shared__ uint32_t s_item, s_nseg, s_cnt;
    for (uint32_t chunk = first_item(); chunk < nchunks; chunk = next_item(&w.hdr->q_base, &s_item)) {
    const uint32_t c_end = min(ns, (chunk + 1u) * kBaseChunk);
    for (uint32_t e0 = chunk * kBaseChunk; e0 < c_end;) {
    if (warp == 0) {
        // the buckets e0, e0 + 1, ... that fit kBaseCap slots together, on
        // consecutive slots
        Seg g{0u, 0u, 0u, 0u};
        const bool have = e0 + lane < c_end;
        if (have) g = w.small[buf][e0 + lane];
        uint32_t inc = g.size;  // inclusive prefix of the sizes over the lanes
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL_MASK, inc, o);
            if (lane >= (uint32_t)o) inc += y;
        }
        const uint32_t ng = (uint32_t)__popc(__ballot_sync(FULL_MASK, have && inc <= (uint32_t)kBaseCap));
        const uint32_t used = __shfl_sync(FULL_MASK, inc, ng ? ng - 1u : 0u);
        if (lane < ng) {
            const uint32_t b = inc - g.size;
            sm.sbase[lane] = b;
            sm.sbegin[lane] = g.begin;
            sm.drun[b] = g.depth;
            sm.RL[b] = g.size;
        }
        if (lane == 0) {
            s_nseg = ng;
            s_cnt = ng ? used : 0u;
        }
    }
    __syncthreads();
    const uint32_t nseg = s_nseg, cnt = s_cnt;
    if (nseg == 0u) {  // never expected: listed buckets hold at most kBaseMax strings
        if (s == 0) atomicOr(&w.hdr->err, kErrSmallOverflow);
        break;
    }
    e0 += nseg;
    bool act = s < cnt;  // the slot lies in a run to rank in this pass
    uint32_t G = 0, id = 0;
    uint64_t k = 0, k2 = 0, o = 0;
    if (act) {
        uint32_t a = 0, b = nseg;  // last segment with sbase <= s
        while (a < b) { uint32_t m = (a + b) >> 1; if (sm.sbase[m] <= s) a = m + 1; else b = m; }
        const uint32_t i = a - 1;
        G = sm.sbegin[i] + (s - sm.sbase[i]);
        sm.R[s] = (uint16_t)sm.sbase[i];
        const Rec r = load_rec(&w.rec[buf][G]);
        k = r.key;
        k2 = r.key2;
        id = r.idx;
        o = r.off;
        sm.K[s] = k;
        if (kWide) sm.K2[s] = k2;
    }
    __syncthreads();
    uint32_t iter = 0;
    for (;; iter++) {
        if (iter >= kBaseMaxIters) {  // never expected: strings end, so runs end
            if (s == 0) atomicOr(&w.hdr->err, kErrBaseIters);
            break;
        }
        // ---- rank inside the run: (key, slot) order keeps index order for ties
        uint32_t np = s;
        if (act) {
            const uint32_t r = sm.R[s];
            const uint32_t e = r + sm.RL[r];
            uint32_t rank = 0, q = r;
            if constexpr (kWide) {
                // (word, second word, slot) order; the second word only on a tie
                for (; q < e; q++) {
                    const uint64_t a = sm.K[q];
                    if (a != k) {
                        rank += a < k ? 1u : 0u;
                    } else {
                        const uint64_t b = sm.K2[q];
                        rank += (b < k2 || (b == k2 && q < s)) ? 1u : 0u;
                    }
                }
            } else {
                for (; q + 4 <= e; q += 4) {
                    const uint64_t k0 = sm.K[q], k1 = sm.K[q + 1], k2 = sm.K[q + 2], k3 = sm.K[q + 3];
                    rank += (k0 < k || (k0 == k && q < s)) ? 1u : 0u;
                    rank += (k1 < k || (k1 == k && q + 1 < s)) ? 1u : 0u;
                    rank += (k2 < k || (k2 == k && q + 2 < s)) ? 1u : 0u;
                    rank += (k3 < k || (k3 == k && q + 3 < s)) ? 1u : 0u;
                }
                for (; q < e; q++) {
                    const uint64_t kq = sm.K[q];
                    rank += (kq < k || (kq == k && q < s)) ? 1u : 0u;
                }
            }
            np = r + rank;
        }
        __syncthreads();
        if (act) {
            sm.K[np] = k;
            sm.K2[np] = k2;
            sm.I[np] = id;
            sm.O[np] = o;
        }
        __syncthreads();
        // ---- decide neighbours inside the ranked runs
        bool head = true;
        uint32_t dold = 0;
        if (act) {
            k = sm.K[s];
            k2 = sm.K2[s];
            id = sm.I[s];
            o = sm.O[s];
            const uint32_t r = sm.R[s];
            dold = sm.drun[r];
            if (s != r) {
                const KT pk = base_key<KT>(sm.K[s - 1], sm.K2[s - 1]);
                const KT ck = base_key<KT>(k, k2);
                if (!keq(pk, ck)) {
                    w.out_lcp[G] = lcp_of_keys(w, dold, pk, ck);
                } else {
                    head = false;
                    if (kends(ck)) w.out_lcp[G] = lcp_of_equal(w, dold + kchars(ck), id);
                }
            }
        }
        // groups of equal keys: inclusive max-scan of the heads over the slots
        uint32_t inc = head ? s : 0u;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL_MASK, inc, d);
            if (lane >= (uint32_t)d) inc = max(inc, y);
        }
        if (lane == 31) sm.wmax[warp] = inc;
        __syncthreads();
        uint32_t sr = inc;
        for (uint32_t v = 0; v < warp; v++) sr = max(sr, sm.wmax[v]);
        sm.SR[s] = sr;
        __syncthreads();
        const bool multi = (s != sr) || (s + 1 < cnt && sm.SR[s + 1] == s);
        const bool go = act && multi && !kends(base_key<KT>(k, k2));
        if (act) {
            if (go) {
                const uint32_t d = dold + KeyTraits<KT>::kBytes;
                if (s == sr) {
                    sm.drun[s] = d;
                    sm.RL[s] = 0;
                }
                sm.R[s] = (uint16_t)sr;
                refill(w.chars, k, k2, o, d, KeyTraits<KT>::kBytes);
                sm.K[s] = k;
                if (kWide) sm.K2[s] = k2;
            } else {
                sm.R[s] = (uint16_t)s;
            }
        }
        __syncthreads();
        if (go) atomicAdd(&sm.RL[sr], 1u);
        act = go;
        if (!__syncthreads_or(go)) break;
    }
    if (s < cnt) w.out_perm[G] = id;
    if (s == 0) atomicAdd(&w.hdr->base_iters, (unsigned long long)(iter + 1));
    __syncthreads();  // shared arrays are rewritten by the next pack
    }
    }
}

// Base case of the buckets of at most kTinyMax strings.  A warp takes the
// list's buckets kTinyChunk at a time and packs consecutive ones into its 32
// lanes (a bucket's strings on consecutive lanes, as many buckets as fit), so
// that small buckets do not leave most lanes idle.  The passes are those of
// k_base (rank every string of an active run by (key, lane), move it there,
// fix the LCP of neighbours whose keys differ, turn groups of equal keys
// without the terminator into runs w bytes deeper) with a per-warp shared
// buffer and ballots instead of block-wide barriers; a bucket's first lane
// is always a run head, so runs never cross buckets, and a warp stops as
// soon as its own buckets are sorted.
constexpr int kTinyWarps = 8;
constexpr uint32_t kTinyChunk = 8;

template <class KT>
__global__ void __launch_bounds__(32 * kTinyWarps) k_tiny(Work w, Params p) {
    constexpr uint32_t kW = KeyTraits<KT>::kBytes;
    __shared__ uint64_t sK[kTinyWarps][32], sK2[kTinyWarps][32], sO[kTinyWarps][32];
    __shared__ uint32_t sI[kTinyWarps][32];
    __shared__ uint8_t sOwn[kTinyWarps][32];  // the pack's bucket of each lane
    __shared__ unsigned long long s_iters;
    const int buf = w.hdr->round & 1u;
    const uint32_t nt = w.hdr->n_tiny_snap;
    const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
    const uint32_t le = lanemask_lt() | (1u << lane);
    if (threadIdx.x == 0) s_iters = 0ull;
    __syncthreads();
    uint32_t my_iters = 0;
    const uint32_t nchunks = (nt + kTinyChunk - 1u) / kTinyChunk;
    for (uint32_t c = blockIdx.x * kTinyWarps + wid; c < nchunks; c += gridDim.x * kTinyWarps) {
    const uint32_t c_end = min(nt, (c + 1u) * kTinyChunk);
    for (uint32_t e0 = c * kTinyChunk; e0 < c_end;) {
        // the buckets e0, e0 + 1, ... that fit 32 lanes together
        Seg sg{0u, 0u, 0u, 0u};
        if (e0 + lane < c_end) sg = w.tiny[buf][e0 + lane];
        uint32_t inc = sg.size;  // inclusive prefix of the sizes over the lanes
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL_MASK, inc, o);
            if (lane >= (uint32_t)o) inc += y;
        }
        const uint32_t nb = (uint32_t)__popc(__ballot_sync(FULL_MASK, e0 + lane < c_end && inc <= 32u));
        if (nb == 0u) {  // never expected: listed buckets hold at most kTinyMax strings
            if (lane == 0) atomicOr(&w.hdr->err, kErrSmallOverflow);
            break;
        }
        const uint32_t used = __shfl_sync(FULL_MASK, inc, nb - 1u);
        if (lane < nb)
            for (uint32_t x = inc - sg.size; x < inc; x++) sOwn[wid][x] = (uint8_t)lane;
        __syncwarp();
        const bool live = lane < used;
        const uint32_t j = live ? sOwn[wid][lane] : 0u;
        const uint32_t jbegin = __shfl_sync(FULL_MASK, sg.begin, j);
        const uint32_t jdepth = __shfl_sync(FULL_MASK, sg.depth, j);
        const uint32_t jend = __shfl_sync(FULL_MASK, inc, j);
        const uint32_t jfirst = jend - __shfl_sync(FULL_MASK, sg.size, j);
        __syncwarp();  // sOwn is rewritten by the next pack
        e0 += nb;
        const uint32_t G = jbegin + (lane - jfirst);
        uint64_t k = 0, k2 = 0, o = 0;
        uint32_t id = 0;
        if (live) {
            const Rec rc = load_rec(&w.rec[buf][G]);
            k = rc.key;
            k2 = rc.key2;
            o = rc.off;
            id = rc.idx;
        }
        uint32_t rs = jfirst, re = jend, d = jdepth;  // my run [rs, re) and its common prefix
        bool act = live;
        for (uint32_t iter = 0;; iter++) {
            if (iter >= kBaseMaxIters) {  // never expected: strings end, so runs end
                if (lane == 0) atomicOr(&w.hdr->err, kErrBaseIters);
                break;
            }
            my_iters++;
            // ---- rank inside the run: (key, lane) order keeps index order for ties
            sK[wid][lane] = k;
            sK2[wid][lane] = k2;
            __syncwarp();
            uint32_t rank = 0;
            if (act) {
                for (uint32_t q = rs; q < re; q++) {
                    const uint64_t kq = sK[wid][q];
                    bool less;
                    if (kq != k) {
                        less = kq < k;
                    } else if constexpr (kW == 16) {  // first words tie: the second word, then the lane
                        const uint64_t k2q = sK2[wid][q];
                        less = k2q < k2 || (k2q == k2 && q < lane);
                    } else {
                        less = q < lane;
                    }
                    rank += less ? 1u : 0u;
                }
            }
            const uint32_t np = act ? rs + rank : lane;
            __syncwarp();
            if (live) {
                sK[wid][np] = k;
                sK2[wid][np] = k2;
                sO[wid][np] = o;
                sI[wid][np] = id;
            }
            __syncwarp();
            uint64_t pk = 0, pk2 = 0;
            if (live) {
                k = sK[wid][lane];
                k2 = sK2[wid][lane];
                o = sO[wid][lane];
                id = sI[wid][lane];
                if (lane) {
                    pk = sK[wid][lane - 1];
                    pk2 = sK2[wid][lane - 1];
                }
            }
            __syncwarp();
            // ---- decide neighbours inside the ranked runs
            const KT ck = base_key<KT>(k, k2);
            bool head = true;
            if (act && lane != rs) {
                const KT pkk = base_key<KT>(pk, pk2);
                if (!keq(pkk, ck)) {
                    w.out_lcp[G] = lcp_of_keys(w, d, pkk, ck);
                } else {
                    head = false;
                    if (kends(ck)) w.out_lcp[G] = lcp_of_equal(w, d + kchars(ck), id);
                }
            }
            // groups of equal keys: [highest head <= lane, next head above lane)
            const uint32_t heads = __ballot_sync(FULL_MASK, head);
            const uint32_t gs = 31u - (uint32_t)__clz(heads & le);
            const uint32_t above = heads & ~le;
            const uint32_t ge = above ? (uint32_t)__ffs(above) - 1u : 32u;
            const bool go = act && ge - gs >= 2u && !kends(ck);
            if (go) {
                rs = gs;
                re = ge;
                d += kW;
                refill(w.chars, k, k2, o, d, kW);
            }
            act = go;
            if (!__any_sync(FULL_MASK, go)) break;
        }
        if (live) w.out_perm[G] = id;
    }
    }
    if ((threadIdx.x & 31u) == 0 && my_iters) atomicAdd(&s_iters, (unsigned long long)my_iters);
    __syncthreads();
    if (threadIdx.x == 0 && s_iters) atomicAdd(&w.hdr->base_iters, s_iters);
}

// Buckets too large for the base case whose strings are all equal, in
// pieces of at most kRunPiece strings (g.depth: the run's first position).
__global__ void k_bigrun(Work w) {
    const int buf = w.hdr->round & 1u;
    const uint32_t nrun = w.hdr->n_bigrun_snap;
    __shared__ uint32_t s_item;
    for (uint32_t r = first_item(); r < nrun; r = next_item(&w.hdr->q_bigrun, &s_item)) {
        const Seg g = w.bigrun[buf][r];
        // equal strings: their common length
        const uint32_t runlcp = lcp_of_equal(w, g.aux, w.rec[buf][g.begin].idx);
#pragma unroll 4
        for (uint32_t i = threadIdx.x; i < g.size; i += blockDim.x) {
            const uint32_t q = g.begin + i;
            w.out_perm[q] = w.rec[buf][q].idx;
            if (q > g.depth) w.out_lcp[q] = runlcp;
        }
    }
}

// ------------------------------------------------------------ fixup

// LCP at a bucket boundary created in a round at depth l: the two neighbours'
// key words at depth l differ, so lcp = l + lcp of the two words.
__global__ void k_fixup(Work w) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x + 1; q < w.n; q += stride) {
        const uint32_t x = w.out_lcp[q];
        if (x & kLcpFlag) {
            const uint32_t l = x & ~kLcpFlag;
            const uint32_t pa = w.out_perm[q - 1], pb = w.out_perm[q];
            if (pa >= w.n || pb >= w.n) {
                atomicOr(&w.hdr->err, kErrPosition);
                continue;
            }
            // the two strings share l characters and differ within the next
            // w <= 16 (the key that put them in different buckets)
            Key16 a, b;
            load_key2(w.chars, w.offsets[pa] + l, a.h, a.l);
            load_key2(w.chars, w.offsets[pb] + l, b.h, b.l);
            if (keq(a, b)) atomicOr(&w.hdr->err, kErrEqualBoundary);
            w.out_lcp[q] = lcp_of_keys(w, l, a, b);
        }
    }
}

// ------------------------------------------------------------ scan (tile sums, down-sweep)

constexpr int kScanThreads = 256;
constexpr int kScanPer = 16;
constexpr uint32_t kScanTile = kScanThreads * kScanPer;

size_t scan_tmp_elems(uint32_t n) { return (size_t)(n + kScanTile - 1) / kScanTile + 1; }

// Tile sums of the input; the CTA that finishes last (a counter in device
// memory, no waiting) scans them in place, writes the total to out[n] and
// resets the counter.
__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t* in, const uint32_t* n_ptr,
                                                              uint32_t* sums, uint32_t* out, uint32_t* done) {
    __shared__ uint32_t wsum[33];
    __shared__ uint32_t s_last;
    const uint32_t n = *n_ptr;
    const uint32_t tiles = (n + kScanTile - 1) / kScanTile;
    for (uint32_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const uint32_t base = tile * kScanTile;
        uint32_t s = 0;
#pragma unroll
        for (int j = 0; j < kScanPer; j++) {
            const uint32_t i = base + j * kScanThreads + threadIdx.x;
            if (i < n) s += in[i];
        }
        uint32_t tot;
        block_excl_sum(s, wsum, &tot);
        if (threadIdx.x == 0) sums[tile] = tot;
    }
    if (threadIdx.x == 0) {
        __threadfence();  // this CTA's tile sums before its count
        s_last = atomicAdd(done, 1u) == gridDim.x - 1u ? 1u : 0u;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const uint32_t per = (tiles + blockDim.x - 1) / blockDim.x;
    const uint32_t lo = min(tiles, threadIdx.x * per), hi = min(tiles, lo + per);
    uint32_t s = 0;
    for (uint32_t i = lo; i < hi; i++) s += __ldcg(sums + i);
    uint32_t tot;
    uint32_t ex = block_excl_sum(s, wsum, &tot);
    for (uint32_t i = lo; i < hi; i++) {
        const uint32_t x = __ldcg(sums + i);
        sums[i] = ex;
        ex += x;
    }
    if (threadIdx.x == 0) {
        out[n] = tot;
        *done = 0u;
    }
}

// Down-sweep: each tile of kScanTile entries goes through shared memory
// (padded, entry i at i + i / 32, so that neither the coalesced copies nor
// the threads' runs of kScanPer consecutive entries conflict on banks), so
// that both its loads and its stores are whole coalesced lines.
__global__ void __launch_bounds__(kScanThreads) k_scan_down(const uint32_t* in, uint32_t* out, const uint32_t* n_ptr,
                                                            const uint32_t* sums) {
    __shared__ uint32_t wsum[33];
    __shared__ uint32_t tb[kScanTile + kScanTile / 32];
    const uint32_t n = *n_ptr;
    const uint32_t tiles = (n + kScanTile - 1) / kScanTile;
    for (uint32_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const uint32_t t0 = tile * kScanTile;
#pragma unroll
        for (int j = 0; j < kScanPer; j++) {
            const uint32_t i = j * kScanThreads + threadIdx.x;
            tb[i + (i >> 5)] = t0 + i < n ? in[t0 + i] : 0u;
        }
        __syncthreads();
        const uint32_t b = threadIdx.x * kScanPer;
        uint32_t v[kScanPer];
        uint32_t s = 0;
#pragma unroll
        for (int j = 0; j < kScanPer; j++) {
            const uint32_t i = b + j;
            v[j] = tb[i + (i >> 5)];
            s += v[j];
        }
        // (block_excl_sum's barriers also end every read of tb above)
        uint32_t ex = block_excl_sum(s, wsum, nullptr) + sums[tile];
#pragma unroll
        for (int j = 0; j < kScanPer; j++) {
            const uint32_t i = b + j;
            tb[i + (i >> 5)] = ex;
            ex += v[j];
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kScanPer; j++) {
            const uint32_t i = j * kScanThreads + threadIdx.x;
            if (t0 + i < n) out[t0 + i] = tb[i + (i >> 5)];
        }
        __syncthreads();
    }
}

// out[0..n) = exclusive prefix sums of in[0..n), out[n] = total, with n read
// from device memory (*n_ptr); n_host (if known) only sizes the grid.  tmp
// holds scan_tmp_elems(n) entries; done is a counter that is zero between
// scans.
cudaError_t launch_scan_u32(const uint32_t* in, uint32_t* out, const uint32_t* n_ptr, const uint32_t* n_host,
                            uint32_t* tmp, uint32_t* done, Prof* pf, cudaStream_t st) {
    uint32_t grid = device_sms() * 8u;
    if (n_host) {
        const uint32_t tiles = (*n_host + kScanTile - 1) / kScanTile;
        grid = max(1u, min(grid, tiles));
    }
    ProfScope ps(pf, kScan, st);
    k_scan_reduce<<<grid, kScanThreads, 0, st>>>(in, n_ptr, tmp, out, done);
    k_scan_down<<<grid, kScanThreads, 0, st>>>(in, out, n_ptr, tmp);
    if (pf) { pf->launches += 1; pf->cls_launches[kScan] += 1; }
    return cudaGetLastError();
}

// ------------------------------------------------------------ launches

static uint32_t grid_for(uint64_t n, uint32_t threads, uint32_t per_sm, uint32_t num_sms) {
    uint64_t g = (n + threads - 1) / threads;
    uint64_t cap = (uint64_t)num_sms * per_sm;
    if (g > cap) g = cap;
    return g ? (uint32_t)g : 1u;
}

uint32_t device_sms() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? (uint32_t)sms : 148u;
}

// Grid of a queue-driven kernel: one CTA per work item when the host knows
// the count (0 = nothing to launch), else `fixed` persistent CTAs.
static uint32_t grid_of(uint32_t fixed, const Hdr* hc, uint32_t known) { return hc ? known : fixed; }

cudaError_t launch_init(const Work& w, const Params& p, Prof* pf, cudaStream_t st) {
    if (w.n && !p.fuse_root) {
        // the shadow arrays only ever hold valid string indices and offsets
        // (a fused root needs no clearing: its round 0 scatters the single
        // root over every position of the shadow array before any reads)
        cudaError_t e = cudaMemsetAsync(w.rec[1], 0, sizeof(Rec) * (size_t)w.n, st);  // index 0, offset 0
        if (e != cudaSuccess) return e;
        ProfScope ps(pf, kInit, st);
        k_init<<<grid_for(w.n, 256, 16, device_sms()), 256, 0, st>>>(w);
    }
    return cudaGetLastError();
}

template <class KT>
static cudaError_t launch_fused_root_t(const Work& w, const Params& p, const Hdr* hc, Prof* pf, cudaStream_t st) {
    {
        ProfScope ps(pf, kSample, st);
        k_sample<KT><<<1, 1024, sizeof(SampleSmem<KT>), st>>>(w, p, 1);
    }
    ProfScope ps(pf, kInit, st);
    const uint32_t g = grid_of(p.num_sms * SSS_INIT_CLASSIFY_MIN_BLOCKS, hc, hc ? hc->total_chunks : 0u);
    if (g) k_init_classify<KT><<<g, kClassifyThreads, 0, st>>>(w, p);
    return cudaGetLastError();
}

cudaError_t launch_fused_root(const Work& w, const Params& p, const Hdr* hc, Prof* pf, cudaStream_t st) {
    if (!p.fuse_root) return cudaSuccess;
    return p.key_bytes == 16 ? launch_fused_root_t<Key16>(w, p, hc, pf, st)
                             : launch_fused_root_t<uint64_t>(w, p, hc, pf, st);
}

cudaError_t launch_roots(const Work& w, const Params& p, const Seg* roots, uint32_t num_roots, Prof* pf,
                         cudaStream_t st) {
    {
        ProfScope ps(pf, kInit, st);
        k_hdr_reset<<<1, 1, 0, st>>>(w);
    }
    ProfScope ps(pf, kInit, st);
    if (roots) {
        if (num_roots)
            k_roots<<<grid_for(num_roots, 256, 4, p.num_sms), 256, 0, st>>>(w, p, roots, num_roots, Seg{});
    } else {
        k_roots<<<1, 32, 0, st>>>(w, p, nullptr, 1u, Seg{0u, w.n, 0u, 0u});
    }
    return cudaGetLastError();
}

cudaError_t launch_plan(const Work& w, const Params& p, Prof* pf, cudaStream_t st, uint32_t advance,
                        cudaGraphConditionalHandle cond) {
    ProfScope ps(pf, kPlan, st);
    k_plan<<<1, 1024, 0, st>>>(w, p, advance, cond);
    return cudaGetLastError();
}

template <class KT>
static cudaError_t launch_round_t(const Work& w, const Params& p, const Hdr* hc, Prof* pf, cudaStream_t st) {
    const uint32_t sms = p.num_sms;
    const uint32_t gL = grid_of(sms * 2u, hc, hc ? hc->L : 0u);
    if (gL) {
        {
            ProfScope ps(pf, kSample, st);
            k_sample<KT><<<gL, 1024, sizeof(SampleSmem<KT>), st>>>(w, p, 0);
        }
        if (p.learned) {
            // one CTA per SM at most: a fit CTA holds most of an SM's shared
            // memory, and most large segments are below the model's minimum size
            cudaError_t e = launch_cdf_fit(w, p, hc ? min(hc->L, sms) : sms, pf, st);
            if (e != cudaSuccess) return e;
        }
        const uint32_t gc = grid_of(sms * 4u, hc, hc ? hc->total_chunks : 0u);
        {
            ProfScope ps(pf, kClassify, st);
            k_classify<KT><<<gc, kClassifyThreads, 0, st>>>(w, p);
        }
        cudaError_t e = launch_scan_u32(w.counts, w.counts_scan, &w.hdr->total_counts, hc ? &hc->total_counts : nullptr,
                                        w.scan_tmp, w.scan_tmp + (w.scan_tmp_max - 1u), pf, st);
        if (e != cudaSuccess) return e;
        {
            ProfScope ps(pf, kScatter, st);
            k_scatter<KT><<<grid_of(sms * SSS_SCATTER_MIN_BLOCKS, hc, hc ? hc->total_chunks : 0u), kScatterThreads,
                            sizeof(ScatterSmem<KT>), st>>>(w, p);
        }
    }
    return cudaGetLastError();
}

template <class KT>
static cudaError_t launch_medium_t(const Work& w, const Params& p, const Hdr* hc, Prof* pf, cudaStream_t st) {
    const uint32_t gm = grid_of(p.num_sms * SSS_MED_MIN_BLOCKS, hc, hc ? hc->n_med_snap : 0u);
    if (gm) {
        ProfScope ps(pf, kMedium, st);
        k_med_round<KT><<<gm, kScatterThreads, sizeof(MedSmem<KT>), st>>>(w, p);
    }
    if (kMedWarpMax > 0u) {
        const uint32_t gw = grid_of(p.num_sms * (32u / kMWWarps), hc,
                                    hc ? (hc->n_medw_snap + kMWWarps - 1u) / kMWWarps : 0u);
        if (gw) {
            ProfScope ps(pf, kMedium, st);
            k_med_warp<KT><<<gw, 32 * kMWWarps, 0, st>>>(w, p);
        }
    }
    return cudaGetLastError();
}

#ifndef SSS_BRANCH_PRIORITIES
#define SSS_BRANCH_PRIORITIES 1
#endif

cudaError_t branches_create(Branches& b) {
    // priorities: the device-wide round first (the chain every later round
    // waits on), then the medium rounds (whose children feed the next
    // round), and the base case of finished buckets fills what is left
    int least = 0, greatest = 0;
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    if (!SSS_BRANCH_PRIORITIES) greatest = least;
    const int middle = greatest < least ? greatest + 1 : greatest;
    const int p_base = least, p_med = middle;
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&b.large, cudaStreamNonBlocking, greatest);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&b.base, cudaStreamNonBlocking, p_base);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&b.medium, cudaStreamNonBlocking, p_med);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&b.tiny, cudaStreamNonBlocking, p_base);
    // the same priorities as stream launch attributes, which stream capture
    // copies into the kernel nodes of a graph (optional: ignored if refused)
    if (e == cudaSuccess) {
        const cudaStream_t ss[4] = {b.large, b.base, b.medium, b.tiny};
        const int pr[4] = {greatest, p_base, p_med, p_base};
        for (int i = 0; i < 4; i++) {
            cudaLaunchAttributeValue v;
            memset(&v, 0, sizeof(v));
            v.priority = pr[i];
            if (cudaStreamSetAttribute(ss[i], cudaLaunchAttributePriority, &v) != cudaSuccess) cudaGetLastError();
        }
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b.fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b.join_large, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b.join_base, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b.join_medium, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b.join_tiny, cudaEventDisableTiming);
    if (e != cudaSuccess) branches_destroy(b);
    return e;
}

void branches_destroy(Branches& b) {
    if (b.large) cudaStreamDestroy(b.large);
    if (b.base) cudaStreamDestroy(b.base);
    if (b.medium) cudaStreamDestroy(b.medium);
    if (b.tiny) cudaStreamDestroy(b.tiny);
    if (b.fork) cudaEventDestroy(b.fork);
    if (b.join_large) cudaEventDestroy(b.join_large);
    if (b.join_base) cudaEventDestroy(b.join_base);
    if (b.join_medium) cudaEventDestroy(b.join_medium);
    if (b.join_tiny) cudaEventDestroy(b.join_tiny);
    b = Branches();
}

static cudaError_t launch_tiny(const Work& w, const Params& p, const Hdr* hc, Prof* pf, cudaStream_t st);
static cudaError_t launch_tiles(const Work& w, const Params& p, const Hdr* hc, uint32_t* out_tiles, Prof* pf,
                                cudaStream_t st);

cudaError_t launch_body(const Work& w, const Params& p, const Hdr* hc, uint32_t* out_tiles, Prof* pf,
                        cudaStream_t st, const Branches* br) {
    const bool wide = p.key_bytes == 16;
    cudaStream_t sl = st, sb = st, sm = st, sy = st;
    cudaError_t e = cudaSuccess;
    if (br) {
        sl = br->large;
        sb = br->base;
        sm = br->medium;
        sy = br->tiny;
        if ((e = cudaEventRecord(br->fork, st)) != cudaSuccess) return e;
        for (cudaStream_t x : {sl, sb, sm, sy})
            if ((e = cudaStreamWaitEvent(x, br->fork, 0)) != cudaSuccess) return e;
    }
    e = wide ? launch_round_t<Key16>(w, p, hc, pf, sl) : launch_round_t<uint64_t>(w, p, hc, pf, sl);
    if (e != cudaSuccess) return e;
    e = wide ? launch_medium_t<Key16>(w, p, hc, pf, sm) : launch_medium_t<uint64_t>(w, p, hc, pf, sm);
    if (e != cudaSuccess) return e;
    if ((e = launch_tiles(w, p, hc, out_tiles, pf, sb)) != cudaSuccess) return e;
    if ((e = launch_tiny(w, p, hc, pf, sy)) != cudaSuccess) return e;
    if (br) {
        const cudaEvent_t joins[4] = {br->join_large, br->join_base, br->join_medium, br->join_tiny};
        const cudaStream_t from[4] = {sl, sb, sm, sy};
        for (int i = 0; i < 4; i++) {
            if ((e = cudaEventRecord(joins[i], from[i])) != cudaSuccess) return e;
            if ((e = cudaStreamWaitEvent(st, joins[i], 0)) != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

// Loop condition of the graph form: another round is needed while the last
// plan left large or medium segments.
__global__ void k_set_cond(Work w, cudaGraphConditionalHandle cond) {
    cudaGraphSetConditional(cond, (w.hdr->L > 0u || w.hdr->n_med_snap > 0u || w.hdr->n_medw_snap > 0u) ? 1u : 0u);
}

cudaError_t launch_set_cond(const Work& w, cudaGraphConditionalHandle cond, cudaStream_t st) {
    k_set_cond<<<1, 1, 0, st>>>(w, cond);
    return cudaGetLastError();
}

// Shared-memory limits of the kernels that need more than 48 KB (set once,
// outside any stream capture).
template <class KT>
static cudaError_t prepare_kernels_t() {
    const auto set = [](const void* f, size_t bytes) {
        return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    };
    cudaError_t e = set((const void*)k_scatter<KT>, sizeof(ScatterSmem<KT>));
    if (e == cudaSuccess) e = set((const void*)k_med_round<KT>, sizeof(MedSmem<KT>));
    if (e == cudaSuccess) e = set((const void*)k_sample<KT>, sizeof(SampleSmem<KT>));
    return e;
}

cudaError_t prepare_kernels(uint32_t cdf_M) {
    cudaError_t e = prepare_kernels_t<uint64_t>();
    if (e == cudaSuccess) e = prepare_kernels_t<Key16>();
    if (e == cudaSuccess) e = prepare_cdf_kernels(cdf_M);
    return e;
}

// The warp-form base case (buckets of at most kTinyMax strings).
static cudaError_t launch_tiny(const Work& w, const Params& p, const Hdr* hc, Prof* pf, cudaStream_t st) {
    const uint32_t gt = grid_of(p.num_sms * 8u, hc,
                                hc ? (hc->n_tiny_snap + kTinyWarps * kTinyChunk - 1) / (kTinyWarps * kTinyChunk) : 0u);
    if (gt) {
        ProfScope ps(pf, kBase, st);
        if (p.key_bytes == 16) k_tiny<Key16><<<gt, 32 * kTinyWarps, 0, st>>>(w, p);
        else k_tiny<uint64_t><<<gt, 32 * kTinyWarps, 0, st>>>(w, p);
    }
    return cudaGetLastError();
}

// The tile-form base case (k_base over chunks of the small list) and the
// large runs of equal strings.  out_tiles: the chunks launched.
static cudaError_t launch_tiles(const Work& w, const Params& p, const Hdr* hc, uint32_t* out_tiles, Prof* pf,
                                cudaStream_t st) {
    const uint32_t sms = p.num_sms;
    const uint32_t tiles = hc ? (hc->n_small_snap + kBaseChunk - 1u) / kBaseChunk : 0u;
    if (!hc || tiles) {
        ProfScope ps(pf, kBase, st);
        const uint32_t g = grid_of(sms * 8u, hc, tiles);
        if (p.key_bytes == 16) k_base<Key16><<<g, kBaseThreads, 0, st>>>(w, p);
        else k_base<uint64_t><<<g, kBaseThreads, 0, st>>>(w, p);
    }
    const uint32_t gr = grid_of(sms * 4u, hc, hc ? hc->n_bigrun_snap : 0u);
    if (gr) {
        ProfScope ps(pf, kRuns, st);
        k_bigrun<<<gr, 256, 0, st>>>(w);
    }
    if (out_tiles) *out_tiles = tiles;
    return cudaGetLastError();
}

cudaError_t launch_small(const Work& w, const Params& p, const Hdr* hc, uint32_t* out_tiles, Prof* pf,
                         cudaStream_t st) {
    cudaError_t e = launch_tiles(w, p, hc, out_tiles, pf, st);
    return e != cudaSuccess ? e : launch_tiny(w, p, hc, pf, st);
}

cudaError_t launch_fixup(const Work& w, Prof* pf, cudaStream_t st) {
    if (w.n > 1) {
        ProfScope ps(pf, kFixup, st);
        k_fixup<<<grid_for(w.n, 256, 16, device_sms()), 256, 0, st>>>(w);
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------ single steps

__global__ void k_gather_keys(const uint8_t* chars, const uint64_t* offsets, const uint32_t* idx,
                              const uint32_t* depth, uint32_t n, uint64_t* out) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint32_t s = idx ? idx[i] : i;
        out[i] = load_key(chars, offsets[s] + depth[i]);
    }
}

cudaError_t launch_gather_keys(const uint8_t* chars, const uint64_t* offsets, const uint32_t* idx,
                               const uint32_t* depth, uint32_t n, uint64_t* out, cudaStream_t st) {
    if (n) k_gather_keys<<<grid_for(n, 256, 16, device_sms()), 256, 0, st>>>(chars, offsets, idx, depth, n, out);
    return cudaGetLastError();
}

cudaError_t launch_build_splitters(const uint64_t* sample, uint32_t count, int k, uint64_t* lvl, uint64_t* ino,
                                   cudaStream_t st) {
    k_build_splitters<<<1, 1024, 0, st>>>(sample, count, k, lvl, ino);
    return cudaGetLastError();
}

__global__ void k_classify_keys(const uint64_t* keys, uint32_t n, const uint64_t* lvl, const uint64_t* inorder,
                                int k, uint16_t* out, int equal_test) {
    __shared__ uint64_t t[kVMax + 1];
    __shared__ uint64_t ino[kVMax];
    const uint32_t v = (1u << k) - 1u;
    for (uint32_t i = threadIdx.x; i < v; i += blockDim.x) { t[i + 1] = lvl[i]; ino[i] = inorder[i]; }
    __syncthreads();
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint64_t key[1] = {keys[i]};
        uint32_t b[1];
        classify_keys_by<1>(equal_test != 0, key, b, (const uint64_t*)t, (const uint64_t*)ino, k);
        out[i] = (uint16_t)b[0];
    }
}

cudaError_t launch_classify(const uint64_t* keys, uint32_t n, const uint64_t* lvl, const uint64_t* ino, int k,
                            uint16_t* out, int equal_test, cudaStream_t st) {
    if (n) k_classify_keys<<<grid_for(n, 256, 8, device_sms()), 256, 0, st>>>(keys, n, lvl, ino, k, out, equal_test);
    return cudaGetLastError();
}

// Batched: indices relative to each set's first string.
__global__ void k_localize(uint32_t* perm, const Seg* roots, uint32_t num_roots) {
    for (uint32_t j = blockIdx.x; j < num_roots; j += gridDim.x) {
        const Seg g = roots[j];
        for (uint32_t i = threadIdx.x; i < g.size; i += blockDim.x) perm[g.begin + i] -= g.begin;
    }
}

cudaError_t launch_localize(uint32_t* perm, const Seg* roots, uint32_t num_roots, Prof* pf, cudaStream_t st) {
    if (num_roots) {
        ProfScope ps(pf, kFixup, st);
        k_localize<<<grid_for((uint64_t)num_roots * 256, 256, 8, device_sms()), 256, 0, st>>>(perm, roots,
                                                                                               num_roots);
    }
    return cudaGetLastError();
}

}  // namespace sss
