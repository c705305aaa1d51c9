// Distribution-round kernels of super scalar string sample sort (S^5,
// Sec. 3.1 of Bingmann & Sanders) for sm_103a.
//
// One round over all large segments at once:
//   k_sample    one CTA per segment: pseudo-random sample of 2v+1 key
//               words, in-shared-memory sort, recursive duplicate-skipping
//               splitter choice, perfect tree in level order + in order
//   k_classify  one CTA per work chunk: tree in shared memory, branch-free
//               descent + one equality test per key, warp-aggregated
//               shared-memory histogram, per-chunk bucket counts out
//   scan        exclusive prefix sum over the bucket-major count matrix
//   k_scatter   one CTA per chunk: classifies again, stable rank of each
//               string inside its bucket (warp match + per-warp counters),
//               out-of-place move into the shadow arrays (the two arrays swap
//               roles each round), new key word gathered where the common
//               prefix grows; chunk 0 of every segment turns its buckets
//               into child segments (Eq. (1) depth rule) and marks the
//               bucket boundaries whose LCP is resolved at the end
//   k_plan      one CTA: lays out the next round (tree depth per segment,
//               work chunks, count-matrix offsets)
// Buckets of at most base_threshold strings go to k_base, a shared-memory
// segmented sort that also emits the LCP entries.
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

// ------------------------------------------------------------ init

__global__ void k_init(Work w) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < w.n; i += stride) {
        w.idx[0][i] = i;
        w.key[0][i] = load_key(w.chars, w.offsets[i]);
        w.out_lcp[i] = 0u;
    }
}

__global__ void k_hdr_reset(Work w) {
    Hdr* h = w.hdr;
    h->n_large = 0; h->n_small = 0; h->n_bigrun = 0; h->err = 0; h->small_elems = 0;
    h->refills = 0ull;
}

// Roots: one segment per set (a single sort is one set).  Set j occupies
// [roots[j].begin, +size) at depth 0; singletons finish here.
__global__ void k_roots(Work w, const Seg* roots, uint32_t num_roots, Seg single, uint32_t base_threshold) {
    Hdr* h = w.hdr;
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < num_roots; j += gridDim.x * blockDim.x) {
        const Seg g = roots ? roots[j] : single;
        if (g.size == 0) continue;
        if (g.size == 1) {
            w.out_perm[g.begin] = g.begin;
        } else if (g.size > base_threshold) {
            uint32_t s = atomicAdd(&h->n_large, 1u);
            if (s < w.lmax) w.large[s] = g; else atomicOr(&h->err, kErrLargeOverflow);
        } else {
            uint32_t s = atomicAdd(&h->n_small, 1u);
            if (s < w.smax) { w.small[s] = g; w.small_size[s] = g.size; atomicAdd(&h->small_elems, g.size); }
            else atomicOr(&h->err, kErrSmallOverflow);
        }
    }
}

// ------------------------------------------------------------ plan

__global__ void __launch_bounds__(1024) k_plan(Work w, Params p) {
    __shared__ uint32_t wsum[33];
    Hdr* h = w.hdr;
    const uint32_t L_all = h->n_large;
    const uint32_t L = min(L_all, w.lmax);
    const uint32_t per = (L + blockDim.x - 1) / blockDim.x;
    const uint32_t lo = min(L, threadIdx.x * per), hi = min(L, lo + per);
    uint32_t sc = 0, sn = 0, st = 0, sa = 0;
    for (uint32_t s = lo; s < hi; s++) {
        Seg g = w.large[s];
        int k = choose_k(g.size, p.k_max);
        uint32_t ch = (g.size + p.chunk - 1) / p.chunk;
        sc += ch;
        sn += ((2u << k) - 1u) * ch;
        st += 1u << k;
        sa += g.size;
    }
    uint32_t tc, tn, tt, ta;
    uint32_t bc = block_excl_sum(sc, wsum, &tc);
    uint32_t bn = block_excl_sum(sn, wsum, &tn);
    uint32_t bt = block_excl_sum(st, wsum, &tt);
    block_excl_sum(sa, wsum, &ta);
    const bool ok = tc <= w.chmax && tn <= w.cmax && tt <= w.tmax && L_all <= w.lmax;
    if (ok) {
        for (uint32_t s = lo; s < hi; s++) {
            Seg g = w.large[s];
            int k = choose_k(g.size, p.k_max);
            uint32_t ch = (g.size + p.chunk - 1) / p.chunk;
            w.plans[s] = SegPlan{g.begin, g.size, g.depth, (uint32_t)k, ch, bc, bn, bt};
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
        h->large_elems_snap = ok ? ta : 0u;
        h->n_small_snap = h->n_small;
        h->n_bigrun_snap = h->n_bigrun;
        h->small_elems_snap = h->small_elems;
        h->n_large = 0;
        h->n_small = 0;
        h->n_bigrun = 0;
        h->small_elems = 0;
    }
}

// ------------------------------------------------------------ sample + tree

// Ascending bitonic sort of s[0..pw) (pw a power of two) by the whole block.
__device__ void bitonic_sort_u64(uint64_t* s, uint32_t pw) {
    for (uint32_t size = 2; size <= pw; size <<= 1) {
        for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
            for (uint32_t i = threadIdx.x; i < pw / 2; i += blockDim.x) {
                uint32_t lo = 2u * i - (i & (stride - 1u));
                uint32_t hi = lo + stride;
                bool asc = (lo & size) == 0;
                uint64_t a = s[lo], b = s[hi];
                if ((a > b) == asc) { s[lo] = b; s[hi] = a; }
            }
            __syncthreads();
        }
    }
}

__device__ __forceinline__ uint32_t lower_bound_u64(const uint64_t* s, uint32_t n, uint64_t x) {
    uint32_t lo = 0, hi = n;
    while (lo < hi) {
        uint32_t m = (lo + hi) >> 1;
        if (s[m] < x) lo = m + 1; else hi = m;
    }
    return lo;
}

__device__ __forceinline__ uint32_t upper_bound_u64(const uint64_t* s, uint32_t n, uint64_t x) {
    uint32_t lo = 0, hi = n;
    while (lo < hi) {
        uint32_t m = (lo + hi) >> 1;
        if (s[m] <= x) lo = m + 1; else hi = m;
    }
    return lo;
}

// Splitter choice of Sec. 3.1 on the sorted sample s[0..cnt): a node owning
// the range a..b takes its middle sample x; its children own a..b' and a'..b
// where b' and a' skip every sample equal to x.  A node whose range is empty
// repeats its parent's splitter.  Level by level, one thread per node.
// lvl[1..v] receives the level-order tree; ra/rb: shared scratch [v+1].
__device__ void select_splitters(const uint64_t* s, uint32_t cnt, int k, uint64_t* lvl, int32_t* ra, int32_t* rb) {
    const uint32_t v = (1u << k) - 1u;
    if (threadIdx.x == 0) { ra[1] = 0; rb[1] = (int32_t)cnt - 1; }
    __syncthreads();
    for (int l = 0; l < k; l++) {
        const uint32_t first = 1u << l;
        for (uint32_t i = first + threadIdx.x; i < 2u * first; i += blockDim.x) {
            int32_t a = ra[i], b = rb[i];
            uint64_t x;
            int32_t bl, ar;
            if (a <= b) {
                int32_t m = a + (b - a) / 2;
                x = s[m];
                int32_t first_eq = (int32_t)lower_bound_u64(s, cnt, x);
                int32_t past_eq = (int32_t)upper_bound_u64(s, cnt, x);
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

// Writes the tree lvl[1..v] to out_lvl[0..v) and its in-order sequence to out_ino[0..v).
__device__ void emit_tree(const uint64_t* lvl, int k, uint64_t* out_lvl, uint64_t* out_ino) {
    const uint32_t v = (1u << k) - 1u;
    for (uint32_t i = 1 + threadIdx.x; i <= v; i += blockDim.x) {
        uint32_t l = 31u - __clz(i);
        uint32_t q = i - (1u << l);
        uint32_t pos = (2u * q + 1u) * (1u << (k - 1 - (int)l)) - 1u;
        out_lvl[i - 1] = lvl[i];
        out_ino[pos] = lvl[i];
    }
}

__global__ void __launch_bounds__(1024) k_sample(Work w, Params p, int cur) {
    __shared__ uint64_t samp[kSampleMax];
    __shared__ uint64_t lvl[kVMax + 1];
    __shared__ int32_t ra[kVMax + 1], rb[kVMax + 1];
    const SegPlan P = w.plans[blockIdx.x];
    const int k = (int)P.k;
    const uint32_t pw = 2u << k;
    const uint32_t cnt = pw - 1u;  // alpha (v + 1) - 1 with alpha = 2
    const uint64_t* keys = w.key[cur];
    const uint64_t base = p.seed ^ ((uint64_t)P.begin * 0x9E3779B97F4A7C15ull) ^ ((uint64_t)P.size << 32);
    for (uint32_t j = threadIdx.x; j < pw; j += blockDim.x) {
        uint64_t x = ~0ull;
        if (j < cnt) {
            uint32_t r = (uint32_t)(mix64(base + (uint64_t)j * 0xD1B54A32D192ED03ull) >> 32);
            uint32_t off = (uint32_t)(((uint64_t)r * P.size) >> 32);
            x = keys[P.begin + off];
        }
        samp[j] = x;
    }
    __syncthreads();
    bitonic_sort_u64(samp, pw);
    select_splitters(samp, cnt, k, lvl, ra, rb);
    emit_tree(lvl, k, w.tree_lvl + P.tree_base, w.tree_ino + P.tree_base);
}

// Stand-alone splitter construction for a caller's sample (sss_build_splitters).
__global__ void __launch_bounds__(1024) k_build_splitters(const uint64_t* sample, uint32_t count, int k,
                                                          uint64_t* out_lvl, uint64_t* out_ino) {
    __shared__ uint64_t samp[kSampleMax];
    __shared__ uint64_t lvl[kVMax + 1];
    __shared__ int32_t ra[kVMax + 1], rb[kVMax + 1];
    uint32_t pw = 1;
    while (pw < count) pw <<= 1;
    for (uint32_t j = threadIdx.x; j < pw; j += blockDim.x) samp[j] = j < count ? sample[j] : ~0ull;
    __syncthreads();
    bitonic_sort_u64(samp, pw);
    select_splitters(samp, count, k, lvl, ra, rb);
    emit_tree(lvl, k, out_lvl, out_ino);
}

// ------------------------------------------------------------ classify + count

constexpr int kClassifyThreads = 256;
constexpr int kClassifyUnroll = 4;

__global__ void __launch_bounds__(kClassifyThreads) k_classify(Work w, Params p, int cur) {
    __shared__ uint64_t t[kVMax + 1];
    __shared__ uint64_t ino[kVMax];
    __shared__ uint32_t hist[kNBMax + 1];
    const uint32_t c = blockIdx.x;
    const uint32_t s = w.chunk_seg[c];
    const SegPlan P = w.plans[s];
    const uint32_t ci = c - P.chunk_base;
    const int k = (int)P.k;
    const uint32_t v = (1u << k) - 1u, nb = 2u * v + 1u;
    for (uint32_t i = threadIdx.x; i < v; i += blockDim.x) {
        t[i + 1] = w.tree_lvl[P.tree_base + i];
        ino[i] = w.tree_ino[P.tree_base + i];
    }
    for (uint32_t b = threadIdx.x; b <= nb; b += blockDim.x) hist[b] = 0;
    __syncthreads();
    const uint32_t lo = P.begin + ci * p.chunk;
    const uint32_t hi = min(lo + p.chunk, P.begin + P.size);
    const uint64_t* keys = w.key[cur];
    const uint32_t lane = threadIdx.x & 31u;
    for (uint32_t base = lo; base < hi; base += kClassifyThreads * kClassifyUnroll) {
        uint64_t kk[kClassifyUnroll];
#pragma unroll
        for (int u = 0; u < kClassifyUnroll; u++) {
            uint32_t e = base + u * kClassifyThreads + threadIdx.x;
            kk[u] = e < hi ? keys[e] : 0ull;
        }
#pragma unroll
        for (int u = 0; u < kClassifyUnroll; u++) {
            uint32_t e = base + u * kClassifyThreads + threadIdx.x;
            uint32_t b = e < hi ? classify_key(kk[u], t, ino, k) : nb;
            uint32_t peers = __match_any_sync(FULL_MASK, b);
            if (lane == (uint32_t)(__ffs(peers) - 1)) atomicAdd(&hist[b], (uint32_t)__popc(peers));
        }
    }
    __syncthreads();
    for (uint32_t b = threadIdx.x; b < nb; b += blockDim.x)
        w.counts[P.count_base + b * P.chunks + ci] = hist[b];
}

// ------------------------------------------------------------ scatter

constexpr int kScatterWarps = kScatterThreads / 32;
constexpr int kBucketsPerThread = (kNBMax + kScatterThreads) / kScatterThreads;  // 8

struct ScatterSmem {
    uint64_t t[kVMax + 1];
    uint64_t ino[kVMax];
    uint32_t run_pos[kNBMax + 1];
    uint32_t rdep[kNBMax + 1];
    uint16_t whist[kScatterWarps][kNBMax + 1];
};

__device__ __forceinline__ void append_child(const Work& w, uint32_t start, uint32_t size, uint32_t cdepth, bool isrun,
                                             uint32_t runlcp, uint32_t base_threshold) {
    Hdr* h = w.hdr;
    if (size <= 1) return;
    if (isrun && size > base_threshold) {
        uint32_t s = atomicAdd(&h->n_bigrun, 1u);
        if (s < w.bmax) w.bigrun[s] = Seg{start, size, cdepth, runlcp};
        else atomicOr(&h->err, kErrRunOverflow);
    } else if (size <= base_threshold) {
        uint32_t s = atomicAdd(&h->n_small, 1u);
        if (s < w.smax) { w.small[s] = Seg{start, size, cdepth, 0u}; w.small_size[s] = size; atomicAdd(&h->small_elems, size); }
        else atomicOr(&h->err, kErrSmallOverflow);
    } else {
        uint32_t s = atomicAdd(&h->n_large, 1u);
        if (s < w.lmax) w.large[s] = Seg{start, size, cdepth, 0u};
        else atomicOr(&h->err, kErrLargeOverflow);
    }
}

__global__ void __launch_bounds__(kScatterThreads) k_scatter(Work w, Params p, int cur) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ScatterSmem& sm = *reinterpret_cast<ScatterSmem*>(smem_raw);
    const uint32_t c = blockIdx.x;
    const uint32_t s = w.chunk_seg[c];
    const SegPlan P = w.plans[s];
    const uint32_t ci = c - P.chunk_base;
    const int k = (int)P.k;
    const uint32_t v = (1u << k) - 1u, nb = 2u * v + 1u;
    for (uint32_t i = threadIdx.x; i < v; i += blockDim.x) {
        sm.t[i + 1] = w.tree_lvl[P.tree_base + i];
        sm.ino[i] = w.tree_ino[P.tree_base + i];
    }
    __syncthreads();
    const uint32_t* S = w.counts_scan + P.count_base;
    const uint32_t S0 = S[0];
    const uint32_t seg_end = P.begin + P.size;
    for (uint32_t b = threadIdx.x; b <= nb; b += blockDim.x) {
        for (int q = 0; q < kScatterWarps; q++) sm.whist[q][b] = 0;
        if (b == nb) continue;
        const uint32_t start = P.begin + (S[b * P.chunks] - S0);
        const uint32_t end = (b + 1 < nb) ? P.begin + (S[(b + 1) * P.chunks] - S0) : seg_end;
        const uint32_t size = end - start;
        sm.run_pos[b] = P.begin + (S[b * P.chunks + ci] - S0);
        bool isrun = false;
        uint32_t cdepth = P.depth, runlcp = 0;
        if (b & 1u) {
            const uint64_t x = sm.ino[b >> 1];
            if (key_ends(x)) { isrun = true; runlcp = P.depth + key_chars(x); }
            else cdepth = P.depth + 8u;
        } else if (b != 0 && b != nb - 1 && size > 0) {
            const uint32_t i = b >> 1;
            cdepth = P.depth + key_lcp(sm.ino[i - 1], sm.ino[i]);
        }
        sm.rdep[b] = size == 1 ? kSingle : ((size == 0 || isrun || cdepth == P.depth) ? kNoRefill : cdepth);
        if (ci == 0 && size > 0) {
            if (start > P.begin) w.out_lcp[start] = kLcpFlag | P.depth;
            append_child(w, start, size, cdepth, isrun, runlcp, p.base_threshold);
        }
    }
    __syncthreads();

    const uint32_t lo = P.begin + ci * p.chunk;
    const uint32_t hi = min(lo + p.chunk, seg_end);
    const uint64_t* key_in = w.key[cur];
    const uint32_t* idx_in = w.idx[cur];
    uint64_t* key_out = w.key[cur ^ 1];
    uint32_t* idx_out = w.idx[cur ^ 1];
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint32_t lt = lanemask_lt();
    uint32_t nref = 0;

    for (uint32_t sub = lo; sub < hi; sub += kSubTile) {
        uint64_t kk[kScatterItems];
        uint32_t ii[kScatterItems], bb[kScatterItems], loc[kScatterItems];
        const uint32_t wbase = sub + warp * (32u * kScatterItems) + lane;
#pragma unroll
        for (int j = 0; j < kScatterItems; j++) {
            uint32_t e = wbase + j * 32u;
            bool ok = e < hi;
            kk[j] = ok ? key_in[e] : 0ull;
            ii[j] = ok ? idx_in[e] : 0u;
        }
#pragma unroll
        for (int j = 0; j < kScatterItems; j++) {
            uint32_t e = wbase + j * 32u;
            bb[j] = e < hi ? classify_key(kk[j], sm.t, sm.ino, k) : nb;
        }
#pragma unroll
        for (int j = 0; j < kScatterItems; j++) {
            const uint32_t b = bb[j];
            const uint32_t peers = __match_any_sync(FULL_MASK, b);
            const uint32_t leader = (uint32_t)__ffs(peers) - 1u;
            uint32_t off = 0;
            if (lane == leader) {
                off = sm.whist[warp][b];
                sm.whist[warp][b] = (uint16_t)(off + (uint32_t)__popc(peers));
            }
            off = __shfl_sync(FULL_MASK, off, leader);
            loc[j] = off + (uint32_t)__popc(peers & lt);
        }
        __syncthreads();
        uint32_t accs[kBucketsPerThread];
#pragma unroll
        for (int q = 0; q < kBucketsPerThread; q++) {
            const uint32_t b = threadIdx.x + q * kScatterThreads;
            uint32_t acc = 0;
            if (b < nb) {
#pragma unroll
                for (int ww = 0; ww < kScatterWarps; ww++) {
                    uint32_t cnt = sm.whist[ww][b];
                    sm.whist[ww][b] = (uint16_t)acc;
                    acc += cnt;
                }
            }
            accs[q] = acc;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kScatterItems; j++) {
            const uint32_t e = wbase + j * 32u;
            if (e < hi) {
                const uint32_t b = bb[j];
                const uint32_t pos = sm.run_pos[b] + sm.whist[warp][b] + loc[j];
                const uint32_t rd = sm.rdep[b];
                if (pos >= seg_end) {
                    atomicOr(&w.hdr->err, kErrPosition);
                } else if (rd == kSingle) {
                    w.out_perm[pos] = ii[j];
                } else {
                    idx_out[pos] = ii[j];
                    key_out[pos] = rd == kNoRefill ? kk[j] : load_key(w.chars, w.offsets[ii[j]] + rd);
                    nref += rd != kNoRefill;
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < kBucketsPerThread; q++) {
            const uint32_t b = threadIdx.x + q * kScatterThreads;
            if (b < nb) {
                sm.run_pos[b] += accs[q];
#pragma unroll
                for (int ww = 0; ww < kScatterWarps; ww++) sm.whist[ww][b] = 0;
            } else if (b == nb) {
#pragma unroll
                for (int ww = 0; ww < kScatterWarps; ww++) sm.whist[ww][b] = 0;
            }
        }
        __syncthreads();
    }
    nref = __reduce_add_sync(FULL_MASK, nref);
    if (lane == 0 && nref) atomicAdd(&w.hdr->refills, (unsigned long long)nref);
}

// ------------------------------------------------------------ base case

constexpr int kBaseThreads = 512;

struct BaseSmem {
    uint64_t K[kBaseCap];
    uint32_t I[kBaseCap];
    uint32_t G[kBaseCap];   // output position of each slot
    uint32_t D[kBaseCap];   // depth of the run a slot belongs to
    uint32_t H[kBaseCap];   // run heads / scan
    uint32_t SB[kBaseMax + 2];  // slot base of each segment of the tile
    uint16_t R[kBaseCap];   // run id (first slot of the run) carried with the element
    uint32_t wsum[33];
};

__device__ __forceinline__ uint32_t upper_bound_u32(const uint32_t* a, uint32_t n, uint32_t x) {
    uint32_t lo = 0, hi = n;
    while (lo < hi) {
        uint32_t m = (lo + hi) >> 1;
        if (a[m] <= x) lo = m + 1; else hi = m;
    }
    return lo;
}

__device__ __forceinline__ uint32_t lower_bound_u32(const uint32_t* a, uint32_t n, uint32_t x) {
    uint32_t lo = 0, hi = n;
    while (lo < hi) {
        uint32_t m = (lo + hi) >> 1;
        if (a[m] < x) lo = m + 1; else hi = m;
    }
    return lo;
}

__device__ __forceinline__ bool base_less(const BaseSmem& sm, uint32_t a, uint32_t b) {
    if (sm.R[a] != sm.R[b]) return sm.R[a] < sm.R[b];
    if (sm.K[a] != sm.K[b]) return sm.K[a] < sm.K[b];
    return sm.I[a] < sm.I[b];
}

// Inclusive max-scan of H[0..cnt) in place; blocked, 8 slots per thread.
__device__ void block_max_scan(uint32_t* H, uint32_t cnt, uint32_t* wsum) {
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    constexpr int kPer = kBaseCap / kBaseThreads;
    uint32_t v[kPer];
    uint32_t run = 0;
#pragma unroll
    for (int j = 0; j < kPer; j++) {
        uint32_t i = threadIdx.x * kPer + j;
        uint32_t x = i < cnt ? H[i] : 0u;
        run = max(run, x);
        v[j] = run;
    }
    uint32_t inc = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(FULL_MASK, inc, o);
        if (lane >= (uint32_t)o) inc = max(inc, y);
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint32_t s = lane < nw ? wsum[lane] : 0u;
        uint32_t si = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(FULL_MASK, si, o);
            if (lane >= (uint32_t)o) si = max(si, y);
        }
        uint32_t ex = __shfl_up_sync(FULL_MASK, si, 1);
        if (lane < nw) wsum[lane] = lane ? ex : 0u;
    }
    __syncthreads();
    uint32_t ex_in_warp = __shfl_up_sync(FULL_MASK, inc, 1);
    if (lane == 0) ex_in_warp = 0;
    const uint32_t prefix = max(wsum[warp], ex_in_warp);
#pragma unroll
    for (int j = 0; j < kPer; j++) {
        uint32_t i = threadIdx.x * kPer + j;
        if (i < cnt) H[i] = max(prefix, v[j]);
    }
    __syncthreads();
}

// One CTA per tile of packed small segments: segments whose packed start lies
// in [t*T, (t+1)*T) (T = base_threshold), at most 2T - 1 strings.  Sorts
// each segment by (key word at its depth, index); runs of equal key words
// without terminator move 8 bytes deeper and are sorted again, until every
// run is decided.  Writes out_perm and the LCP of every slot but a
// segment's first.
__global__ void __launch_bounds__(kBaseThreads) k_base(Work w, Params p, int buf, uint32_t ns, uint32_t total) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BaseSmem& sm = *reinterpret_cast<BaseSmem*>(smem_raw);
    const uint32_t T = p.base_threshold;
    const uint32_t t0 = blockIdx.x * T;
    if (t0 >= total) return;
    const uint32_t t1 = min(t0 + T, total);
    const uint32_t lo = lower_bound_u32(w.small_off, ns, t0);
    const uint32_t hi = lower_bound_u32(w.small_off, ns, t1);
    if (lo >= hi) return;
    const uint32_t slot0 = w.small_off[lo];
    const uint32_t cnt = (hi < ns ? w.small_off[hi] : total) - slot0;
    const uint32_t nseg = hi - lo;
    for (uint32_t i = threadIdx.x; i < nseg; i += blockDim.x) sm.SB[i] = w.small_off[lo + i] - slot0;
    __syncthreads();
    const uint64_t* key_in = w.key[buf];
    const uint32_t* idx_in = w.idx[buf];
    uint32_t pw = 1;
    while (pw < cnt) pw <<= 1;
    for (uint32_t q = threadIdx.x; q < pw; q += blockDim.x) {
        if (q < cnt) {
            const uint32_t i = upper_bound_u32(sm.SB, nseg, q) - 1u;
            const Seg g = w.small[lo + i];
            const uint32_t r = q - sm.SB[i];
            sm.G[q] = g.begin + r;
            sm.D[q] = g.depth;
            sm.R[q] = (uint16_t)sm.SB[i];
            sm.K[q] = key_in[g.begin + r];
            sm.I[q] = idx_in[g.begin + r];
        } else {
            sm.R[q] = 0xFFFFu;
            sm.K[q] = ~0ull;
            sm.I[q] = 0xFFFFFFFFu;
        }
    }
    __syncthreads();
    for (uint32_t iter = 0;; iter++) {
        if (iter >= kBaseMaxIters) {  // never expected: strings end, so runs end
            if (threadIdx.x == 0) atomicOr(&w.hdr->err, kErrBaseIters);
            return;
        }
        // segmented sort: (run, key, index) order keeps every run in its slots
        for (uint32_t size = 2; size <= pw; size <<= 1) {
            for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
                for (uint32_t i = threadIdx.x; i < pw / 2; i += blockDim.x) {
                    const uint32_t a = 2u * i - (i & (stride - 1u));
                    const uint32_t b = a + stride;
                    const bool asc = (a & size) == 0;
                    if (base_less(sm, b, a) == asc) {
                        uint64_t tk = sm.K[a]; sm.K[a] = sm.K[b]; sm.K[b] = tk;
                        uint32_t ti = sm.I[a]; sm.I[a] = sm.I[b]; sm.I[b] = ti;
                        uint16_t tr = sm.R[a]; sm.R[a] = sm.R[b]; sm.R[b] = tr;
                    }
                }
                __syncthreads();
            }
        }
        // decide neighbours: a key change fixes the LCP; equal keys holding the
        // terminator are equal strings; equal keys without it stay in a run
        for (uint32_t q = threadIdx.x; q < cnt; q += blockDim.x) {
            bool head = true;
            if (q != sm.R[q]) {
                const uint64_t a = sm.K[q - 1], b = sm.K[q];
                if (a != b) {
                    w.out_lcp[sm.G[q]] = sm.D[q] + key_lcp(a, b);
                } else {
                    head = false;
                    if (key_ends(b)) w.out_lcp[sm.G[q]] = sm.D[q] + key_chars(b);
                }
            }
            sm.H[q] = head ? q : 0u;
        }
        __syncthreads();
        block_max_scan(sm.H, cnt, sm.wsum);
        bool any = false;
        for (uint32_t q = threadIdx.x; q < cnt; q += blockDim.x) {
            const uint32_t head = sm.H[q];
            const bool multi = (q != head) || (q + 1 < cnt && sm.H[q + 1] == q);
            const bool act = multi && !key_ends(sm.K[q]);
            if (act) {
                const uint32_t d = sm.D[q] + 8u;
                sm.D[q] = d;
                sm.K[q] = load_key(w.chars, w.offsets[sm.I[q]] + d);
                sm.R[q] = (uint16_t)head;
                any = true;
            } else {
                sm.R[q] = (uint16_t)q;
            }
        }
        if (!__syncthreads_or(any)) break;
    }
    for (uint32_t q = threadIdx.x; q < cnt; q += blockDim.x) w.out_perm[sm.G[q]] = sm.I[q];
}

// Buckets too large for the base case whose strings are all equal.
__global__ void k_bigrun(Work w, int buf, uint32_t nrun) {
    for (uint32_t r = blockIdx.x; r < nrun; r += gridDim.x) {
        const Seg g = w.bigrun[r];
        for (uint32_t i = threadIdx.x; i < g.size; i += blockDim.x) {
            const uint32_t q = g.begin + i;
            w.out_perm[q] = w.idx[buf][q];
            if (i > 0) w.out_lcp[q] = g.aux;
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
            const uint64_t a = load_key(w.chars, w.offsets[pa] + l);
            const uint64_t b = load_key(w.chars, w.offsets[pb] + l);
            if (a == b) atomicOr(&w.hdr->err, kErrEqualBoundary);
            w.out_lcp[q] = l + (a == b ? 8u : key_lcp(a, b));
        }
    }
}

// ------------------------------------------------------------ scan (3 phase)

constexpr int kScanThreads = 256;
constexpr int kScanPer = 16;
constexpr uint32_t kScanTile = kScanThreads * kScanPer;

size_t scan_tmp_elems(uint32_t n) { return (size_t)(n + kScanTile - 1) / kScanTile + 1; }

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t* in, uint32_t n, uint32_t* sums) {
    __shared__ uint32_t wsum[33];
    const uint32_t base = blockIdx.x * kScanTile;
    uint32_t s = 0;
#pragma unroll
    for (int j = 0; j < kScanPer; j++) {
        uint32_t i = base + j * kScanThreads + threadIdx.x;
        if (i < n) s += in[i];
    }
    uint32_t tot;
    block_excl_sum(s, wsum, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_scan_tiles(uint32_t* sums, uint32_t ntiles, uint32_t* total_out) {
    __shared__ uint32_t wsum[33];
    const uint32_t per = (ntiles + blockDim.x - 1) / blockDim.x;
    const uint32_t lo = min(ntiles, threadIdx.x * per), hi = min(ntiles, lo + per);
    uint32_t s = 0;
    for (uint32_t i = lo; i < hi; i++) s += sums[i];
    uint32_t tot;
    uint32_t ex = block_excl_sum(s, wsum, &tot);
    for (uint32_t i = lo; i < hi; i++) {
        uint32_t x = sums[i];
        sums[i] = ex;
        ex += x;
    }
    if (threadIdx.x == 0) *total_out = tot;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_down(const uint32_t* in, uint32_t* out, uint32_t n,
                                                            const uint32_t* sums) {
    __shared__ uint32_t wsum[33];
    const uint32_t base = blockIdx.x * kScanTile + threadIdx.x * kScanPer;
    uint32_t v[kScanPer];
    uint32_t s = 0;
#pragma unroll
    for (int j = 0; j < kScanPer; j++) {
        uint32_t i = base + j;
        v[j] = i < n ? in[i] : 0u;
        s += v[j];
    }
    uint32_t ex = block_excl_sum(s, wsum, nullptr) + sums[blockIdx.x];
#pragma unroll
    for (int j = 0; j < kScanPer; j++) {
        uint32_t i = base + j;
        if (i < n) out[i] = ex;
        ex += v[j];
    }
}

// out[0..n) = exclusive prefix sums of in, out[n] = total.  tmp holds
// scan_tmp_elems(n) entries.
cudaError_t launch_scan_u32(const uint32_t* in, uint32_t* out, uint32_t n, uint32_t* tmp, Prof* pf,
                            cudaStream_t st) {
    if (n == 0) return cudaMemsetAsync(out, 0, sizeof(uint32_t), st);
    const uint32_t tiles = (n + kScanTile - 1) / kScanTile;
    ProfScope ps(pf, kScan, st);
    k_scan_reduce<<<tiles, kScanThreads, 0, st>>>(in, n, tmp);
    k_scan_tiles<<<1, 1024, 0, st>>>(tmp, tiles, out + n);
    k_scan_down<<<tiles, kScanThreads, 0, st>>>(in, out, n, tmp);
    if (pf) { pf->launches += 2; pf->cls_launches[kScan] += 2; }
    return cudaGetLastError();
}

// ------------------------------------------------------------ launches

static int g_num_sms = 0;

static int num_sms() {
    if (!g_num_sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_num_sms <= 0) g_num_sms = 148;
    }
    return g_num_sms;
}

static uint32_t grid_for(uint64_t n, uint32_t threads, uint32_t per_sm) {
    uint64_t g = (n + threads - 1) / threads;
    uint64_t cap = (uint64_t)num_sms() * per_sm;
    if (g > cap) g = cap;
    return g ? (uint32_t)g : 1u;
}

cudaError_t launch_init(const Work& w, Prof* pf, cudaStream_t st) {
    if (w.n) {
        // the shadow index array only ever holds valid string indices
        cudaError_t e = cudaMemsetAsync(w.idx[1], 0, sizeof(uint32_t) * (size_t)w.n, st);
        if (e != cudaSuccess) return e;
        ProfScope ps(pf, kInit, st);
        k_init<<<grid_for(w.n, 256, 16), 256, 0, st>>>(w);
    }
    return cudaGetLastError();
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
            k_roots<<<grid_for(num_roots, 256, 4), 256, 0, st>>>(w, roots, num_roots, Seg{}, p.base_threshold);
    } else {
        k_roots<<<1, 32, 0, st>>>(w, nullptr, 1u, Seg{0u, w.n, 0u, 0u}, p.base_threshold);
    }
    return cudaGetLastError();
}

cudaError_t launch_plan(const Work& w, const Params& p, Prof* pf, cudaStream_t st) {
    ProfScope ps(pf, kPlan, st);
    k_plan<<<1, 1024, 0, st>>>(w, p);
    return cudaGetLastError();
}

cudaError_t launch_round(const Work& w, const Params& p, int cur, uint32_t L, uint32_t total_chunks,
                         uint32_t total_counts, Prof* pf, cudaStream_t st) {
    cudaFuncSetAttribute(k_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(ScatterSmem));
    {
        ProfScope ps(pf, kSample, st);
        k_sample<<<L, 1024, 0, st>>>(w, p, cur);
    }
    {
        ProfScope ps(pf, kClassify, st);
        k_classify<<<total_chunks, kClassifyThreads, 0, st>>>(w, p, cur);
    }
    cudaError_t e = launch_scan_u32(w.counts, w.counts_scan, total_counts, w.scan_tmp, pf, st);
    if (e != cudaSuccess) return e;
    {
        ProfScope ps(pf, kScatter, st);
        k_scatter<<<total_chunks, kScatterThreads, sizeof(ScatterSmem), st>>>(w, p, cur);
    }
    return cudaGetLastError();
}

cudaError_t launch_small(const Work& w, const Params& p, int buf, uint32_t n_small, uint32_t n_bigrun,
                         uint32_t small_total, uint32_t* out_tiles, Prof* pf, cudaStream_t st) {
    cudaFuncSetAttribute(k_base, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(BaseSmem));
    uint32_t tiles = 0;
    if (n_small) {
        cudaError_t e = launch_scan_u32(w.small_size, w.small_off, n_small, w.scan_tmp, pf, st);
        if (e != cudaSuccess) return e;
        tiles = (small_total + p.base_threshold - 1) / p.base_threshold;
        ProfScope ps(pf, kBase, st);
        k_base<<<tiles, kBaseThreads, sizeof(BaseSmem), st>>>(w, p, buf, n_small, small_total);
    }
    if (n_bigrun) {
        ProfScope ps(pf, kRuns, st);
        k_bigrun<<<grid_for((uint64_t)n_bigrun * 256, 256, 4), 256, 0, st>>>(w, buf, n_bigrun);
    }
    if (out_tiles) *out_tiles = tiles;
    return cudaGetLastError();
}

cudaError_t launch_fixup(const Work& w, Prof* pf, cudaStream_t st) {
    if (w.n > 1) {
        ProfScope ps(pf, kFixup, st);
        k_fixup<<<grid_for(w.n, 256, 16), 256, 0, st>>>(w);
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
    if (n) k_gather_keys<<<grid_for(n, 256, 16), 256, 0, st>>>(chars, offsets, idx, depth, n, out);
    return cudaGetLastError();
}

cudaError_t launch_build_splitters(const uint64_t* sample, uint32_t count, int k, uint64_t* lvl, uint64_t* ino,
                                   cudaStream_t st) {
    k_build_splitters<<<1, 1024, 0, st>>>(sample, count, k, lvl, ino);
    return cudaGetLastError();
}

__global__ void k_classify_keys(const uint64_t* keys, uint32_t n, const uint64_t* lvl, const uint64_t* inorder,
                                int k, uint16_t* out) {
    __shared__ uint64_t t[kVMax + 1];
    __shared__ uint64_t ino[kVMax];
    const uint32_t v = (1u << k) - 1u;
    for (uint32_t i = threadIdx.x; i < v; i += blockDim.x) { t[i + 1] = lvl[i]; ino[i] = inorder[i]; }
    __syncthreads();
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        out[i] = (uint16_t)classify_key(keys[i], t, ino, k);
}

cudaError_t launch_classify(const uint64_t* keys, uint32_t n, const uint64_t* lvl, const uint64_t* ino, int k,
                            uint16_t* out, cudaStream_t st) {
    if (n) k_classify_keys<<<grid_for(n, 256, 8), 256, 0, st>>>(keys, n, lvl, ino, k, out);
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
        k_localize<<<grid_for((uint64_t)num_roots * 256, 256, 8), 256, 0, st>>>(perm, roots, num_roots);
    }
    return cudaGetLastError();
}

}  // namespace sss
