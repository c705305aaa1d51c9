// Learned bucket proposal: a monotone piecewise-linear CDF of a segment's
// key words, fitted on a sample of the segment (0.1 % of its strings, at
// least 2,048 and at most 65,536 keys) with hand-written forward and
// backward passes and Adam, all in FP32 on one CTA per segment.  (An
// addition to the paper; its closest idea is the jump tables of App. A.2
// that replace part of the splitter-tree descent.)
//
// Model with M pieces over the input coordinate t in [0, M] (cdf_coord:
// piece m is [m, m + 1)): increments d_j = softplus(theta_j), T = sum_j d_j,
// knots C_j = (d_0 + ... + d_{j-1}) / T, and for a key in piece m with
// fraction f: F = C_m + f d_m / T.  Loss: mean over the sample of
// (F_s - y_s)^2 with y_s = (j_s + 1/2) / (v + 1), j_s the number of
// splitters below sample key s (the splitter interval the tree gives it), so
// that floor(F (v + 1)) proposes that interval.  Gradient, term by term:
//   dF_s/dd_j = ([j < m_s] + f_s [j = m_s]) / T - F_s / T
//   dL/dd_j   = (sum_{s: m_s > j} g_s + sum_{s: m_s = j} g_s f_s - sum_s g_s F_s) / T,
//               g_s = 2 (F_s - y_s) / S
//   dL/dtheta_j = dL/dd_j * sigmoid(theta_j)
// Inside piece m, with a = C_m and b = d_m / T, F_s = a + b f_s, so every
// sum over the samples of a piece is a polynomial in a and b whose
// coefficients are the piece's sample statistics n_m, sum f, sum f^2,
// sum y and sum y f:
//   sum_{s in m} g_s       = (2/S) (n a + b sum f - sum y)
//   sum_{s in m} g_s f_s   = (2/S) (a sum f + b sum f^2 - sum y f)
//   sum_{s in m} g_s F_s   = (2/S) (n a^2 + 2 a b sum f + b^2 sum f^2 - a sum y - b sum y f)
// The statistics are gathered once per fit; each Adam step then costs O(M)
// whatever the sample size.
#include "sss_internal.cuh"

namespace sss {

constexpr int kFitThreads = 1024;

__device__ __forceinline__ float softplus_f(float t) { return t > 20.0f ? t : log1pf(expf(t)); }
__device__ __forceinline__ float sigmoid_f(float t) { return 1.0f / (1.0f + expf(-t)); }

// Exclusive prefix sums of a[0..n) in place (blockDim.x threads, a multiple
// of 32); returns the total.  wsum: 33 floats of shared scratch.
__device__ float block_excl_scan_f(float* a, uint32_t n, float* wsum) {
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const uint32_t per = (n + blockDim.x - 1) / blockDim.x;
    const uint32_t lo = min(n, threadIdx.x * per), hi = min(n, lo + per);
    float x = 0.0f;
    for (uint32_t i = lo; i < hi; i++) x += a[i];
    float inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float y = __shfl_up_sync(0xFFFFFFFFu, inc, o);
        if (lane >= (uint32_t)o) inc += y;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const float s = lane < nw ? wsum[lane] : 0.0f;
        float si = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const float y = __shfl_up_sync(0xFFFFFFFFu, si, o);
            if (lane >= (uint32_t)o) si += y;
        }
        if (lane < nw) wsum[lane] = si - s;
        if (lane == nw - 1) wsum[32] = si;
    }
    __syncthreads();
    float ex = wsum[warp] + inc - x;
    const float total = wsum[32];
    for (uint32_t i = lo; i < hi; i++) {
        const float v = a[i];
        a[i] = ex;
        ex += v;
    }
    __syncthreads();
    return total;
}

// Shared-memory arrays of one fit (M pieces).
struct CdfShared {
    float *theta, *m1, *m2, *P, *grad, *D;  // [M] each, P has M + 1, m1 and m2 M + 2; D = softplus(theta)
    float *sn, *sf, *sff, *sy, *syf;    // [M] per-piece sample statistics
    float* wsum;                        // [33]
    float* red;                         // [4]
};

__device__ __forceinline__ CdfShared carve(float* base, uint32_t M) {
    CdfShared c;
    float* p = base;
    c.theta = p; p += M;
    c.m1 = p; p += M + 2;
    c.m2 = p; p += M + 2;
    c.P = p; p += M + 1;
    c.grad = p; p += M;
    c.D = p; p += M;
    c.sn = p; p += M;
    c.sf = p; p += M;
    c.sff = p; p += M;
    c.sy = p; p += M;
    c.syf = p; p += M;
    c.wsum = p; p += 33;
    c.red = p;
    return c;
}

__host__ __device__ constexpr size_t cdf_floats(uint32_t M) { return (size_t)11 * M + 5 + 33 + 4; }

// Fit kernel's extra shared memory after the float arrays: the splitters,
// the digit groups' counts and largest keys, and the input coordinate.
struct FitExtra {
    uint64_t ino[kVMax];
    uint64_t gmax[256];
    uint32_t cnt[256];
    CdfNorm nrm;
    unsigned long long kmin, kmax;
};

static size_t align_up_16(size_t x) { return (x + 15) / 16 * 16; }

size_t cdf_fit_smem(uint32_t M) { return align_up_16(sizeof(float) * cdf_floats(M)) + sizeof(FitExtra); }

// Piece and fraction of input coordinate t in [0, M].
__device__ __forceinline__ void cdf_place(float t, uint32_t M, int& m, float& f) {
    const uint32_t mm = min((uint32_t)fmaxf(t, 0.0f), M - 1u);
    m = (int)mm;
    f = fminf(1.0f, fmaxf(0.0f, t - (float)mm));
}

__device__ __forceinline__ void zero_stats(const CdfShared& c, uint32_t M) {
    for (uint32_t j = threadIdx.x; j < M; j += blockDim.x) {
        c.sn[j] = 0.0f; c.sf[j] = 0.0f; c.sff[j] = 0.0f; c.sy[j] = 0.0f; c.syf[j] = 0.0f;
    }
}

// One sample per lane (piece m, fraction f, target y; m < 0: none) into
// the piece statistics.  Called by all lanes of a warp.  Samples of one
// key value share a piece, and one value can hold most of a sample (the
// word "http://w" of URLs): when the whole warp has one piece, its sums are
// reduced by shuffles and added once, instead of 32 atomics on one address.
__device__ __forceinline__ void add_stats_warp(const CdfShared& c, int m, float f, float y) {
    const uint32_t peers = __match_any_sync(0xFFFFFFFFu, m);
    if (peers == 0xFFFFFFFFu) {
        if (m < 0) return;
        float n = 1.0f, sf = f, sff = f * f, sy = y, syf = y * f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            n += __shfl_xor_sync(0xFFFFFFFFu, n, o);
            sf += __shfl_xor_sync(0xFFFFFFFFu, sf, o);
            sff += __shfl_xor_sync(0xFFFFFFFFu, sff, o);
            sy += __shfl_xor_sync(0xFFFFFFFFu, sy, o);
            syf += __shfl_xor_sync(0xFFFFFFFFu, syf, o);
        }
        if ((threadIdx.x & 31u) == 0) {
            atomicAdd(&c.sn[m], n);
            atomicAdd(&c.sf[m], sf);
            atomicAdd(&c.sff[m], sff);
            atomicAdd(&c.sy[m], sy);
            atomicAdd(&c.syf[m], syf);
        }
    } else if (m >= 0) {
        atomicAdd(&c.sn[m], 1.0f);
        atomicAdd(&c.sf[m], f);
        atomicAdd(&c.sff[m], f * f);
        atomicAdd(&c.sy[m], y);
        atomicAdd(&c.syf[m], y * f);
    }
}

// Knots of the current parameters: D[j] = d_j, P[j] = d_0 + ... + d_{j-1};
// returns T.
__device__ float cdf_knots(const CdfShared& c, uint32_t M) {
    for (uint32_t j = threadIdx.x; j < M; j += blockDim.x) {
        const float d = softplus_f(c.theta[j]);
        c.D[j] = d;
        c.P[j] = d;
    }
    __syncthreads();
    return block_excl_scan_f(c.P, M, c.wsum);
}

// dL/dtheta into c.grad from the piece statistics of S samples (see the
// file comment), for the parameters in c.theta.  Leaves the unnormalised
// knots in c.P; returns T.  Ends synchronised.
__device__ float cdf_grad_stats(const CdfShared& c, uint32_t M, float S) {
    const uint32_t lane = threadIdx.x & 31u;
    if (threadIdx.x == 0) c.red[0] = 0.0f;
    const float T = cdf_knots(c, M);
    const float invT = 1.0f / T, k2 = 2.0f / S;
    float gF = 0.0f;
    for (uint32_t m = threadIdx.x; m < M; m += blockDim.x) {
        const float a = c.P[m] * invT, b = c.D[m] * invT;
        const float n = c.sn[m], sf = c.sf[m], sff = c.sff[m], sy = c.sy[m], syf = c.syf[m];
        c.grad[m] = k2 * (n * a + b * sf - sy);  // sum of g over the piece
        gF += k2 * (n * a * a + 2.0f * a * b * sf + b * b * sff - a * sy - b * syf);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) gF += __shfl_xor_sync(0xFFFFFFFFu, gF, o);
    if (lane == 0) atomicAdd(&c.red[0], gF);
    __syncthreads();
    const float totG = block_excl_scan_f(c.grad, M, c.wsum);  // grad[m] = G_0 + ... + G_{m-1}
    const float G = c.red[0];
    for (uint32_t m = threadIdx.x; m < M; m += blockDim.x) {
        const float a = c.P[m] * invT, b = c.D[m] * invT;
        const float n = c.sn[m], sf = c.sf[m], sff = c.sff[m], sy = c.sy[m], syf = c.syf[m];
        const float Gm = k2 * (n * a + b * sf - sy);
        const float Hm = k2 * (a * sf + b * sff - syf);
        const float suffix = totG - c.grad[m] - Gm;  // G_{m+1} + ... + G_{M-1}
        c.grad[m] = (suffix + Hm - G) * invT * sigmoid_f(c.theta[m]);
    }
    __syncthreads();
    return T;
}

// Starting parameters of a fit: the piecewise-linear function through one
// point per piece that holds samples, (mean t, mean target) of its samples,
// and (0, 0), (M, 1) at the ends, read at the knots; theta_j =
// softplus^-1 of its increments (at least 1e-6).  The points rise with t
// (targets do not decrease with the key), so the start is monotone, and a
// piece whose samples are one key value gets that key's target exactly.
// Uses c.grad, c.m1 and c.m2 as scratch and leaves m1 = m2 = 0 for Adam.
__device__ void cdf_start_from_points(const CdfShared& c, uint32_t M) {
    for (uint32_t m = threadIdx.x; m < M; m += blockDim.x) c.grad[m] = c.sn[m] > 0.0f ? 1.0f : 0.0f;
    __syncthreads();
    const uint32_t np = (uint32_t)block_excl_scan_f(c.grad, M, c.wsum);  // grad[m]: rank among the pieces with samples
    for (uint32_t m = threadIdx.x; m < M; m += blockDim.x) {
        const float n = c.sn[m];
        if (n > 0.0f) {
            const uint32_t q = (uint32_t)c.grad[m] + 1u;
            c.m1[q] = (float)m + c.sf[m] / n;
            c.m2[q] = c.sy[m] / n;
        }
    }
    if (threadIdx.x == 0) {
        c.m1[0] = 0.0f;
        c.m2[0] = 0.0f;
        c.m1[np + 1] = (float)M;
        c.m2[np + 1] = 1.0f;
    }
    __syncthreads();
    for (uint32_t j = threadIdx.x; j <= M; j += blockDim.x) {
        // the last point at or before knot j, then the line to the next one
        uint32_t a = 0, b = np + 1;
        while (a < b) {
            const uint32_t mid = (a + b + 1) >> 1;
            if (c.m1[mid] <= (float)j) a = mid; else b = mid - 1;
        }
        float y = c.m2[a];
        if (a < np + 1) {
            const float t0 = c.m1[a], t1 = c.m1[a + 1];
            const float r = t1 > t0 ? ((float)j - t0) / (t1 - t0) : 0.0f;
            y = c.m2[a] + fminf(1.0f, fmaxf(0.0f, r)) * (c.m2[a + 1] - c.m2[a]);
        }
        c.P[j] = y;
    }
    __syncthreads();
    for (uint32_t j = threadIdx.x; j < M; j += blockDim.x) {
        const float d = fmaxf(c.P[j + 1] - c.P[j], 1e-6f);
        c.theta[j] = d > 20.0f ? d : logf(expm1f(d));
    }
    __syncthreads();
    for (uint32_t j = threadIdx.x; j < M + 2; j += blockDim.x) {
        c.m1[j] = 0.0f;
        c.m2[j] = 0.0f;
    }
    __syncthreads();
}

constexpr uint32_t kFitMinSample = 2048;   // keys of the smallest fit sample
constexpr uint32_t kFitMaxSample = 65536;  // keys of the largest (0.1 % of a 64M-string segment)

// Position j of a segment's fit sample (a seeded hash, like the splitter
// sample but drawn independently of it).
__device__ __forceinline__ uint32_t fit_pos(uint64_t seed, uint32_t begin, uint32_t size, uint32_t j) {
    const uint64_t base = seed ^ ((uint64_t)begin * 0x9E3779B97F4A7C15ull) ^ ((uint64_t)size << 32);
    const uint32_t r = (uint32_t)(mix64(base + (uint64_t)j * 0xD1B54A32D192ED03ull) >> 32);
    return (uint32_t)(((uint64_t)r * size) >> 32);
}

__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(0xFFFFFFFFu, x, o);
        x = y < x ? y : x;
    }
    return x;
}
__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(0xFFFFFFFFu, x, o);
        x = y > x ? y : x;
    }
    return x;
}

__device__ __forceinline__ FitExtra& fit_extra(float* base, uint32_t M) {
    return *reinterpret_cast<FitExtra*>(reinterpret_cast<char*>(base) + ((sizeof(float) * cdf_floats(M) + 15) & ~(size_t)15));
}

// One CTA per planned segment of at least kLearnedMinSize strings: draw
// the fit sample, derive the model's input coordinate (cdf_coord) from it,
// gather the piece statistics, fit the model and store its knots and input
// coordinate.
__global__ void __launch_bounds__(kFitThreads) k_cdf_fit(Work w, Params p) {
    extern __shared__ __align__(16) float fit_smem[];
    const uint32_t M = p.cdf_M;
    const CdfShared c = carve(fit_smem, M);
    FitExtra& X = fit_extra(fit_smem, M);
    const uint32_t L = w.hdr->L;
    const Rec* recs = w.rec[w.hdr->round & 1u];
    const uint32_t tid = threadIdx.x, lane = tid & 31u;
    const uint64_t sseed = p.seed ^ 0x6C8E9CF570932BD5ull;
    __shared__ uint32_t s_item;
    for (uint32_t seg = first_item(); seg < L; seg = next_item(&w.hdr->q_fit, &s_item)) {
    const SegPlan P = w.plans[seg];
    if (P.size < kLearnedMinSize) continue;
    const uint32_t v = (1u << P.k) - 1u;
    const uint32_t S = min(kFitMaxSample, max(kFitMinSample, P.size / 1000u));
    for (uint32_t i = tid; i < v; i += blockDim.x) X.ino[i] = w.tree_ino[P.tree_base + i];
    for (uint32_t d = tid; d < 256; d += blockDim.x) {
        X.cnt[d] = 0;
        X.gmax[d] = 0ull;
        X.nrm.gmin[d] = ~0ull;
    }
    if (tid == 0) {
        X.kmin = ~0ull;
        X.kmax = 0ull;
    }
    zero_stats(c, M);
    __syncthreads();
    // 1. the sample's smallest and largest keys: the shared leading bytes c
    {
        unsigned long long lo = ~0ull, hi = 0ull;
        for (uint32_t s = tid; s < S; s += blockDim.x) {
            const unsigned long long key = recs[P.begin + fit_pos(sseed, P.begin, P.size, s)].key;
            lo = key < lo ? key : lo;
            hi = key > hi ? key : hi;
        }
        lo = warp_min_u64(lo);
        hi = warp_max_u64(hi);
        if (lane == 0) {
            atomicMin(&X.kmin, lo);
            atomicMax(&X.kmax, hi);
        }
    }
    __syncthreads();
    const uint64_t kmin = X.kmin, kmax = X.kmax;
    const uint32_t cb = kmin == kmax ? 8u : (uint32_t)__clzll((long long)(kmin ^ kmax)) >> 3;
    // 2. the digit groups: keys, smallest and largest key of each
    if (cb < 8u) {
        for (uint32_t s0 = tid & ~31u; s0 < S; s0 += blockDim.x) {  // whole warps
            const uint32_t s = s0 + lane;
            unsigned long long key = 0ull;
            uint32_t d = 256u;
            if (s < S) {
                key = recs[P.begin + fit_pos(sseed, P.begin, P.size, s)].key;
                d = (uint32_t)(key >> (56u - 8u * cb)) & 0xFFu;
            }
            // one digit for the whole warp (most of a URL sample): one update
            const uint32_t peers = __match_any_sync(0xFFFFFFFFu, d);
            if (peers == 0xFFFFFFFFu) {
                const unsigned long long lo = warp_min_u64(key), hi = warp_max_u64(key);
                if (lane == 0 && d < 256u) {
                    atomicAdd(&X.cnt[d], 32u);
                    atomicMin(reinterpret_cast<unsigned long long*>(&X.nrm.gmin[d]), lo);
                    atomicMax(reinterpret_cast<unsigned long long*>(&X.gmax[d]), hi);
                }
            } else if (d < 256u) {
                atomicAdd(&X.cnt[d], 1u);
                atomicMin(reinterpret_cast<unsigned long long*>(&X.nrm.gmin[d]), key);
                atomicMax(reinterpret_cast<unsigned long long*>(&X.gmax[d]), key);
            }
        }
    }
    __syncthreads();
    // pieces of each group: one, plus a share of the rest proportional to
    // the group's keys; what rounding leaves goes to the largest group.  One
    // thread a digit group; the first piece of each group is a prefix sum.
    {
        const uint32_t cnt = tid < 256u ? X.cnt[tid] : 0u;
        const uint32_t G = (uint32_t)__syncthreads_count(cnt > 0u);  // groups with sample keys
        const bool one_each = G <= M;
        const uint32_t spare = one_each ? M - G : M;
        const uint32_t K = cnt ? (one_each ? 1u : 0u) + (spare * cnt) / S : 0u;  // spare * cnt < 2^28
        if (tid == 0) {
            X.kmin = 0ull;  // reused: largest group (count, digit) and total pieces
            X.kmax = 0ull;
        }
        __syncthreads();
        if (tid < 256u && cnt) {
            atomicMax(&X.kmin, ((unsigned long long)cnt << 8) | tid);
            atomicAdd(&X.kmax, (unsigned long long)K);
        }
        // exclusive prefix of K over the 256 digits (warps 0-7)
        uint32_t inc = K;
        const uint32_t w8 = tid >> 5;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, inc, o);
            if (lane >= (uint32_t)o) inc += y;
        }
        __shared__ uint32_t wtot[8];
        if (tid < 256u && lane == 31u) wtot[w8] = inc;
        __syncthreads();
        if (tid < 256u) {
            uint32_t before = 0;
            for (uint32_t q = 0; q < w8; q++) before += wtot[q];
            const uint32_t big = (uint32_t)(X.kmin & 0xFFull);
            const uint32_t rem = M - (uint32_t)X.kmax;
            X.nrm.O[tid] = (uint16_t)(before + inc - K + (tid > big ? rem : 0u));
        }
        if (tid == 0) {
            X.nrm.kmin = kmin;
            X.nrm.kmax = kmax;
            X.nrm.c = cb;
            X.nrm.pad = 0;
            X.nrm.O[256] = (uint16_t)M;
            for (uint32_t d = 257; d < 260; d++) X.nrm.O[d] = 0;
        }
    }
    for (uint32_t d = tid; d < 256; d += blockDim.x) {
        const uint64_t g0 = X.nrm.gmin[d], g1 = X.gmax[d];
        X.nrm.gscale[d] = (X.cnt[d] && g1 > g0) ? 1.0f / __ull2float_rn(g1 - g0) : 0.0f;
        if (!X.cnt[d]) X.nrm.gmin[d] = 0ull;
    }
    __syncthreads();
    // 3. piece statistics: each sample key's piece, fraction and target
    for (uint32_t s0 = tid & ~31u; s0 < S; s0 += blockDim.x) {  // whole warps
        const uint32_t s = s0 + lane;
        int m = -1;
        float f = 0.0f, y = 0.0f;
        if (s < S) {
            const uint64_t key = recs[P.begin + fit_pos(sseed, P.begin, P.size, s)].key;
            cdf_place(cdf_coord(key, X.nrm, M), M, m, f);
            uint32_t a = 0, b = v;  // splitters below the key
            while (a < b) {
                const uint32_t mid = (a + b) >> 1;
                if (X.ino[mid] < key) a = mid + 1; else b = mid;
            }
            y = ((float)a + 0.5f) / (float)(v + 1u);
        }
        add_stats_warp(c, m, f, y);
    }
    for (uint32_t j = tid; j < M; j += blockDim.x) {
        c.theta[j] = 0.0f;  // uniform: F(t) = t / M
        c.m1[j] = 0.0f;
        c.m2[j] = 0.0f;
    }
    __syncthreads();
    if (p.cdf_steps > 0) cdf_start_from_points(c, M);
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (uint32_t step = 0; step < p.cdf_steps; step++) {
        cdf_grad_stats(c, M, (float)S);
        const float c1 = 1.0f - powf(b1, (float)(step + 1)), c2 = 1.0f - powf(b2, (float)(step + 1));
        for (uint32_t j = tid; j < M; j += blockDim.x) {
            const float g = c.grad[j];
            const float a = b1 * c.m1[j] + (1.0f - b1) * g;
            const float b = b2 * c.m2[j] + (1.0f - b2) * g * g;
            c.m1[j] = a;
            c.m2[j] = b;
            c.theta[j] -= p.cdf_lr * (a / c1) / (sqrtf(b / c2) + eps);
        }
        __syncthreads();
    }
    // knots of the fitted model and its input coordinate
    const float T = cdf_knots(c, M);
    float* tab = w.cdf_tab + (size_t)seg * (M + 1);
    for (uint32_t j = tid; j < M; j += blockDim.x) tab[j] = c.P[j] / T;
    {
        const uint32_t* src = reinterpret_cast<const uint32_t*>(&X.nrm);
        uint32_t* dst = reinterpret_cast<uint32_t*>(w.cdf_norm + seg);
        for (uint32_t j = tid; j < sizeof(CdfNorm) / 4; j += blockDim.x) dst[j] = src[j];
    }
    if (tid == 0) {
        tab[M] = 1.0f;
        atomicAdd(&w.hdr->learned_models, 1u);
    }
    __syncthreads();  // shared arrays are rewritten by the next segment
    }
}

cudaError_t prepare_cdf_kernels(uint32_t M) {
    const size_t smem = cdf_fit_smem(M);
    cudaError_t e = cudaFuncSetAttribute(k_cdf_fit, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return e;
}

cudaError_t launch_cdf_fit(const Work& w, const Params& p, uint32_t grid, Prof* pf, cudaStream_t st) {
    const size_t smem = cdf_fit_smem(p.cdf_M);
    ProfScope ps(pf, kLearned, st);
    k_cdf_fit<<<grid, kFitThreads, smem, st>>>(w, p);
    return cudaGetLastError();
}

// Loss and gradient for given parameters and samples (sss_cdf_loss_grad):
// samples at u in [0, 1] (t = u M), the same gradient code as the fit; the
// loss is summed sample by sample.
__global__ void __launch_bounds__(kFitThreads) k_cdf_loss_grad(const float* theta, uint32_t M, const float* u,
                                                               const float* y, uint32_t S, float* loss,
                                                               float* grad) {
    extern __shared__ __align__(16) float fit_smem[];
    const CdfShared c = carve(fit_smem, M);
    const uint32_t lane = threadIdx.x & 31u;
    for (uint32_t j = threadIdx.x; j < M; j += blockDim.x) c.theta[j] = theta[j];
    zero_stats(c, M);
    __syncthreads();
    for (uint32_t s0 = threadIdx.x & ~31u; s0 < S; s0 += blockDim.x) {  // whole warps
        const uint32_t s = s0 + lane;
        int m = -1;
        float f = 0.0f, ys = 0.0f;
        if (s < S) {
            cdf_place(fminf(1.0f, fmaxf(0.0f, u[s])) * (float)M, M, m, f);
            ys = y[s];
        }
        add_stats_warp(c, m, f, ys);
    }
    __syncthreads();
    const float T = cdf_grad_stats(c, M, (float)S);
    for (uint32_t j = threadIdx.x; j < M; j += blockDim.x) grad[j] = c.grad[j];
    if (threadIdx.x == 0) c.red[1] = 0.0f;
    __syncthreads();
    float sq = 0.0f;
    for (uint32_t s = threadIdx.x; s < S; s += blockDim.x) {
        int m;
        float f;
        cdf_place(fminf(1.0f, fmaxf(0.0f, u[s])) * (float)M, M, m, f);
        const float F = (c.P[m] + f * c.D[m]) / T;
        const float e = F - y[s];
        sq += e * e;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xFFFFFFFFu, sq, o);
    if (lane == 0) atomicAdd(&c.red[1], sq);
    __syncthreads();
    if (threadIdx.x == 0) *loss = c.red[1] / (float)S;
}

cudaError_t launch_cdf_loss_grad(const float* theta, uint32_t M, const float* u, const float* y, uint32_t S,
                                 float* loss, float* grad, cudaStream_t st) {
    const size_t smem = sizeof(float) * cdf_floats(M);
    cudaError_t e = cudaFuncSetAttribute(k_cdf_loss_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_cdf_loss_grad<<<1, kFitThreads, smem, st>>>(theta, M, u, y, S, loss, grad);
    return cudaGetLastError();
}

}  // namespace sss
