// Learned bucket proposal: a monotone piecewise-linear CDF of a segment's
// key words, fitted on the segment's own sorted splitter sample with
// hand-written forward and backward passes and Adam, all in FP32 on one CTA
// per segment.  (An addition to the paper; its closest idea is the jump
// tables of App. A.2 that replace part of the splitter-tree descent.)
//
// Model with M pieces on u in [0, 1]: increments d_j = softplus(theta_j),
// T = sum_j d_j, knots C_j = (d_0 + ... + d_{j-1}) / T, and for u in piece m
// with fraction f: F(u) = C_m + f d_m / T.  Loss: mean over the sample of
// (F(u_s) - y_s)^2 with y_s = (j_s + 1/2) / (v + 1), j_s the number of
// splitters below sample key s (the splitter interval the tree gives it), so
// that floor(F (v + 1)) proposes that interval.  Gradient, term by term:
//   dF_s/dd_j = ([j < m_s] + f_s [j = m_s]) / T - F_s / T
//   dL/dd_j   = (sum_{s: m_s > j} g_s + sum_{s: m_s = j} g_s f_s - sum_s g_s F_s) / T,
//               g_s = 2 (F_s - y_s) / S
//   dL/dtheta_j = dL/dd_j * sigmoid(theta_j)
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

// Shared-memory arrays of one fit.
struct CdfShared {
    float *theta, *D, *P, *A, *B, *grad, *m1, *m2;  // [M] each, P has M + 1
    int* ms;                                         // [S] piece of each sample (non-decreasing)
    float *fs, *ys;                                  // [S] fraction in the piece, target
    float *cg, *cgf;                                 // [S] prefix sums over the samples
    float* wsum;                                     // [33]
    float* red;                                      // [2]
};

__device__ __forceinline__ CdfShared carve(float* base, uint32_t M, uint32_t S) {
    CdfShared c;
    float* p = base;
    c.theta = p; p += M;
    c.D = p; p += M;
    c.P = p; p += M + 1;
    c.A = p; p += M;
    c.B = p; p += M;
    c.grad = p; p += M;
    c.m1 = p; p += M;
    c.m2 = p; p += M;
    c.ms = reinterpret_cast<int*>(p); p += S;
    c.fs = p; p += S;
    c.ys = p; p += S;
    c.cg = p; p += S;
    c.cgf = p; p += S;
    c.wsum = p; p += 33;
    c.red = p;
    return c;
}

size_t cdf_fit_smem(uint32_t M) {
    return sizeof(float) * ((size_t)8 * M + 1 + 5 * (size_t)kSampleMax + 33 + 2);
}

// Forward pass, loss and gradient (into c.grad) for the samples (ms, fs, ys;
// ms non-decreasing).  Returns the loss.  Ends synchronised.
__device__ float cdf_loss_grad_dev(const CdfShared& c, uint32_t M, uint32_t S) {
    const uint32_t lane = threadIdx.x & 31u;
    for (uint32_t j = threadIdx.x; j < M; j += blockDim.x) {
        const float d = softplus_f(c.theta[j]);
        c.D[j] = d;
        c.P[j] = d;
        c.A[j] = 0.0f;
        c.B[j] = 0.0f;
    }
    if (threadIdx.x == 0) { c.red[0] = 0.0f; c.red[1] = 0.0f; }
    __syncthreads();
    const float T = block_excl_scan_f(c.P, M, c.wsum);  // P[j] = d_0 + ... + d_{j-1}
    const float invT = 1.0f / T;
    float gF = 0.0f, sq = 0.0f;
    for (uint32_t s = threadIdx.x; s < S; s += blockDim.x) {
        const int m = c.ms[s];
        const float f = c.fs[s];
        const float F = (c.P[m] + f * c.D[m]) * invT;
        const float e = F - c.ys[s];
        const float g = 2.0f * e / (float)S;
        c.cg[s] = g;
        c.cgf[s] = g * f;
        gF += g * F;
        sq += e * e;
    }
    __syncthreads();
    // A[m] = sum of g over the samples in piece m, B[m] = sum of g f: the
    // samples are sorted, so a piece's samples are consecutive
    const float totg = block_excl_scan_f(c.cg, S, c.wsum);
    const float totgf = block_excl_scan_f(c.cgf, S, c.wsum);
    for (uint32_t s = threadIdx.x; s < S; s += blockDim.x) {
        const int m = c.ms[s];
        if (s == 0 || c.ms[s - 1] != m) {  // first sample of its piece
            atomicAdd(&c.A[m], -c.cg[s]);
            atomicAdd(&c.B[m], -c.cgf[s]);
        }
        if (s + 1 == S || c.ms[s + 1] != m) {  // last sample of its piece
            atomicAdd(&c.A[m], s + 1 == S ? totg : c.cg[s + 1]);
            atomicAdd(&c.B[m], s + 1 == S ? totgf : c.cgf[s + 1]);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        gF += __shfl_xor_sync(0xFFFFFFFFu, gF, o);
        sq += __shfl_xor_sync(0xFFFFFFFFu, sq, o);
    }
    if (lane == 0) {
        atomicAdd(&c.red[0], gF);
        atomicAdd(&c.red[1], sq);
    }
    __syncthreads();  // every sample's contribution to A, B and red is in
    for (uint32_t j = threadIdx.x; j < M; j += blockDim.x) c.grad[j] = c.A[j];
    __syncthreads();
    const float totA = block_excl_scan_f(c.grad, M, c.wsum);  // grad[j] = A_0 + ... + A_{j-1}
    const float G = c.red[0];
    for (uint32_t j = threadIdx.x; j < M; j += blockDim.x) {
        const float suffix = totA - c.grad[j] - c.A[j];  // A_{j+1} + ... + A_{M-1}
        const float dd = (suffix + c.B[j] - G) * invT;
        c.grad[j] = dd * sigmoid_f(c.theta[j]);
    }
    __syncthreads();
    return c.red[1] / (float)S;
}

// piece and fraction of each sample's u
__device__ __forceinline__ void cdf_place(float u, uint32_t M, int& m, float& f) {
    const float t = u * (float)M;
    const uint32_t mm = min((uint32_t)t, M - 1u);
    m = (int)mm;
    f = t - (float)mm;
}

// One CTA per planned segment of at least kLearnedMinSize strings: fit the
// model on the segment's sorted sample (written by k_sample) and store its
// knots, kmin and scale.
__global__ void __launch_bounds__(kFitThreads) k_cdf_fit(Work w, Params p) {
    extern __shared__ __align__(16) float fit_smem[];
    const uint32_t M = p.cdf_M;
    const uint32_t L = w.hdr->L;
    __shared__ uint32_t s_item;
    for (uint32_t seg = first_item(); seg < L; seg = next_item(&w.hdr->q_fit, &s_item)) {
    const SegPlan P = w.plans[seg];
    if (P.size < kLearnedMinSize) continue;
    const uint32_t S = (2u << P.k) - 1u;
    const CdfShared c = carve(fit_smem, M, kSampleMax);
    const uint64_t* samp = w.cdf_samp + (size_t)seg * kSampleMax;
    const uint64_t kmin = samp[0], kmax = samp[S - 1];
    const float scale = kmax > kmin ? 1.0f / __ull2float_rn(kmax - kmin) : 0.0f;
    const uint64_t* ino = w.tree_ino + P.tree_base;
    const uint32_t v = (1u << P.k) - 1u;
    for (uint32_t s = threadIdx.x; s < S; s += blockDim.x) {
        int m;
        float f;
        const uint64_t key = samp[s];
        cdf_place(cdf_u(key, kmin, scale), M, m, f);
        uint32_t a = 0, b = v;  // splitters below the key
        while (a < b) { const uint32_t mid = (a + b) >> 1; if (ino[mid] < key) a = mid + 1; else b = mid; }
        c.ms[s] = m;
        c.fs[s] = f;
        c.ys[s] = ((float)a + 0.5f) / (float)(v + 1u);
    }
    for (uint32_t j = threadIdx.x; j < M; j += blockDim.x) {
        c.theta[j] = 0.0f;  // uniform: F(u) = u
        c.m1[j] = 0.0f;
        c.m2[j] = 0.0f;
        c.A[j] = 0.0f;
    }
    __syncthreads();
    if (p.cdf_steps > 0) {
        // start from the sample's histogram over the pieces: increment of
        // piece j proportional to (samples in j + 1/16), theta = softplus^-1
        for (uint32_t s = threadIdx.x; s < S; s += blockDim.x) {
            const int m = c.ms[s];
            if (s == 0 || c.ms[s - 1] != m) atomicAdd(&c.A[m], -(float)s);
            if (s + 1 == S || c.ms[s + 1] != m) atomicAdd(&c.A[m], (float)(s + 1));
        }
        __syncthreads();
        for (uint32_t j = threadIdx.x; j < M; j += blockDim.x) {
            const float d = c.A[j] + 0.0625f;
            c.theta[j] = d > 20.0f ? d : logf(expm1f(d));
        }
        __syncthreads();
    }
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (uint32_t step = 0; step < p.cdf_steps; step++) {
        cdf_loss_grad_dev(c, M, S);
        const float c1 = 1.0f - powf(b1, (float)(step + 1)), c2 = 1.0f - powf(b2, (float)(step + 1));
        for (uint32_t j = threadIdx.x; j < M; j += blockDim.x) {
            const float g = c.grad[j];
            const float a = b1 * c.m1[j] + (1.0f - b1) * g;
            const float b = b2 * c.m2[j] + (1.0f - b2) * g * g;
            c.m1[j] = a;
            c.m2[j] = b;
            c.theta[j] -= p.cdf_lr * (a / c1) / (sqrtf(b / c2) + eps);
        }
        __syncthreads();
    }
    // knots of the fitted model
    for (uint32_t j = threadIdx.x; j < M; j += blockDim.x) c.P[j] = softplus_f(c.theta[j]);
    __syncthreads();
    const float T = block_excl_scan_f(c.P, M, c.wsum);
    float* tab = w.cdf_tab + (size_t)seg * (M + 1);
    for (uint32_t j = threadIdx.x; j < M; j += blockDim.x) tab[j] = c.P[j] / T;
    if (threadIdx.x == 0) {
        tab[M] = 1.0f;
        w.cdf_kmin[seg] = kmin;
        w.cdf_scale[seg] = scale;
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

// Loss and gradient for given parameters and samples (sss_cdf_loss_grad).
__global__ void __launch_bounds__(kFitThreads) k_cdf_loss_grad(const float* theta, uint32_t M, const float* u,
                                                               const float* y, uint32_t S, float* loss,
                                                               float* grad) {
    extern __shared__ __align__(16) float fit_smem[];
    const CdfShared c = carve(fit_smem, M, kSampleMax);
    for (uint32_t j = threadIdx.x; j < M; j += blockDim.x) c.theta[j] = theta[j];
    for (uint32_t s = threadIdx.x; s < S; s += blockDim.x) {
        int m;
        float f;
        cdf_place(fminf(1.0f, fmaxf(0.0f, u[s])), M, m, f);
        c.ms[s] = m;
        c.fs[s] = f;
        c.ys[s] = y[s];
    }
    __syncthreads();
    const float L = cdf_loss_grad_dev(c, M, S);
    for (uint32_t j = threadIdx.x; j < M; j += blockDim.x) grad[j] = c.grad[j];
    if (threadIdx.x == 0) *loss = L;
}

cudaError_t launch_cdf_loss_grad(const float* theta, uint32_t M, const float* u, const float* y, uint32_t S,
                                 float* loss, float* grad, cudaStream_t st) {
    const size_t smem = cdf_fit_smem(M);
    cudaError_t e = cudaFuncSetAttribute(k_cdf_loss_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_cdf_loss_grad<<<1, kFitThreads, smem, st>>>(theta, M, u, y, S, loss, grad);
    return cudaGetLastError();
}

}  // namespace sss
