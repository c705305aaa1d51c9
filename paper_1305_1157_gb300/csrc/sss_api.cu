// Host driver and C ABI of the GB300 S^5 library (declared in include/sss.h).
//
// The round loop: every distribution round runs over all large segments at
// once (k_sample, k_classify, scan, k_scatter), beside the per-CTA rounds of
// the medium segments and the base case of the buckets that became small in
// the previous round; then k_plan lays out the next round and the host reads
// back the header holding its sizes.  The loop ends when no large or medium
// segment is left; the base case of the last round's small buckets and a
// pass that resolves the LCP entries at bucket boundaries finish the sort.
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/sss.h"
#include "sss_internal.cuh"
#include "sss_alphabet.cuh"

using namespace sss;

namespace {

std::mutex g_mu;
sss_options g_opt = {10, 128u, 8192u, 32768u, 0x5eedull, 4096u, 4u, 0.005f, 0u, 0u, 16u, 0u, 0u, 0u};
sss_stats g_stats;
Prof g_prof;
std::vector<int> g_tl_cls;       // timeline of the last profiled host-driven call
std::vector<double> g_tl_start, g_tl_end;
char g_err[512] = "no error";

constexpr int kMaxDevices = 64;

struct DevPool {
    void* ws = nullptr;
    size_t ws_bytes = 0;
    Hdr* hh = nullptr;  // pinned host copy of the device header
    void* io = nullptr; // device buffers of sss_sort_host
    size_t io_bytes = 0;
    void* alpha_scan = nullptr;  // alphabet compression: header + string lengths
    size_t alpha_scan_bytes = 0;
    void* alpha_pack = nullptr;  // alphabet compression: packed offsets + packed strings
    size_t alpha_pack_bytes = 0;
    AlphaHdr* ah_host = nullptr; // pinned host copy of the alphabet header
    cudaStream_t io_stream = nullptr;  // sss_sort_host's copies and sort (non-blocking, library-owned)
};
DevPool g_pool[kMaxDevices];
Branches g_branches[kMaxDevices];  // concurrent round-body branches, created on first use


int fail(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

int cuda_fail(cudaError_t e, const char* where) {
    return fail(SSS_ERR_CUDA, "%s: %s (%s)", where, cudaGetErrorString(e), cudaGetErrorName(e));
}

#define CK(call, where)                                  \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(e_, where); \
    } while (0)

// The branch streams and events of the current device (created once).
int get_branches(const Branches** out) {
    int dev = 0;
    CK(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(SSS_ERR_INVALID, "device %d out of range", dev);
    Branches& b = g_branches[dev];
    if (!b.base) CK(branches_create(b), "branch streams");
    *out = &b;
    return SSS_OK;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct Layout {
    size_t total = 0;
    size_t o_rec0, o_rec1, o_counts, o_counts_scan, o_tlvl, o_tino, o_plans, o_chunk_seg,
        o_large, o_med0, o_med1, o_medw0, o_medw1, o_small0, o_small1, o_tiny0, o_tiny1,
        o_bigrun0, o_bigrun1, o_bids, o_scan_tmp, o_hdr, o_roots,
        o_cdf_tab, o_cdf_norm;
    uint32_t cmax, tmax, lmax, chmax, smax, ymax, bmax, scan_tmp_max, mmax;
};

uint32_t g_sms = 0;  // SM count of the first device used (sizes the count matrix)

uint32_t sms_for_layout() {
    if (!g_sms) {
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0)
            g_sms = (uint32_t)sms;
        else
            g_sms = 160;  // no device (host-only size query): a bound above GB300's 152
        cudaGetLastError();
    }
    return g_sms;
}

Layout layout_for(uint32_t n, const sss_options& o, uint32_t num_roots, bool learned = false) {
    Layout L;
    const uint64_t nn = n ? n : 1;
    const uint64_t T = o.base_threshold;
    const uint64_t M = o.medium_threshold;
    const uint64_t sms = sms_for_layout();
    // large segments exceed M strings; device-wide rounds use at least
    // ceil(total / (sms * kChunksPerSM)) strings per chunk, so their chunks
    // number at most sms * kChunksPerSM + (one partial chunk per segment)
    const uint64_t lmax = nn / (M + 1) + 2;
    // chunks are >= max(ceil(total / (sms * kChunksPerSM)), kSubTile) strings
    // unless capped by the chunk option
    uint64_t full_chunks = sms * kChunksPerSM;
    if (full_chunks < nn / o.chunk + 1) full_chunks = nn / o.chunk + 1;
    if (full_chunks > nn / kSubTile + 1) full_chunks = nn / kSubTile + 1;
    const uint64_t chmax = full_chunks + lmax + 1;
    const uint64_t cmax = (uint64_t)kNBMax * chmax + 64;
    const uint64_t tmax = nn / 16 + 2 * lmax + 64;  // 2^k <= size / 16 per segment
    const uint64_t mmax = nn / (T + 1) + 2;
    // tile-form small buckets hold more than kTinyMax strings (when the
    // threshold allows any), warp-form ones at least 2
    const uint64_t smax = (T > kTinyMax ? nn / (kTinyMax + 1) : 0) + num_roots + 2;
    const uint64_t ymax = nn / 2 + num_roots + 2;
    const uint64_t bmax = nn / (T + 1) + nn / kRunPiece + 2;  // runs > T strings, in pieces
    const uint64_t scan_tmp = scan_tmp_elems((uint32_t)cmax) + 1;
    L.cmax = (uint32_t)cmax; L.tmax = (uint32_t)tmax; L.lmax = (uint32_t)lmax; L.chmax = (uint32_t)chmax;
    L.smax = (uint32_t)smax; L.ymax = (uint32_t)ymax; L.bmax = (uint32_t)bmax; L.scan_tmp_max = (uint32_t)scan_tmp;
    L.mmax = (uint32_t)mmax;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t r = off; off = align_up(off + bytes, 256); return r; };
    L.o_rec0 = take(sizeof(Rec) * nn);
    L.o_rec1 = take(sizeof(Rec) * nn);
    L.o_counts = take(4 * (cmax + 1));
    L.o_counts_scan = take(4 * (cmax + 1));
    L.o_tlvl = take(16 * tmax);  // 16 bytes a node: room for wide keys
    L.o_tino = take(16 * tmax);
    L.o_plans = take(sizeof(SegPlan) * lmax);
    L.o_chunk_seg = take(4 * chmax);
    L.o_large = take(sizeof(Seg) * lmax);
    L.o_med0 = take(sizeof(Seg) * mmax);
    L.o_med1 = take(sizeof(Seg) * mmax);
    L.o_medw0 = take(sizeof(Seg) * mmax);
    L.o_medw1 = take(sizeof(Seg) * mmax);
    L.o_small0 = take(sizeof(Seg) * smax);
    L.o_small1 = take(sizeof(Seg) * smax);
    L.o_tiny0 = take(sizeof(Seg) * ymax);
    L.o_tiny1 = take(sizeof(Seg) * ymax);
    L.o_bigrun0 = take(sizeof(Seg) * bmax);
    L.o_bigrun1 = take(sizeof(Seg) * bmax);
    L.o_bids = take(sizeof(uint16_t) * nn);
    L.o_scan_tmp = take(4 * scan_tmp);
    L.o_hdr = take(sizeof(Hdr));
    L.o_roots = take(sizeof(Seg) * (num_roots ? num_roots : 1));
    L.o_cdf_tab = L.o_cdf_norm = 0;
    if (learned) {
        L.o_cdf_tab = take(sizeof(float) * ((size_t)o.cdf_segments + 1) * lmax);
        L.o_cdf_norm = take(sizeof(CdfNorm) * lmax);
    }
    L.total = off;
    return L;
}

Work make_work(const Layout& L, char* ws, const uint8_t* chars, const uint64_t* offsets, uint32_t n,
               uint32_t* perm, uint32_t* lcp) {
    Work w;
    memset(&w, 0, sizeof(w));
    w.chars = chars; w.offsets = offsets; w.n = n; w.out_perm = perm; w.out_lcp = lcp;
    w.rec[0] = (Rec*)(ws + L.o_rec0);
    w.rec[1] = (Rec*)(ws + L.o_rec1);
    w.counts = (uint32_t*)(ws + L.o_counts);
    w.counts_scan = (uint32_t*)(ws + L.o_counts_scan);
    w.tree_lvl = (uint64_t*)(ws + L.o_tlvl);
    w.tree_ino = (uint64_t*)(ws + L.o_tino);
    w.plans = (SegPlan*)(ws + L.o_plans);
    w.chunk_seg = (uint32_t*)(ws + L.o_chunk_seg);
    w.large = (Seg*)(ws + L.o_large);
    w.med[0] = (Seg*)(ws + L.o_med0);
    w.med[1] = (Seg*)(ws + L.o_med1);
    w.medw[0] = (Seg*)(ws + L.o_medw0);
    w.medw[1] = (Seg*)(ws + L.o_medw1);
    w.small[0] = (Seg*)(ws + L.o_small0);
    w.small[1] = (Seg*)(ws + L.o_small1);
    w.tiny[0] = (Seg*)(ws + L.o_tiny0);
    w.tiny[1] = (Seg*)(ws + L.o_tiny1);
    w.bigrun[0] = (Seg*)(ws + L.o_bigrun0);
    w.bigrun[1] = (Seg*)(ws + L.o_bigrun1);
    w.bids = (uint16_t*)(ws + L.o_bids);
    w.scan_tmp = (uint32_t*)(ws + L.o_scan_tmp);
    w.hdr = (Hdr*)(ws + L.o_hdr);
    if (L.o_cdf_tab) {
        w.cdf_tab = (float*)(ws + L.o_cdf_tab);
        w.cdf_norm = (CdfNorm*)(ws + L.o_cdf_norm);
    }
    w.cmax = L.cmax; w.tmax = L.tmax; w.lmax = L.lmax; w.chmax = L.chmax;
    w.smax = L.smax; w.ymax = L.ymax; w.bmax = L.bmax; w.scan_tmp_max = L.scan_tmp_max; w.mmax = L.mmax;
    return w;
}

int check_options(const sss_options& o) {
    if (o.k_max < 1 || o.k_max > kKMax) return fail(SSS_ERR_INVALID, "k_max must be in 1..%d", kKMax);
    if (o.base_threshold < 16 || o.base_threshold > kBaseMax)
        return fail(SSS_ERR_INVALID, "base_threshold must be in 16..%u", kBaseMax);
    if (o.medium_threshold < o.base_threshold || o.medium_threshold > kMedMax)
        return fail(SSS_ERR_INVALID, "medium_threshold must be in base_threshold..%u", kMedMax);
    if (o.chunk < kSubTile || o.chunk % kSubTile) return fail(SSS_ERR_INVALID, "chunk must be a positive multiple of %u", kSubTile);
    if (o.cdf_segments < 16 || o.cdf_segments > 4096 || (o.cdf_segments & (o.cdf_segments - 1)))
        return fail(SSS_ERR_INVALID, "cdf_segments must be a power of two in 16..4096");
    if (o.key_bytes != 8 && o.key_bytes != 16) return fail(SSS_ERR_INVALID, "key_bytes must be 8 or 16");
    if (o.classifier > 1) return fail(SSS_ERR_INVALID, "classifier must be 0 (unroll) or 1 (equal)");
    if (o.alphabet > 1) return fail(SSS_ERR_INVALID, "alphabet must be 0 (off) or 1 (compress small alphabets)");
    if (o.radix > 2) return fail(SSS_ERR_INVALID, "radix must be 0 (trees), 1 (by sample entropy) or 2 (always)");
    return SSS_OK;
}

int get_pool(DevPool** out) {
    int dev = 0;
    CK(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(SSS_ERR_INVALID, "device %d out of range", dev);
    DevPool& P = g_pool[dev];
    if (!P.hh) CK(cudaMallocHost((void**)&P.hh, sizeof(Hdr)), "cudaMallocHost(header)");
    *out = &P;
    return SSS_OK;
}

int pool_reserve(DevPool& P, size_t bytes) {
    if (P.ws_bytes >= bytes) return SSS_OK;
    if (P.ws) { cudaFree(P.ws); P.ws = nullptr; P.ws_bytes = 0; }
    cudaError_t e = cudaMalloc(&P.ws, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(SSS_ERR_NOMEM, "cudaMalloc of %zu workspace bytes failed: %s", bytes, cudaGetErrorString(e));
    }
    P.ws_bytes = bytes;
    return SSS_OK;
}

// Grow-only device buffer.
int grow_buffer(void** buf, size_t* have, size_t need, const char* what) {
    if (*have >= need) return SSS_OK;
    if (*buf) { cudaFree(*buf); *buf = nullptr; *have = 0; }
    cudaError_t e = cudaMalloc(buf, need);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(SSS_ERR_NOMEM, "cudaMalloc of %zu %s bytes failed: %s", need, what, cudaGetErrorString(e));
    }
    *have = need;
    return SSS_OK;
}

// Alphabet compression of one call (App. A.2): the alphabet from a sample
// of the strings, the packed copy the sort then runs on (when g >= 2), and
// the exact scan over all strings only when the packing pass finds a
// character the sample missed or outgrows the estimated buffer.
struct AlphaRun {
    bool on = false;
    uint32_t sigma = 0, g = 0, launches = 0;
    const uint8_t* chars = nullptr;
    const uint64_t* off = nullptr;
    const uint32_t* len = nullptr;
    AlphaHdr* ah = nullptr;
};

constexpr uint32_t kAlphaSample = 16384;  // strings of the sampled scan

int alpha_readback(DevPool& P, AlphaHdr* ah, cudaStream_t st) {
    CK(cudaMemcpyAsync(P.ah_host, ah, sizeof(AlphaHdr), cudaMemcpyDeviceToHost, st), "alphabet readback");
    CK(cudaStreamSynchronize(st), "alphabet pass");
    return SSS_OK;
}

uint32_t alpha_sigma(const AlphaHdr& h) {
    uint32_t sigma = 0;
    for (int j = 0; j < 8; j++) sigma += (uint32_t)__builtin_popcount(h.present[j]);
    return sigma;
}

// Packs with ah->present as the alphabet into a buffer of `capacity` bytes;
// *flags: the pass's kAlphaMiss / kAlphaFull.
int alpha_pack(DevPool& P, const uint8_t* chars, const uint64_t* offsets, uint32_t n, uint32_t g, uint32_t sigma,
               uint64_t capacity, Prof* pf, cudaStream_t st, AlphaRun* ar, uint32_t* flags) {
    const size_t b_off = align_up(8ull * n, 256);
    // 64 bytes of slack after the last string for the 8-byte key-word reads
    int rc = grow_buffer(&P.alpha_pack, &P.alpha_pack_bytes, b_off + align_up(capacity + 64, 256), "alphabet pack");
    if (rc) return rc;
    uint64_t* off2 = (uint64_t*)P.alpha_pack;
    uint8_t* chars2 = (uint8_t*)P.alpha_pack + b_off;
    CK(cudaMemsetAsync(&ar->ah->flags, 0, sizeof(uint32_t), st), "alphabet flags reset");
    CK(cudaMemsetAsync(&ar->ah->cursor, 0, sizeof(unsigned long long), st), "alphabet cursor reset");
    CK(launch_alpha_pack(chars, offsets, n, g, sigma, ar->ah, chars2, capacity, off2, (uint32_t*)ar->len, pf, st),
       "alphabet pack");
    ar->launches++;
    rc = alpha_readback(P, ar->ah, st);
    if (rc) return rc;
    *flags = P.ah_host->flags;
    ar->chars = chars2;
    ar->off = off2;
    return SSS_OK;
}

int alpha_prologue(DevPool& P, const uint8_t* chars, const uint64_t* offsets, uint32_t n, Prof* pf,
                   cudaStream_t st, AlphaRun* ar) {
    ar->on = true;
    if (!P.ah_host) CK(cudaMallocHost((void**)&P.ah_host, sizeof(AlphaHdr)), "cudaMallocHost(alphabet header)");
    const size_t b_hdr = align_up(sizeof(AlphaHdr), 256), b_len = align_up(4ull * n, 256);
    int rc = grow_buffer(&P.alpha_scan, &P.alpha_scan_bytes, b_hdr + b_len, "alphabet scan");
    if (rc) return rc;
    ar->ah = (AlphaHdr*)P.alpha_scan;
    ar->len = (const uint32_t*)((char*)P.alpha_scan + b_hdr);
    // 1. the alphabet and mean length of a sample
    const uint32_t step = n > kAlphaSample ? n / kAlphaSample : 1u;
    CK(cudaMemsetAsync(ar->ah, 0, sizeof(AlphaHdr), st), "alphabet header reset");
    CK(launch_alpha_scan(chars, offsets, n, step, ar->ah, pf, st), "alphabet scan");
    ar->launches++;
    rc = alpha_readback(P, ar->ah, st);
    if (rc) return rc;
    ar->sigma = alpha_sigma(*P.ah_host);
    ar->g = alpha_group(ar->sigma);  // sigma' of the sample >= 16: so is the whole input's
    if (ar->g < 2) return SSS_OK;
    // 2. pack into a buffer sized from the sample's mean length
    const double mean = P.ah_host->strings ? (double)P.ah_host->chars / P.ah_host->strings : 0.0;
    const uint64_t per = (uint64_t)((1.25 * mean + 8.0) / ar->g) + 16u;
    uint64_t capacity = (uint64_t)n * per;
    const size_t b_off = align_up(8ull * n, 256);
    if (P.alpha_pack_bytes > b_off + 320 && P.alpha_pack_bytes - b_off - 320 > capacity)
        capacity = P.alpha_pack_bytes - b_off - 320;  // reuse a larger buffer as it is
    uint32_t flags = 0;
    rc = alpha_pack(P, chars, offsets, n, ar->g, ar->sigma, capacity, pf, st, ar, &flags);
    if (rc || !flags) return rc;
    // 3. the sample missed a character or the estimate was short: the exact
    // alphabet and sizes of all strings, then pack again
    CK(cudaMemsetAsync(ar->ah, 0, sizeof(AlphaHdr), st), "alphabet header reset");
    CK(launch_alpha_scan(chars, offsets, n, 1u, ar->ah, pf, st), "alphabet scan");
    ar->launches++;
    rc = alpha_readback(P, ar->ah, st);
    if (rc) return rc;
    ar->sigma = alpha_sigma(*P.ah_host);
    ar->g = alpha_group(ar->sigma);
    ar->chars = nullptr;
    ar->off = nullptr;
    if (ar->g < 2) return SSS_OK;
    rc = alpha_pack(P, chars, offsets, n, ar->g, ar->sigma, P.ah_host->total[ar->g - 1], pf, st, ar, &flags);
    if (rc) return rc;
    if (flags) return fail(SSS_ERR_INTERNAL, "alphabet packing failed after the exact scan (flags 0x%x)", flags);
    return SSS_OK;
}

int read_hdr(Hdr* hh, const Work& w, cudaStream_t st) {
    CK(cudaMemcpyAsync(hh, w.hdr, sizeof(Hdr), cudaMemcpyDeviceToHost, st), "header readback");
    CK(cudaStreamSynchronize(st), "round");
    if (hh->err) return fail(SSS_ERR_INTERNAL, "device consistency check failed (flags 0x%x)", hh->err);
    return SSS_OK;
}

// The whole sort on an initialised Work with the host driving the rounds
// (see the file comment): one header readback per round.  Each round body
// runs the base case of the previous round's small children, the
// device-wide round and the medium rounds as concurrent branches (br), or
// one after the other on st (br null).
int run_sort(const Work& w, const sss_options& o, const Seg* roots_dev, uint32_t num_roots, Hdr* hh,
             cudaStream_t st, sss_stats* stats, bool learned = false, bool concurrent = true,
             bool reset_prof = true) {
    Params p{learned ? 1 : 0, o.cdf_segments, o.cdf_steps, o.cdf_lr, o.k_max, o.base_threshold,
             o.medium_threshold, o.chunk, o.seed, device_sms(), learned ? 8u : o.key_bytes,
             learned ? 0u : o.classifier, learned ? 0u : o.radix,
             (!roots_dev && !learned && w.n > o.medium_threshold) ? 1u : 0u};
    Prof* pf = &g_prof;
    if (reset_prof) pf->reset(o.profile != 0);
    memset(stats, 0, sizeof(*stats));
    CK(prepare_kernels(o.cdf_segments), "kernel attributes");
    CK(launch_init(w, p, pf, st), "init");
    CK(launch_roots(w, p, roots_dev, num_roots, pf, st), "roots");
    CK(launch_plan(w, p, pf, st), "plan");
    const Branches* br = nullptr;
    int rc = concurrent ? get_branches(&br) : SSS_OK;
    if (rc) return rc;
    rc = read_hdr(hh, w, st);
    if (rc) return rc;
    CK(launch_fused_root(w, p, hh, pf, st), "root round");
    for (uint32_t round = 0; hh->L > 0 || hh->n_med_snap > 0 || hh->n_medw_snap > 0; round++) {
        if (round >= 1u << 22) return fail(SSS_ERR_INTERNAL, "round limit exceeded");
        if (round < SSS_MAX_ROUNDS_LOGGED) {
            stats->round_segments[round] = hh->L + hh->n_med_snap + hh->n_medw_snap;
            stats->round_active[round] = hh->large_elems_snap + hh->med_elems_snap;
        }
        stats->rounds++;
        stats->round_strings += (uint64_t)hh->large_elems_snap + hh->med_elems_snap;
        stats->medium_strings += hh->med_elems_snap;
        stats->base_strings += (uint64_t)hh->small_elems_snap + hh->tiny_elems_snap;
        uint32_t tiles = 0;
        const unsigned long long lk0 = hh->learned_keys, lm0 = hh->learned_misses;
        CK(launch_body(w, p, hh, &tiles, pf, st, br), "round");
        stats->base_tiles += tiles;
        CK(launch_plan(w, p, pf, st, 1u), "plan");  // and hdr->round += 1 (flips the buffers and lists)
        rc = read_hdr(hh, w, st);
        if (rc) return rc;
        if (round < SSS_MAX_ROUNDS_LOGGED) {  // the learned proposals of this round
            stats->round_learned_keys[round] = hh->learned_keys - lk0;
            stats->round_learned_misses[round] = hh->learned_misses - lm0;
        }
    }
    {
        uint32_t tiles = 0;
        CK(launch_small(w, p, hh, &tiles, pf, st), "base case");
        stats->base_tiles += tiles;
        stats->base_strings += (uint64_t)hh->small_elems_snap + hh->tiny_elems_snap;
    }
    CK(launch_fixup(w, pf, st), "lcp fixup");
    if (roots_dev) CK(launch_localize(w.out_perm, roots_dev, num_roots, pf, st), "localize");
    rc = read_hdr(hh, w, st);
    if (rc) return rc;
    stats->refilled_strings = hh->refills + hh->med_refills;
    stats->medium_refilled_strings = hh->med_refills;
    stats->base_iterations = hh->base_iters;
    stats->learned_keys = hh->learned_keys;
    stats->learned_misses = hh->learned_misses;
    stats->learned_models = hh->learned_models;
    stats->radix_segments = hh->radix_segments;
    for (int i = 0; i < 8; i++) stats->base_segment_hist[i] = hh->small_hist[i];
    stats->launches = pf->launches;
    stats->profiled = pf->enabled ? 1u : 0u;
    for (int i = 0; i < kClasses; i++) stats->prof_launches[i] = pf->cls_launches[i];
    pf->collect(stats->prof_ms);
    pf->timeline(g_tl_cls, g_tl_start, g_tl_end);
    return SSS_OK;
}

// ------------------------------------------------------------ graph form
//
// The same sort as one CUDA graph: prologue (init, roots, plan), a
// conditional WHILE node whose body is one round (four concurrent branches:
// tile-form and warp-form base case of the previous round's small children,
// device-wide round, medium rounds; then plan and advance) and whose last
// kernel decides on the device whether another round is needed, then the
// epilogue (base case of the last round's children, LCP fixup, index
// rebasing).
// Kernels take their work counts from the device header, so one launch runs
// the whole sort without host round-trips.  Instantiated graphs are cached
// per device and reused while the call's buffers and options are unchanged.

struct GraphKey {
    const void *chars, *offsets, *perm, *lcp, *ws, *roots, *alpha_dig, *alpha_len;
    uint32_t n, num_roots, alpha_g;
    sss_options opt;
    int learned;
    bool operator==(const GraphKey& o) const { return memcmp(this, &o, sizeof(GraphKey)) == 0; }
};

struct GraphCache {
    bool valid = false;
    GraphKey key;
    cudaGraphExec_t exec = nullptr;
    uint32_t launches_prologue = 0, launches_body = 0, launches_epilogue = 0;
};
GraphCache g_graph[kMaxDevices];

int build_graph(const Work& w, const Params& p, const Seg* roots_dev, uint32_t num_roots, GraphCache& gc) {
    // captured on streams of our own (the caller's may be the legacy default
    // stream, which cannot be captured); the graph is launched on the caller's
    cudaStream_t st = nullptr, body_st = nullptr;
    Branches br;  // the body's concurrent branches (capture streams and fork/join events)
    CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking), "capture stream");
    cudaError_t se = cudaStreamCreateWithFlags(&body_st, cudaStreamNonBlocking);
    if (se == cudaSuccess) se = branches_create(br);
    auto free_branches = [&]() { branches_destroy(br); };
    if (se != cudaSuccess) {
        free_branches();
        if (body_st) cudaStreamDestroy(body_st);
        cudaStreamDestroy(st);
        return cuda_fail(se, "capture streams");
    }
    cudaGraph_t graph = nullptr;
    cudaError_t err = cudaSuccess;
    auto done = [&](cudaError_t e, const char* where) -> int {
        cudaStreamCaptureStatus cs;
        if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
            cudaGraph_t g2 = nullptr;
            cudaStreamEndCapture(st, &g2);
            if (g2) cudaGraphDestroy(g2);
        }
        free_branches();
        cudaStreamDestroy(body_st);
        cudaStreamDestroy(st);
        cudaGetLastError();
        return cuda_fail(e, where);
    };
    Prof counter;  // counts kernel launches per part
    counter.reset(false);
    if ((err = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
        return done(err, "begin capture");
    cudaStreamCaptureStatus cs;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    if ((err = cudaStreamGetCaptureInfo(st, &cs, nullptr, &graph, &deps, nullptr, &ndeps)) != cudaSuccess)
        return done(err, "capture info");
    cudaGraphConditionalHandle cond;
    if ((err = cudaGraphConditionalHandleCreate(&cond, graph, 0, 0)) != cudaSuccess)
        return done(err, "conditional handle");
    // prologue
    if ((err = launch_init(w, p, &counter, st)) != cudaSuccess ||
        (err = launch_roots(w, p, roots_dev, num_roots, &counter, st)) != cudaSuccess ||
        (err = launch_plan(w, p, &counter, st)) != cudaSuccess ||
        (err = launch_fused_root(w, p, nullptr, &counter, st)) != cudaSuccess ||
        (err = launch_set_cond(w, cond, st)) != cudaSuccess)
        return done(err, "graph prologue");
    gc.launches_prologue = counter.launches + 1;
    // the round loop
    if ((err = cudaStreamGetCaptureInfo(st, &cs, nullptr, &graph, &deps, nullptr, &ndeps)) != cudaSuccess)
        return done(err, "capture info");
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t loop;
    if ((err = cudaGraphAddNode(&loop, graph, deps, nullptr, ndeps, &cp)) != cudaSuccess)
        return done(err, "conditional node");
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    if ((err = cudaStreamUpdateCaptureDependencies(st, &loop, nullptr, 1, cudaStreamSetCaptureDependencies)) !=
        cudaSuccess)
        return done(err, "capture dependencies");
    if ((err = cudaStreamBeginCaptureToGraph(body_st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) !=
        cudaSuccess)
        return done(err, "begin body capture");
    counter.reset(false);
    if ((err = launch_body(w, p, nullptr, nullptr, &counter, body_st, &br)) != cudaSuccess ||
        (err = launch_plan(w, p, &counter, body_st, 2u, cond)) != cudaSuccess) {
        cudaGraph_t b2 = nullptr;
        cudaStreamEndCapture(body_st, &b2);
        return done(err, "graph body");
    }
    gc.launches_body = counter.launches;
    cudaGraph_t body_out = nullptr;
    if ((err = cudaStreamEndCapture(body_st, &body_out)) != cudaSuccess) return done(err, "end body capture");
    // epilogue
    counter.reset(false);
    if ((err = launch_small(w, p, nullptr, nullptr, &counter, st)) != cudaSuccess ||
        (err = launch_fixup(w, &counter, st)) != cudaSuccess ||
        (roots_dev && (err = launch_localize(w.out_perm, roots_dev, num_roots, &counter, st)) != cudaSuccess))
        return done(err, "graph epilogue");
    gc.launches_epilogue = counter.launches;
    cudaGraph_t full = nullptr;
    if ((err = cudaStreamEndCapture(st, &full)) != cudaSuccess) return done(err, "end capture");
    free_branches();
    cudaStreamDestroy(body_st);
    cudaStreamDestroy(st);
    cudaGraphExec_t exec = nullptr;
    // kernel nodes keep the priority of the stream they were captured on
    err = cudaGraphInstantiate(&exec, full, cudaGraphInstantiateFlagUseNodePriority);
    cudaGraphDestroy(full);
    if (err != cudaSuccess) {
        cudaGetLastError();
        return cuda_fail(err, "graph instantiate");
    }
    gc.exec = exec;
    return SSS_OK;
}

int run_sort_graph(const Work& w, const sss_options& o, const Seg* roots_dev, uint32_t num_roots, Hdr* hh,
                   cudaStream_t st, sss_stats* stats, bool learned, const GraphKey& key) {
    Params p{learned ? 1 : 0, o.cdf_segments, o.cdf_steps, o.cdf_lr, o.k_max, o.base_threshold,
             o.medium_threshold, o.chunk, o.seed, device_sms(), learned ? 8u : o.key_bytes,
             learned ? 0u : o.classifier, learned ? 0u : o.radix,
             (!roots_dev && !learned && w.n > o.medium_threshold) ? 1u : 0u};
    memset(stats, 0, sizeof(*stats));
    int dev = 0;
    CK(cudaGetDevice(&dev), "cudaGetDevice");
    GraphCache& gc = g_graph[dev];
    if (!gc.valid || !(gc.key == key)) {
        if (gc.exec) cudaGraphExecDestroy(gc.exec);
        gc = GraphCache();
        CK(prepare_kernels(o.cdf_segments), "kernel attributes");
        const int rc = build_graph(w, p, roots_dev, num_roots, gc);
        if (rc) return rc;
        gc.key = key;
        gc.valid = true;
    }
    CK(cudaGraphLaunch(gc.exec, st), "graph launch");
    const int rc = read_hdr(hh, w, st);
    if (rc) return rc;
    stats->rounds = hh->round;
    stats->refilled_strings = hh->refills + hh->med_refills;
    stats->medium_refilled_strings = hh->med_refills;
    stats->base_iterations = hh->base_iters;
    stats->learned_keys = hh->learned_keys;
    stats->learned_misses = hh->learned_misses;
    stats->learned_models = hh->learned_models;
    stats->radix_segments = hh->radix_segments;
    for (int i = 0; i < 8; i++) stats->base_segment_hist[i] = hh->small_hist[i];
    stats->launches = gc.launches_prologue + hh->round * gc.launches_body + gc.launches_epilogue;
    return SSS_OK;
}

int sort_common(const uint8_t* chars, const uint64_t* offsets, uint32_t n, uint32_t* perm, uint32_t* lcp,
                void* ws_user, size_t ws_user_bytes, const uint64_t* set_begin, uint32_t num_sets, void* stream,
                bool learned = false) {
    cudaStream_t st = (cudaStream_t)stream;
    int rc = check_options(g_opt);
    if (rc) return rc;
    if (n == 0) return SSS_OK;
    if (!chars || !offsets || !perm || !lcp) return fail(SSS_ERR_INVALID, "null pointer argument");
    if (n == 0xFFFFFFFFu) return fail(SSS_ERR_TOO_LARGE, "n must be below 2^32 - 1");
    DevPool* P = nullptr;
    rc = get_pool(&P);
    if (rc) return rc;
    g_prof.reset(g_opt.profile != 0);
    AlphaRun ar;
    if (g_opt.alphabet && !ws_user) {
        rc = alpha_prologue(*P, chars, offsets, n, &g_prof, st, &ar);
        if (rc) return rc;
        if (ar.g >= 2) {  // sort the packed copy instead
            chars = ar.chars;
            offsets = ar.off;
        }
    }
    const Layout L = layout_for(n, g_opt, num_sets, learned);
    char* ws;
    if (ws_user) {
        if (ws_user_bytes < L.total)
            return fail(SSS_ERR_NOMEM, "workspace of %zu bytes is below the %zu needed", ws_user_bytes, L.total);
        if ((uintptr_t)ws_user % 256) return fail(SSS_ERR_INVALID, "workspace must be 256-byte aligned");
        ws = (char*)ws_user;
    } else {
        rc = pool_reserve(*P, L.total);
        if (rc) return rc;
        ws = (char*)P->ws;
    }
    Work w = make_work(L, ws, chars, offsets, n, perm, lcp);
    if (ar.g >= 2) {  // LCP entries in characters of the original strings
        w.alpha_g = ar.g;
        w.alpha_dig = ar.ah->dig;
        w.alpha_len = ar.len;
    }
    Seg* roots_dev = nullptr;
    if (set_begin) {
        std::vector<Seg> roots(num_sets);
        for (uint32_t j = 0; j < num_sets; j++) {
            if (set_begin[j + 1] < set_begin[j]) return fail(SSS_ERR_INVALID, "set_begin must be non-decreasing");
            roots[j] = Seg{(uint32_t)set_begin[j], (uint32_t)(set_begin[j + 1] - set_begin[j]), 0u, 0u};
        }
        roots_dev = (Seg*)(ws + L.o_roots);
        if (num_sets) CK(cudaMemcpyAsync(roots_dev, roots.data(), sizeof(Seg) * num_sets, cudaMemcpyHostToDevice, st),
                         "roots upload");
        CK(cudaStreamSynchronize(st), "roots upload");
    }
    sss_stats stats;
    if (g_opt.graph || (set_begin && !g_opt.profile)) {
        GraphKey key;
        memset(&key, 0, sizeof(key));
        key.chars = chars; key.offsets = offsets; key.perm = perm; key.lcp = lcp; key.ws = ws;
        key.roots = roots_dev; key.n = n; key.num_roots = num_sets; key.opt = g_opt; key.learned = learned;
        key.alpha_g = w.alpha_g; key.alpha_dig = w.alpha_dig; key.alpha_len = w.alpha_len;
        key.opt.profile = 0;
        rc = run_sort_graph(w, g_opt, roots_dev, num_sets, P->hh, st, &stats, learned, key);
        stats.launches += ar.launches;
    } else {
        rc = run_sort(w, g_opt, roots_dev, num_sets, P->hh, st, &stats, learned, true, false);
    }
    if (rc) return rc;
    if (ar.on) {
        stats.alphabet_symbols = ar.sigma;
        stats.alphabet_group = ar.g >= 2 ? ar.g : 1u;
    }
    g_stats = stats;
    return SSS_OK;
}


// The set boundaries of a batched call as a host array: set_begin may point
// to host or to device memory (a device array is copied, num_sets + 1
// entries, on the caller's stream).  Checks set_begin[0] = 0,
// set_begin[num_sets] = n and that it never decreases.
int host_set_begin(const uint64_t* set_begin, uint32_t num_sets, uint32_t n, cudaStream_t st,
                   std::vector<uint64_t>& out) {
    if (!set_begin) return fail(SSS_ERR_INVALID, "null set_begin");
    if (num_sets == 0xFFFFFFFFu) return fail(SSS_ERR_TOO_LARGE, "num_sets must be below 2^32 - 1");
    out.resize((size_t)num_sets + 1);
    cudaPointerAttributes a;
    memset(&a, 0, sizeof(a));
    const bool on_device = cudaPointerGetAttributes(&a, set_begin) == cudaSuccess &&
                           (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged);
    cudaGetLastError();
    if (on_device) {
        CK(cudaMemcpyAsync(out.data(), set_begin, 8ull * out.size(), cudaMemcpyDeviceToHost, st), "set_begin readback");
        CK(cudaStreamSynchronize(st), "set_begin readback");
    } else {
        memcpy(out.data(), set_begin, 8ull * out.size());
    }
    if (out[0] != 0 || out[num_sets] != n) return fail(SSS_ERR_INVALID, "set_begin must start at 0 and end at n");
    for (uint32_t j = 0; j < num_sets; j++)
        if (out[j + 1] < out[j]) return fail(SSS_ERR_INVALID, "set_begin must be non-decreasing");
    return SSS_OK;
}

}  // namespace

extern "C" {

int sss_sort(const uint8_t* chars, const uint64_t* offsets, uint32_t n, uint32_t* out_perm, uint32_t* out_lcp,
             void* stream) {
    std::lock_guard<std::mutex> g(g_mu);
    return sort_common(chars, offsets, n, out_perm, out_lcp, nullptr, 0, nullptr, 0, stream);
}

size_t sss_workspace_size(uint32_t n) {
    std::lock_guard<std::mutex> g(g_mu);
    return layout_for(n, g_opt, 0).total;
}

int sss_sort_ws(const uint8_t* chars, const uint64_t* offsets, uint32_t n, uint32_t* out_perm, uint32_t* out_lcp,
                void* workspace, size_t workspace_bytes, void* stream) {
    std::lock_guard<std::mutex> g(g_mu);
    if (n && !workspace) return fail(SSS_ERR_INVALID, "null workspace");
    return sort_common(chars, offsets, n, out_perm, out_lcp, workspace, workspace_bytes, nullptr, 0, stream);
}

int sss_sort_batched(const uint8_t* chars, const uint64_t* offsets, uint32_t n, const uint64_t* set_begin,
                     uint32_t num_sets, uint32_t* out_perm, uint32_t* out_lcp, void* stream) {
    std::lock_guard<std::mutex> g(g_mu);
    std::vector<uint64_t> sb;
    int rc = host_set_begin(set_begin, num_sets, n, (cudaStream_t)stream, sb);
    if (rc) return rc;
    return sort_common(chars, offsets, n, out_perm, out_lcp, nullptr, 0, sb.data(), num_sets, stream);
}

int sss_sort_host(const uint8_t* chars, uint64_t chars_bytes, const uint64_t* offsets, uint32_t n,
                  uint32_t* out_perm, uint32_t* out_lcp) {
    std::lock_guard<std::mutex> g(g_mu);
    if (n == 0) return SSS_OK;
    if (!chars || !offsets || !out_perm || !out_lcp || chars_bytes == 0)
        return fail(SSS_ERR_INVALID, "null pointer or empty chars");
    DevPool* P = nullptr;
    int rc = get_pool(&P);
    if (rc) return rc;
    const size_t b_chars = align_up(chars_bytes + 16, 256), b_off = align_up(8ull * n, 256),
                 b_out = align_up(4ull * n, 256);
    const size_t need = b_chars + b_off + 2 * b_out;
    if (P->io_bytes < need) {
        if (P->io) cudaFree(P->io);
        P->io = nullptr;
        P->io_bytes = 0;
        cudaError_t e = cudaMalloc(&P->io, need);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(SSS_ERR_NOMEM, "cudaMalloc of %zu io bytes failed", need);
        }
        P->io_bytes = need;
    }
    char* base = (char*)P->io;
    uint8_t* d_chars = (uint8_t*)base;
    uint64_t* d_off = (uint64_t*)(base + b_chars);
    uint32_t* d_perm = (uint32_t*)(base + b_chars + b_off);
    uint32_t* d_lcp = (uint32_t*)(base + b_chars + b_off + b_out);
    // a stream of the library's own: the copies and the sort neither wait
    // for nor hold up work the caller has on the legacy default stream
    if (!P->io_stream) CK(cudaStreamCreateWithFlags(&P->io_stream, cudaStreamNonBlocking), "io stream");
    cudaStream_t st = P->io_stream;
    CK(cudaMemcpyAsync(d_chars, chars, chars_bytes, cudaMemcpyHostToDevice, st), "chars upload");
    CK(cudaMemcpyAsync(d_off, offsets, 8ull * n, cudaMemcpyHostToDevice, st), "offsets upload");
    // the sort between the copies runs as one graph launch (no per-round
    // host round-trip) unless the caller asked for timed host-driven rounds
    const sss_options saved = g_opt;
    if (!g_opt.profile) g_opt.graph = 1;
    rc = sort_common(d_chars, d_off, n, d_perm, d_lcp, nullptr, 0, nullptr, 0, st);
    g_opt = saved;
    if (rc) return rc;
    CK(cudaMemcpyAsync(out_perm, d_perm, 4ull * n, cudaMemcpyDeviceToHost, st), "perm download");
    CK(cudaMemcpyAsync(out_lcp, d_lcp, 4ull * n, cudaMemcpyDeviceToHost, st), "lcp download");
    CK(cudaStreamSynchronize(st), "download");
    return SSS_OK;
}

int sss_sort_learned(const uint8_t* chars, const uint64_t* offsets, uint32_t n, uint32_t* out_perm,
                     uint32_t* out_lcp, void* stream, sss_learned_stats* stats) {
    std::lock_guard<std::mutex> g(g_mu);
    const int rc = sort_common(chars, offsets, n, out_perm, out_lcp, nullptr, 0, nullptr, 0, stream, true);
    if (rc == SSS_OK && stats) {
        memset(stats, 0, sizeof(*stats));
        if (n) {
            stats->proposals = g_stats.learned_keys;
            stats->misses = g_stats.learned_misses;
            stats->models = g_stats.learned_models;
            stats->miss_rate = g_stats.learned_keys ? (double)g_stats.learned_misses / (double)g_stats.learned_keys : 0.0;
        }
    }
    return rc;
}

int sss_gather_keys(const uint8_t* chars, const uint64_t* offsets, const uint32_t* idx, const uint32_t* depth,
                    uint32_t n, uint64_t* out_keys, void* stream) {
    std::lock_guard<std::mutex> g(g_mu);
    if (n == 0) return SSS_OK;
    if (!chars || !offsets || !depth || !out_keys) return fail(SSS_ERR_INVALID, "null pointer argument");
    CK(launch_gather_keys(chars, offsets, idx, depth, n, out_keys, (cudaStream_t)stream), "gather keys");
    return SSS_OK;
}

int sss_build_splitters(const uint64_t* sample, uint32_t count, int32_t k, uint64_t* out_level, uint64_t* out_inorder,
                        void* stream) {
    std::lock_guard<std::mutex> g(g_mu);
    if (k < 1 || k > kKMax) return fail(SSS_ERR_INVALID, "k must be in 1..%d", kKMax);
    if (count < 1 || count > (2u << k) - 1u) return fail(SSS_ERR_INVALID, "count must be in 1..2^(k+1)-1");
    if (!sample || !out_level || !out_inorder) return fail(SSS_ERR_INVALID, "null pointer argument");
    CK(launch_build_splitters(sample, count, k, out_level, out_inorder, (cudaStream_t)stream), "build splitters");
    return SSS_OK;
}

int sss_classify(const uint64_t* keys, uint32_t n, const uint64_t* level, const uint64_t* inorder, int32_t k,
                 uint16_t* out_bucket, void* stream) {
    std::lock_guard<std::mutex> g(g_mu);
    if (k < 1 || k > kKMax) return fail(SSS_ERR_INVALID, "k must be in 1..%d", kKMax);
    if (n == 0) return SSS_OK;
    if (!keys || !level || !inorder || !out_bucket) return fail(SSS_ERR_INVALID, "null pointer argument");
    CK(launch_classify(keys, n, level, inorder, k, out_bucket, 0, (cudaStream_t)stream), "classify");
    return SSS_OK;
}

int sss_classify_equal(const uint64_t* keys, uint32_t n, const uint64_t* level, int32_t k, uint16_t* out_bucket,
                       void* stream) {
    std::lock_guard<std::mutex> g(g_mu);
    if (k < 1 || k > kKMax) return fail(SSS_ERR_INVALID, "k must be in 1..%d", kKMax);
    if (n == 0) return SSS_OK;
    if (!keys || !level || !out_bucket) return fail(SSS_ERR_INVALID, "null pointer argument");
    // the equality test at every node needs no in-order array
    CK(launch_classify(keys, n, level, level, k, out_bucket, 1, (cudaStream_t)stream), "classify");
    return SSS_OK;
}

int sss_cdf_loss_grad(const float* theta, uint32_t M, const float* u, const float* y, uint32_t S, float* out_loss,
                      float* out_grad, void* stream) {
    std::lock_guard<std::mutex> g(g_mu);
    if (M < 1 || M > 4096) return fail(SSS_ERR_INVALID, "M must be in 1..4096");
    if (S < 1 || S > (1u << 22)) return fail(SSS_ERR_INVALID, "S must be in 1..2^22");
    if (!theta || !u || !y || !out_loss || !out_grad) return fail(SSS_ERR_INVALID, "null pointer argument");
    CK(launch_cdf_loss_grad(theta, M, u, y, S, out_loss, out_grad, (cudaStream_t)stream), "cdf loss/grad");
    return SSS_OK;
}

int sss_set_options(const sss_options* opt) {
    std::lock_guard<std::mutex> g(g_mu);
    if (!opt) return fail(SSS_ERR_INVALID, "null options");
    int rc = check_options(*opt);
    if (rc) return rc;
    g_opt = *opt;
    return SSS_OK;
}

int sss_get_options(sss_options* opt) {
    std::lock_guard<std::mutex> g(g_mu);
    if (!opt) return fail(SSS_ERR_INVALID, "null options");
    *opt = g_opt;
    return SSS_OK;
}

int sss_get_last_stats(sss_stats* stats) {
    std::lock_guard<std::mutex> g(g_mu);
    if (!stats) return fail(SSS_ERR_INVALID, "null stats");
    *stats = g_stats;
    return SSS_OK;
}

int sss_get_last_timeline(uint32_t cap, int32_t* cls, double* start_ms, double* end_ms, uint32_t* out_count) {
    std::lock_guard<std::mutex> g(g_mu);
    if (!out_count || (cap && (!cls || !start_ms || !end_ms))) return fail(SSS_ERR_INVALID, "null pointer argument");
    const size_t n = g_tl_cls.size();
    *out_count = (uint32_t)n;
    for (size_t i = 0; i < n && i < cap; i++) {
        cls[i] = g_tl_cls[i];
        start_ms[i] = g_tl_start[i];
        end_ms[i] = g_tl_end[i];
    }
    return SSS_OK;
}

const char* sss_last_error(void) { return g_err; }

int sss_release(void) {
    std::lock_guard<std::mutex> g(g_mu);
    int cur = 0;
    cudaGetDevice(&cur);
    for (int d = 0; d < kMaxDevices; d++) {
        DevPool& P = g_pool[d];
        if (g_graph[d].exec) {
            cudaSetDevice(d);
            cudaGraphExecDestroy(g_graph[d].exec);
            g_graph[d] = GraphCache();
        }
        if (g_branches[d].base) {
            cudaSetDevice(d);
            branches_destroy(g_branches[d]);
        }
        if (!P.ws && !P.io && !P.hh && !P.alpha_scan && !P.alpha_pack && !P.ah_host && !P.io_stream) continue;
        cudaSetDevice(d);
        if (P.ws) cudaFree(P.ws);
        if (P.io) cudaFree(P.io);
        if (P.alpha_scan) cudaFree(P.alpha_scan);
        if (P.alpha_pack) cudaFree(P.alpha_pack);
        if (P.hh) cudaFreeHost(P.hh);
        if (P.ah_host) cudaFreeHost(P.ah_host);
        if (P.io_stream) cudaStreamDestroy(P.io_stream);
        P = DevPool();
    }
    cudaSetDevice(cur);
    return SSS_OK;
}

const char* sss_version(void) { return "sss-gb300 0.1"; }

}  // extern "C"

// ------------------------------------------------------------ autotuner
//
// Coordinate descent over the knobs that shape the work: tree depth (v =
// 2^k - 1 splitters, k = 5..10), base-case threshold, medium threshold, the
// device-wide work-item size, the key width (8 or 16 characters) and the
// classifier (equality test after the descent or at every node).  Each candidate is timed as the median of
// three graph-form batched sorts of the caller's tuning batch (after one
// untimed run that also builds its graph).  The winner is appended to a
// JSON-lines cache keyed by device and batch shape.

namespace {

std::string tune_key(uint32_t n, uint32_t num_sets) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp prop;
    memset(&prop, 0, sizeof(prop));
    cudaGetDeviceProperties(&prop, dev);
    // batch shape: strings and sets, each rounded to two significant digits
    auto round2 = [](uint64_t x) {
        uint64_t m = 1;
        while (x >= 100) { x /= 10; m *= 10; }
        return x * m;
    };
    char buf[256];
    snprintf(buf, sizeof(buf), "%s|sm%d|n%llu|sets%llu", prop.name, prop.multiProcessorCount,
             (unsigned long long)round2(n), (unsigned long long)round2(num_sets));
    for (char* c = buf; *c; c++)
        if (*c == '"' || *c == '\\') *c = '_';
    return std::string(buf);
}

bool cache_lookup(const char* path, const std::string& key, sss_options& o, double& ms) {
    if (!path) return false;
    FILE* f = fopen(path, "r");
    if (!f) return false;
    char line[1024];
    bool found = false;
    const std::string want = "{\"key\": \"" + key + "\",";
    while (fgets(line, sizeof(line), f)) {
        if (strncmp(line, want.c_str(), want.size()) != 0) continue;
        int k = 0;
        unsigned b = 0, m = 0, c = 0, kb = 0, cl = 0;
        double t = 0;
        if (sscanf(line + want.size(),
                   " \"k_max\": %d, \"base_threshold\": %u, \"medium_threshold\": %u, \"chunk\": %u, "
                   "\"key_bytes\": %u, \"classifier\": %u, \"ms\": %lf",
                   &k, &b, &m, &c, &kb, &cl, &t) == 7) {
            o.k_max = k; o.base_threshold = b; o.medium_threshold = m; o.chunk = c; o.key_bytes = kb;
            o.classifier = cl;
            ms = t;
            found = true;  // the last entry for a key wins
        }
    }
    fclose(f);
    return found;
}

void cache_store(const char* path, const std::string& key, const sss_options& o, double ms) {
    if (!path) return;
    FILE* f = fopen(path, "a");
    if (!f) return;
    fprintf(f,
            "{\"key\": \"%s\", \"k_max\": %d, \"base_threshold\": %u, \"medium_threshold\": %u, \"chunk\": %u, "
            "\"key_bytes\": %u, \"classifier\": %u, \"ms\": %.4f}\n",
            key.c_str(), o.k_max, o.base_threshold, o.medium_threshold, o.chunk, o.key_bytes, o.classifier, ms);
    fclose(f);
}

}  // namespace

extern "C" int sss_autotune_batched(const uint8_t* chars, const uint64_t* offsets, uint32_t n,
                                    const uint64_t* set_begin_arg, uint32_t num_sets, uint32_t* out_perm,
                                    uint32_t* out_lcp, const char* cache_path, sss_options* out_best,
                                    double* out_ms, void* stream) {
    std::lock_guard<std::mutex> g(g_mu);
    if (!out_best) return fail(SSS_ERR_INVALID, "null pointer argument");
    std::vector<uint64_t> sb;
    {
        const int rc0 = host_set_begin(set_begin_arg, num_sets, n, (cudaStream_t)stream, sb);
        if (rc0) return rc0;
    }
    const uint64_t* set_begin = sb.data();
    const std::string key = tune_key(n, num_sets);
    sss_options best = g_opt;
    double best_ms = 0.0;
    if (cache_lookup(cache_path, key, best, best_ms) && check_options(best) == SSS_OK) {
        g_opt = best;
        *out_best = best;
        if (out_ms) *out_ms = best_ms;
        return SSS_OK;
    }
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0), "event");
    CK(cudaEventCreate(&e1), "event");
    const sss_options saved = g_opt;
    auto time_opts = [&](const sss_options& o, double& ms) -> int {
        g_opt = o;
        int rc = sort_common(chars, offsets, n, out_perm, out_lcp, nullptr, 0, set_begin, num_sets, st);
        if (rc) return rc;
        double t[3];
        for (int r = 0; r < 3; r++) {
            cudaEventRecord(e0, st);
            rc = sort_common(chars, offsets, n, out_perm, out_lcp, nullptr, 0, set_begin, num_sets, st);
            if (rc) return rc;
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            float f = 0.f;
            cudaEventElapsedTime(&f, e0, e1);
            t[r] = f;
        }
        std::sort(t, t + 3);
        ms = t[1];
        return SSS_OK;
    };
    int rc = time_opts(best, best_ms);
    const int ks[] = {5, 6, 7, 8, 9, 10};
    const uint32_t bases[] = {32, 64, 96, 128};
    const uint32_t meds[] = {512, 1024, 2048, 4096, 8192};
    const uint32_t chunks[] = {8192, 16384, 32768, 65536};
    const uint32_t widths[] = {8, 16};
    for (int pass = 0; pass < 2 && rc == SSS_OK; pass++) {
        for (int knob = 0; knob < 6 && rc == SSS_OK; knob++) {
            const int count = knob == 0 ? 6 : knob == 1 ? 4 : knob == 2 ? 5 : knob == 3 ? 4 : 2;
            for (int c = 0; c < count && rc == SSS_OK; c++) {
                sss_options o = best;
                if (knob == 0) o.k_max = ks[c];
                else if (knob == 1) o.base_threshold = bases[c];
                else if (knob == 2) o.medium_threshold = meds[c];
                else if (knob == 3) o.chunk = chunks[c];
                else if (knob == 4) o.key_bytes = widths[c];
                else o.classifier = (uint32_t)c;
                if (o.medium_threshold < o.base_threshold) continue;
                if (memcmp(&o, &best, sizeof(o)) == 0 || check_options(o) != SSS_OK) continue;
                double ms = 0.0;
                rc = time_opts(o, ms);
                if (rc == SSS_OK && ms < best_ms) {
                    best = o;
                    best_ms = ms;
                }
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) {
        g_opt = saved;
        return rc;
    }
    g_opt = best;
    cache_store(cache_path, key, best, best_ms);
    *out_best = best;
    if (out_ms) *out_ms = best_ms;
    return SSS_OK;
}

// ------------------------------------------------------------ allocation-free sort
//
// sss_sort_noalloc serves callers that must not allocate device memory: its
// scratch is one static device array of kNoAllocScratchBytes, which every GPU
// that loads this library holds until the process exits.

namespace {

constexpr uint32_t kNoAllocMaxStrings = 1u << 16;
constexpr size_t kNoAllocScratchBytes = (size_t)8 << 20;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

void* g_noalloc_ptr[kMaxDevices];  // device address of g_noalloc_scratch, per device
Hdr g_noalloc_hdr[kMaxDevices];    // pageable host copy of the round header, per device

}  // namespace

extern "C" int sss_sort_noalloc(const uint8_t* chars, const uint64_t* offsets, uint32_t n, uint32_t* out_perm,
                                uint32_t* out_lcp, void* stream) {
    std::lock_guard<std::mutex> g(g_mu);
    int rc = check_options(g_opt);
    if (rc) return rc;
    if (n == 0) return SSS_OK;
    if (!chars || !offsets || !out_perm || !out_lcp) return fail(SSS_ERR_INVALID, "null pointer argument");
    if (n > kNoAllocMaxStrings)
        return fail(SSS_ERR_TOO_LARGE, "sss_sort_noalloc sorts at most %u strings, got %u", kNoAllocMaxStrings, n);
    const Layout L = layout_for(n, g_opt, 0);
    if (L.total > kNoAllocScratchBytes)
        return fail(SSS_ERR_TOO_LARGE, "%zu scratch bytes needed under the current options, %zu available",
                    L.total, kNoAllocScratchBytes);
    int dev = 0;
    CK(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(SSS_ERR_INVALID, "device %d out of range", dev);
    if (!g_noalloc_ptr[dev]) {
        // first call on this device: host code needs the array's device address
        void* p = nullptr;
        CK(cudaGetSymbolAddress(&p, g_noalloc_scratch), "cudaGetSymbolAddress(noalloc scratch)");
        g_noalloc_ptr[dev] = p;
    }
    Work w = make_work(L, (char*)g_noalloc_ptr[dev], chars, offsets, n, out_perm, out_lcp);
    sss_options o = g_opt;
    o.profile = 0;  // no timing events
    sss_stats stats;
    // serial round bodies: no library streams or events are created for it
    rc = run_sort(w, o, nullptr, 0, &g_noalloc_hdr[dev], (cudaStream_t)stream, &stats, false, false);
    if (rc) {
        // kernels of this call may still be queued: let them finish before
        // the shared array can be handed to the next call (the status was
        // already recorded)
        cudaStreamSynchronize((cudaStream_t)stream);
        cudaGetLastError();
        return rc;
    }
    g_stats = stats;
    return SSS_OK;
}
