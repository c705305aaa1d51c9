// Alphabet compression (App. A.2, "Practical Refinements"): when only
// sigma' distinct non-terminator characters occur, several characters fit
// one byte, so one key word covers more of each string and the rounds step
// deeper per key.
//
// GB300 form: instead of translating characters at every key load, the
// strings are rewritten once, at HBM speed, into a packed copy in which
// byte k of string s holds the g characters s[kg .. kg+g-1] as the digits
// of a base-(sigma'+1) number, most significant first.  A character's digit
// is its rank among the characters that occur (1..sigma'); the terminator
// and every position after it are digit 0.  g is the largest count with
// (sigma'+1)^g <= 256 (DNA, sigma' = 4: g = 3, so a 16-byte key covers 48
// characters).  The rewrite preserves the order (first differing character
// -> first differing digit of the same byte -> first differing byte, and a
// string that ends first gets digit 0 there, below every character) and
// equality, so the unchanged sort of the packed strings yields the same
// permutation.  Its LCP entries come out in characters: the kernels that
// write them (base case, large runs, boundary fixup) take the first
// differing byte's digits from a table (lcp_of_keys) and equal strings'
// lengths from the packing pass (lcp_of_equal).  A packed string is
// ceil(len/g) digit bytes (each at least sigma'+1 >= 2 to the power g-1, so
// never 0), a zero terminator byte and zero padding to a multiple of 8 bytes.
//
// Passes: k_alpha_scan on a sample of the strings gives the alphabet and
// the mean length; k_alpha_pack then finds each string's length, allocates,
// packs and checks every character against the sampled alphabet.  Only if a
// character was missing from the sample (or the estimated buffer was too
// small) does the host run the exact scan over all strings and pack again.
#include "sss_alphabet.cuh"

namespace sss {

#define FULL_MASK 0xFFFFFFFFu

namespace {

constexpr int kAlphaThreads = 256;
constexpr uint32_t kAlphaWarps = kAlphaThreads / 32;

// One wave of resident CTAs for a grid-stride loop over `items`.
template <class K>
uint32_t alpha_grid(K kernel, uint64_t items) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kAlphaThreads, 0) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    const uint64_t want = (items + kAlphaThreads - 1) / kAlphaThreads;
    const uint64_t cap = (uint64_t)device_sms() * (uint64_t)per_sm;
    return (uint32_t)std::max<uint64_t>(1, std::min(want, cap));
}

// ---- warp staging: the 32 strings of a warp are usually stored back to
// back; one coalesced copy of their bytes into shared memory replaces 32
// scattered walks through global memory.
constexpr uint32_t kStage = 4096;     // staged bytes per warp
constexpr uint32_t kStageTail = 128;  // bytes staged past the last string's start

// The staged global range [lo, hi) of a warp (lo == hi: nothing staged).
struct Stage {
    uint64_t lo, hi;
};

// Stages the bytes from the first lane's string start to kStageTail bytes
// past the last active lane's (cut at the end of that string's 4 KiB page)
// when the active lanes' string starts increase and the range fits; every
// staged byte lies between two string starts of the same array or in a page
// holding a string byte.  All lanes of the warp call it.
__device__ Stage stage_warp(uint64_t addr, bool act, uint8_t* buf) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t live = __ballot_sync(FULL_MASK, act);
    const uint64_t prev = __shfl_up_sync(FULL_MASK, addr, 1);
    const bool inc = !act || lane == 0u || prev < addr;
    Stage sg{0ull, 0ull};
    if (!__all_sync(FULL_MASK, inc) || live == 0u) return sg;
    const uint32_t last = 31u - (uint32_t)__clz((int)live);
    const uint64_t first_a = __shfl_sync(FULL_MASK, addr, 0);
    const uint64_t last_a = __shfl_sync(FULL_MASK, addr, last);
    const uint64_t lo = first_a & ~15ull;
    const uint64_t page_end = (last_a & ~4095ull) + 4096ull;
    uint64_t hi = last_a + kStageTail < page_end ? last_a + kStageTail : page_end;
    hi = (hi + 15ull) & ~15ull;  // still within the page: page_end is a multiple of 16
    if (hi - lo > kStage) return sg;
    for (uint64_t c = lo + 16ull * lane; c < hi; c += 16ull * 32u)
        *reinterpret_cast<uint4*>(buf + (c - lo)) = __ldg(reinterpret_cast<const uint4*>(c));
    __syncwarp();
    sg.lo = lo;
    sg.hi = hi;
    return sg;
}

// The aligned 8-byte word at global address wa: from the stage when staged,
// else from global memory.
__device__ __forceinline__ uint64_t word_at(uint64_t wa, const Stage& sg, const uint8_t* buf) {
    if (wa >= sg.lo && wa + 8ull <= sg.hi) return *reinterpret_cast<const uint64_t*>(buf + (wa - sg.lo));
    return __ldg(reinterpret_cast<const uint64_t*>(wa));
}

// Length of the string at addr: its words up to the terminator (every word
// read holds a byte of the string or its terminator).
__device__ uint32_t string_length(uint64_t addr, const Stage& sg, const uint8_t* buf) {
    uint32_t from = (uint32_t)(addr & 7u);
    uint32_t len = 0;
    for (uint64_t wa = addr & ~7ull;; wa += 8ull) {
        const uint64_t zm = zero_byte_mask(word_at(wa, sg, buf)) & (~0ull << (8u * from));
        if (zm) return len + ((uint32_t)(__ffsll((long long)zm) - 1) >> 3) - from;
        len += 8u - from;
        from = 0;
    }
}

// Marks the characters of word x from byte `from` (0..7) up to its first
// zero byte in seen[], adds their count to len; true if the word holds the
// terminator.
__device__ __forceinline__ bool scan_word(uint64_t x, uint32_t from, uint8_t* seen, uint32_t& len) {
    const uint64_t zm = zero_byte_mask(x) & (~0ull << (8u * from));
    const uint32_t end = zm ? (uint32_t)(__ffsll((long long)zm) - 1) >> 3 : 8u;
#pragma unroll
    for (uint32_t b = 0; b < 8u; b++)
        if (b >= from && b < end) seen[(uint32_t)(x >> (8u * b)) & 0xFFu] = 1u;
    len += end - from;
    return zm != 0ull;
}

// Marks the characters of the string at s in seen[]; returns its length.
__device__ uint32_t scan_string(const uint8_t* s, uint8_t* seen) {
    const uint64_t addr = reinterpret_cast<uint64_t>(s);
    uint32_t from = (uint32_t)(addr & 7u);
    uint32_t len = 0;
    for (const uint64_t* w = reinterpret_cast<const uint64_t*>(addr & ~7ull);; w++) {
        if (scan_word(__ldg(w), from, seen, len)) return len;
        from = 0;
    }
}

__global__ void __launch_bounds__(kAlphaThreads) k_alpha_scan(const uint8_t* __restrict__ chars,
                                                             const uint64_t* __restrict__ offsets, uint32_t n,
                                                             uint32_t step, AlphaHdr* ah) {
    __shared__ uint8_t seen[256];
    __shared__ unsigned long long tot[kAlphaMaxGroup + 1];
    __shared__ uint32_t cnt;
    seen[threadIdx.x] = 0u;
    if (threadIdx.x <= kAlphaMaxGroup) tot[threadIdx.x] = 0ull;
    if (threadIdx.x == 0) cnt = 0u;
    __syncthreads();
    unsigned long long my[kAlphaMaxGroup + 1];  // packed bytes for g = 1..8, characters
#pragma unroll
    for (uint32_t g = 0; g <= kAlphaMaxGroup; g++) my[g] = 0ull;
    uint32_t mine = 0;
    const uint64_t m = ((uint64_t)n + step - 1u) / step;  // strings scanned
    for (uint64_t j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t L = scan_string(chars + offsets[j * step], seen);
        mine++;
#pragma unroll
        for (uint32_t g = 0; g < kAlphaMaxGroup; g++) my[g] += alpha_packed_bytes(L, g + 1u);
        my[kAlphaMaxGroup] += L;
    }
#pragma unroll
    for (uint32_t g = 0; g <= kAlphaMaxGroup; g++) {
        unsigned long long v = my[g];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL_MASK, v, o);
        if ((threadIdx.x & 31u) == 0 && v) atomicAdd(&tot[g], v);
    }
    mine = __reduce_add_sync(FULL_MASK, mine);
    if ((threadIdx.x & 31u) == 0 && mine) atomicAdd(&cnt, mine);
    __syncthreads();
    // seen[0] is never set: the scan stops at the terminator
    if (seen[threadIdx.x]) atomicOr(&ah->present[threadIdx.x >> 5], 1u << (threadIdx.x & 31u));
    if (threadIdx.x < kAlphaMaxGroup && tot[threadIdx.x]) atomicAdd(&ah->total[threadIdx.x], tot[threadIdx.x]);
    if (threadIdx.x == kAlphaMaxGroup && tot[kAlphaMaxGroup]) atomicAdd(&ah->chars, tot[kAlphaMaxGroup]);
    if (threadIdx.x == 0 && cnt) atomicAdd(&ah->strings, cnt);
}

// Digits of a packed byte v (g digits of base b <= 16), most significant
// first, one per nibble from the top of the word; the rest are zero.
__device__ __forceinline__ uint32_t nibble_digits(uint32_t v, uint32_t g, uint32_t b) {
    uint32_t r = 0;
    for (uint32_t j = 0; j < g; j++) {
        r |= (v % b) << (32u - 4u * (g - j));
        v /= b;
    }
    return r;
}

constexpr uint8_t kNoCode = 0x80;  // code of a character outside the alphabet

// Writes string s (L characters) packed G per byte to dst (8-byte aligned,
// alpha_packed_bytes(L, G) bytes); returns the OR of the character codes
// (kNoCode set: a character outside the alphabet).  Step t makes output
// word t from the characters [8Gt, 8Gt + 8G): it reads the aligned 8-byte
// words holding them (each holding at least one character), shifts them so
// that every character sits at a fixed register byte, clears the bytes past
// the end (digit 0) and combines the digits of each output byte.
template <uint32_t G>
__device__ uint32_t pack_string(uint64_t addr, uint32_t L, uint32_t base, const uint8_t* code, const Stage& sg,
                                const uint8_t* buf, uint64_t* dst) {
    constexpr uint32_t kStep = 8u * G;  // characters per output word
    const uint64_t a8 = addr & ~7ull;
    const uint32_t sh = 8u * (uint32_t)(addr & 7u);
    const uint32_t nw = ((uint32_t)(addr & 7u) + L + 7u) >> 3;  // words holding characters
    uint32_t seen = 0;
    for (uint32_t p0 = 0; p0 < L; p0 += kStep) {
        const uint32_t w0 = p0 >> 3;  // p0 is a multiple of 8
        uint64_t x[G + 1];
#pragma unroll
        for (uint32_t k = 0; k <= G; k++) x[k] = (w0 + k < nw) ? word_at(a8 + 8ull * (w0 + k), sg, buf) : 0ull;
        const uint32_t rem = L - p0;  // characters left (bytes at or past it become digit 0)
        uint64_t y[G];
#pragma unroll
        for (uint32_t k = 0; k < G; k++) {
            uint64_t v = sh ? (x[k] >> sh) | (x[k + 1] << (64u - sh)) : x[k];
            if (rem < 8u * (k + 1u)) v = rem <= 8u * k ? 0ull : v & ((1ull << (8u * (rem - 8u * k))) - 1ull);
            y[k] = v;
        }
        uint64_t out = 0ull;
#pragma unroll
        for (uint32_t o = 0; o < 8u; o++) {
            uint32_t val = 0;
#pragma unroll
            for (uint32_t j = 0; j < G; j++) {
                const uint32_t t = o * G + j;  // character of the step
                const uint32_t c = code[(uint32_t)(y[t >> 3] >> (8u * (t & 7u))) & 0xFFu];
                seen |= c;
                val = val * base + c;
            }
            out |= (uint64_t)val << (8u * o);
        }
        *dst++ = out;
    }
    // the terminator byte (and padding): a zero word unless the last word
    // already ended with digit-0 bytes
    if ((((L + G - 1u) / G) & 7u) == 0u) *dst = 0ull;
    return seen;
}

template <uint32_t G>
__global__ void __launch_bounds__(kAlphaThreads) k_alpha_pack(const uint8_t* __restrict__ chars,
                                                             const uint64_t* __restrict__ offsets, uint32_t n,
                                                             uint32_t sigma, AlphaHdr* ah, uint8_t* out,
                                                             uint64_t capacity, uint64_t* __restrict__ out_off,
                                                             uint32_t* __restrict__ len_out) {
    __shared__ uint8_t code[256];
    __shared__ __align__(16) uint8_t stage[kAlphaWarps][kStage];
    __shared__ unsigned long long wbase[kAlphaWarps + 1];
    const uint32_t base = sigma + 1u;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    {
        // rank of character c among those of the alphabet (1-based); the
        // terminator 0; kNoCode for the others
        const uint32_t c = threadIdx.x;
        uint32_t below = 0;
        for (uint32_t j = 0; j < (c >> 5); j++) below += __popc(ah->present[j]);
        const uint32_t wd = ah->present[c >> 5];
        below += __popc(wd & ((1u << (c & 31u)) - 1u));
        code[c] = c == 0u ? (uint8_t)0u : ((wd >> (c & 31u)) & 1u) ? (uint8_t)(below + 1u) : kNoCode;
        if (blockIdx.x == 0) ah->dig[c] = nibble_digits(c, G, base);
    }
    __syncthreads();
    uint8_t* buf = stage[warp];
    uint32_t flags = 0;
    const uint32_t stride = gridDim.x * blockDim.x;
    // the whole CTA takes part in each step (one allocation per step)
    for (uint32_t i0 = blockIdx.x * blockDim.x; i0 < n; i0 += stride) {
        const uint32_t i = i0 + threadIdx.x;
        const bool act = i < n;
        const uint64_t addr = reinterpret_cast<uint64_t>(chars) + (act ? offsets[i] : 0ull);
        const Stage sg = stage_warp(addr, act, buf);
        const uint32_t L = act ? string_length(addr, sg, buf) : 0u;
        const unsigned long long size = act ? alpha_packed_bytes(L, G) : 0ull;
        // this string's place: exclusive prefix over the CTA + one atomicAdd
        unsigned long long inc = size;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(FULL_MASK, inc, o);
            if (lane >= (uint32_t)o) inc += y;
        }
        if (lane == 31u) wbase[warp] = inc;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long t = 0ull;
            for (uint32_t v = 0; v < kAlphaWarps; v++) {
                const unsigned long long x = wbase[v];
                wbase[v] = t;
                t += x;
            }
            wbase[kAlphaWarps] = atomicAdd(&ah->cursor, t);
        }
        __syncthreads();
        const unsigned long long pos = wbase[kAlphaWarps] + wbase[warp] + inc - size;
        if (act) {
            len_out[i] = L;
            if (pos + size <= capacity) {
                out_off[i] = pos;
                if (pack_string<G>(addr, L, base, code, sg, buf, reinterpret_cast<uint64_t*>(out + pos)) & kNoCode)
                    flags |= kAlphaMiss;
            } else {
                flags |= kAlphaFull;
            }
        }
        __syncthreads();  // the stage and wbase are reused by the next step
    }
    flags = __reduce_or_sync(FULL_MASK, flags);
    if (lane == 0 && flags) atomicOr(&ah->flags, flags);
}

}  // namespace

cudaError_t launch_alpha_scan(const uint8_t* chars, const uint64_t* offsets, uint32_t n, uint32_t step,
                              AlphaHdr* ah, Prof* pf, cudaStream_t st) {
    ProfScope ps(pf, kAlphabet, st);
    const uint64_t m = ((uint64_t)n + step - 1u) / step;
    k_alpha_scan<<<alpha_grid(k_alpha_scan, m), kAlphaThreads, 0, st>>>(chars, offsets, n, step, ah);
    return cudaGetLastError();
}

cudaError_t launch_alpha_pack(const uint8_t* chars, const uint64_t* offsets, uint32_t n, uint32_t g,
                              uint32_t sigma, AlphaHdr* ah, uint8_t* out, uint64_t capacity, uint64_t* out_off,
                              uint32_t* len_out, Prof* pf, cudaStream_t st) {
    ProfScope ps(pf, kAlphabet, st);
    switch (g) {
#define SSS_PACK_CASE(G_)                                                                                   \
    case G_:                                                                                                \
        k_alpha_pack<G_><<<alpha_grid(k_alpha_pack<G_>, n), kAlphaThreads, 0, st>>>(                        \
            chars, offsets, n, sigma, ah, out, capacity, out_off, len_out);                                 \
        break;
        SSS_PACK_CASE(2)
        SSS_PACK_CASE(3)
        SSS_PACK_CASE(4)
        SSS_PACK_CASE(5)
        SSS_PACK_CASE(6)
        SSS_PACK_CASE(7)
        SSS_PACK_CASE(8)
#undef SSS_PACK_CASE
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace sss
