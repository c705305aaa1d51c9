// Alphabet compression passes (sss_alphabet.cu): device header, sizes and
// launchers.  The sort kernels see only Work::alpha_* (sss_internal.cuh).
#pragma once

#include "sss_internal.cuh"

namespace sss {

constexpr uint32_t kAlphaMaxGroup = 8;  // characters per byte at most (sigma' = 1)

// Device header of the alphabet passes, read back by the host between them.
struct AlphaHdr {
    uint32_t present[8];                       // scan: bit c set when character c occurs (c != 0)
    unsigned long long total[kAlphaMaxGroup];  // scan: [g - 1] packed bytes of the scanned strings for g
    unsigned long long chars;                  // scan: characters of the scanned strings
    uint32_t strings;                          // scan: strings scanned
    uint32_t flags;                            // pack: kAlphaMiss | kAlphaFull
    unsigned long long cursor;                 // pack: bytes allocated
    uint32_t dig[256];                         // pack: digits of each packed byte (Work::alpha_dig)
};
constexpr uint32_t kAlphaMiss = 1u;  // a character outside the scanned alphabet
constexpr uint32_t kAlphaFull = 2u;  // the packed strings did not fit the buffer

// Packed size of a string of len characters with g characters per byte:
// ceil(len / g) digit bytes, the terminator, zero padding to 8 bytes.
__host__ __device__ __forceinline__ uint64_t alpha_packed_bytes(uint64_t len, uint32_t g) {
    return ((len + g - 1) / g + 1 + 7) & ~7ull;
}

// Largest g with (sigma + 1)^g <= 256 (at most kAlphaMaxGroup); 1 when
// sigma >= 16 or sigma == 0 (nothing to gain).
__host__ __device__ __forceinline__ uint32_t alpha_group(uint32_t sigma) {
    if (sigma == 0 || sigma >= 16) return 1u;
    uint32_t g = 0, p = 1;
    while (g < kAlphaMaxGroup && p * (sigma + 1) <= 256u) { p *= sigma + 1; g++; }
    return g;
}

// Scans the strings i = 0, step, 2*step, ... (all for step 1): their
// characters into ah->present, their number and length sums into
// ah->strings / ah->chars / ah->total.
cudaError_t launch_alpha_scan(const uint8_t* chars, const uint64_t* offsets, uint32_t n, uint32_t step,
                              AlphaHdr* ah, Prof* pf, cudaStream_t st);
// Rewrites every string with g characters per byte (digits of base
// sigma + 1, character ranks from ah->present) into out (capacity bytes;
// 8-byte aligned strings in allocation order), their starts into out_off,
// their lengths into len_out and the digit table of the packed bytes into
// ah->dig.  A character outside ah->present sets kAlphaMiss, a string that
// does not fit sets kAlphaFull (the output is then unusable).
cudaError_t launch_alpha_pack(const uint8_t* chars, const uint64_t* offsets, uint32_t n, uint32_t g,
                              uint32_t sigma, AlphaHdr* ah, uint8_t* out, uint64_t capacity, uint64_t* out_off,
                              uint32_t* len_out, Prof* pf, cudaStream_t st);

}  // namespace sss
