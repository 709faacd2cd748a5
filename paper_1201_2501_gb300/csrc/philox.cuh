// philox.cuh -- Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, "Parallel random
// numbers: as easy as 1, 2, 3", SC 2011), host and device, and the draws of the hashing parameters.
#pragma once
#include <stdint.h>

#ifdef __CUDACC__
#define SFFT_HD __host__ __device__ __forceinline__
#else
#define SFFT_HD inline
#endif

namespace sfft {

struct Words4 {
    uint32_t w[4];
};

SFFT_HD void mul_hi_lo(uint32_t a, uint32_t b, uint32_t* hi, uint32_t* lo) {
#if defined(__CUDA_ARCH__)
    *hi = __umulhi(a, b);
    *lo = a * b;
#else
    const uint64_t p = (uint64_t)a * (uint64_t)b;
    *hi = (uint32_t)(p >> 32);
    *lo = (uint32_t)p;
#endif
}

// Ten rounds of the Philox-4x32 S-box with the Weyl key schedule.
SFFT_HD Words4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#if defined(__CUDA_ARCH__)
#pragma unroll
#endif
    for (int r = 0; r < 10; ++r) {
        uint32_t hi0, lo0, hi1, lo1;
        mul_hi_lo(M0, c0, &hi0, &lo0);
        mul_hi_lo(M1, c2, &hi1, &lo1);
        const uint32_t n0 = hi1 ^ c1 ^ k0;
        const uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += W0;
        k1 += W1;
    }
    Words4 out;
    out.w[0] = c0;
    out.w[1] = c1;
    out.w[2] = c2;
    out.w[3] = c3;
    return out;
}

// Counter (round, sub-step, kind, request); key = the 64-bit seed.
enum DrawKind : uint32_t { kKindExact = 0, kKindLocate = 1, kKindInner = 2, kKindEstimate = 3 };

SFFT_HD Words4 draw(uint64_t seed, uint32_t request, uint32_t round, uint32_t sub, uint32_t kind) {
    return philox4x32_10(round, sub, kind, request, (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32));
}

// sigma uniform on the odd residues, b uniform on [0, n): Algorithm 1 "Choose sigma ... Choose b".
SFFT_HD void exact_hash(uint64_t seed, uint32_t request, uint32_t round, uint32_t nmask, uint32_t* sigma,
                        uint32_t* b) {
    const Words4 w = draw(seed, request, round, 0, kKindExact);
    *sigma = (w.w[0] & nmask) | 1u;
    *b = w.w[1] & nmask;
}

// sigma^{-1} modulo 2^32 (hence modulo every power of two n): Newton steps y <- y (2 - sigma y).
SFFT_HD uint32_t inverse_odd(uint32_t sigma) {
    uint32_t y = sigma;  // correct to 3 bits
    for (int i = 0; i < 5; ++i) y = y * (2u - sigma * y);
    return y;
}

}  // namespace sfft
