// The Gaussian test matrix Omega of Alg. 1 step 3 as device functions:
// entry (row, col) of the draw for (seed, batch) is a pure function of those
// four words, so every kernel that needs a block of Omega (the streaming
// fill, the batched one-CTA factorisation) evaluates the same values.
#pragma once

#include <cstdint>
#include <type_traits>
#include <cuda_bf16.h>

namespace eod {
namespace {

// ---------------------------------------------------------------- Omega ----
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32 -> 64-bit products, the key advanced by the golden-ratio Weyl
// constants between rounds.
__device__ __forceinline__ void philox_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        const uint32_t lo0 = 0xD2511F53u * c[0], hi0 = __umulhi(0xD2511F53u, c[0]);
        const uint32_t lo1 = 0xCD9E8D57u * c[2], hi1 = __umulhi(0xCD9E8D57u, c[2]);
        const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    }
}

// Round a double to the nearest BF16 value (8 significant bits), ties to
// even, by integer rounding at bit 45 of the binary64 encoding (the carry
// propagates into the exponent when the mantissa overflows).
__device__ __forceinline__ double round_bf16_from_f64(double g) {
    unsigned long long b = (unsigned long long)__double_as_longlong(g);
    const unsigned long long lsb = (b >> 45) & 1ull;
    b += 0x00000FFFFFFFFFFFull + lsb;
    b &= ~0x00001FFFFFFFFFFFull;
    return __longlong_as_double((long long)b);
}

// The draw in FP64 from the two Philox words (the definition of Omega).
__device__ __forceinline__ double omega_value_f64(uint32_t x0, uint32_t x1) {
    const double u1 = ((double)x0 + 0.5) * 0x1p-32;
    const double u2 = ((double)x1 + 0.5) * 0x1p-32;
    const double radius = sqrt(-2.0 * log(u1));
    const double angle = (2.0 * 3.141592653589793) * u2;
    return round_bf16_from_f64(radius * cos(angle));
}

// The same draw evaluated in FP32 when that provably gives the same BF16
// value.  u1, u2 and the transcendental functions are taken in FP32 (logf /
// log1pf / sqrtf / cospif, each within a few ulp); -2 ln u1 is formed from
// 1 - u1 through log1pf when u1 >= 1/2, so its relative error stays at a few
// 2^-24 everywhere.  Their combined error in g is below (13/|cos| + 6) float
// ulps of g; if no BF16 rounding midpoint lies within twice that distance of
// the FP32 result, both roundings agree and the FP32 value is returned,
// otherwise the FP64 formula decides.
template <typename T>
__device__ __forceinline__ T omega_value_fast(uint64_t seed, uint32_t row, uint32_t col, uint32_t batch) {
    uint32_t c[4] = {row, col, batch, 0u};
    philox_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    const uint32_t x0 = c[0], x1 = c[1];
    float L;
    if (x0 < 0x80000000u) {
        const float u1 = ((float)x0 + 0.5f) * 0x1p-32f;
        L = -2.f * logf(u1);
    } else {
        const float v = ((float)(0xFFFFFFFFu - x0) + 0.5f) * 0x1p-32f;
        L = -2.f * log1pf(-v);
    }
    const float cs = cospif(2.f * (((float)x1 + 0.5f) * 0x1p-32f));
    const float g = sqrtf(L) * cs;
    const int low = (int)(__float_as_uint(g) & 0xFFFFu);
    const float guard = 26.f / fabsf(cs) + 12.f;
    if (fabsf((float)(low - 0x8000)) > guard && isfinite(g)) {
        // the BF16 value itself, converted without an FP64 instruction
        const __nv_bfloat16 b = __float2bfloat16_rn(g);
        if constexpr (std::is_same<T, __nv_bfloat16>::value) return b;
        else return (T)__bfloat162float(b);
    }
    const double v = omega_value_f64(x0, x1);   // exactly a BF16 value
    if constexpr (std::is_same<T, __nv_bfloat16>::value) return __float2bfloat16_rn((float)v);
    else return (T)v;
}

}  // namespace
}  // namespace eod
