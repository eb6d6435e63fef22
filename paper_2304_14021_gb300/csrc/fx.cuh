// fx.cuh - block fixed-point arithmetic for the FP64-accurate residual on the
// integer pipes (k_residual_fx.cu).
//
// GB300 issues FP64 arithmetic at about 1/64 of its FP32 rate, so an FP64
// stencil residual is bound by the FP64 pipe.  Here the FP64 iterate is
// converted per tile and time level to 64-bit integers in a common binary
// unit, the stencil sums (integer coefficients) are then exact integer
// additions, and the few products with the problem's coefficients are formed
// from 32x32-bit integer products with the coefficients' full 53-bit
// mantissas.  Every rounding is a truncation at 2^-57 or below of the largest
// term in the tile, as fine as the rounding of the same sums in FP64.
//
// All helpers are __host__ __device__ so that their arithmetic can be checked
// on the CPU against 128-bit integer and long double references.
#pragma once

#include <math.h>
#include <stdint.h>

#if defined(__CUDACC__)
#define FX_HD __host__ __device__ __forceinline__
#else
#define FX_HD inline
#endif

namespace pint {

FX_HD int fx_clz64(uint64_t a) {
#if defined(__CUDA_ARCH__)
    return __clzll((long long)a);
#else
    return a ? __builtin_clzll(a) : 64;
#endif
}

// Biased exponent field of a double given its upper 32 bits.
FX_HD int fx_expfield(uint32_t hi) { return (int)((hi >> 20) & 0x7FFu); }

// Unit exponent of a tile whose largest biased exponent field is f: every
// |u| < 2^E with E = f - 1022.
FX_HD int fx_tile_exp(int f) { return f - 1022; }

// The low word of (hi:lo) >> s, 0 <= s < 32.
FX_HD uint32_t fx_funnel_r(uint32_t lo, uint32_t hi, int s) {
#if defined(__CUDA_ARCH__)
    return __funnelshift_r(lo, hi, s);
#else
    return (uint32_t)((((uint64_t)hi << 32) | lo) >> s);
#endif
}

// floor(L M / 2^S) for L signed, 0 <= M < 2^63 and S >= 0, whenever the
// quotient fits in 64 bits (S >= 127: the sign word).  The exact 128-bit
// product is formed from its four 32-bit words and the window selected by S;
// S is the same for every thread of a block (uniform branches pick the words).
FX_HD int64_t fx_mul_shr(int64_t L, int64_t M, int S) {
    const uint64_t lo = (uint64_t)L * (uint64_t)M;
#if defined(__CUDA_ARCH__)
    const int64_t hi = __mul64hi(L, M);
#else
    const int64_t hi = (int64_t)(((__int128)L * (__int128)M) >> 64);
#endif
    const uint32_t w0 = (uint32_t)lo, w1 = (uint32_t)(lo >> 32), w2 = (uint32_t)hi, w3 = (uint32_t)((uint64_t)hi >> 32);
    const uint32_t ws = (uint32_t)((int32_t)w3 >> 31);
    uint32_t rx, ry;
    if (S < 32) {
        rx = fx_funnel_r(w0, w1, S);
        ry = fx_funnel_r(w1, w2, S);
    } else if (S < 64) {
        rx = fx_funnel_r(w1, w2, S - 32);
        ry = fx_funnel_r(w2, w3, S - 32);
    } else if (S < 96) {
        rx = fx_funnel_r(w2, w3, S - 64);
        ry = fx_funnel_r(w3, ws, S - 64);
    } else if (S < 128) {
        rx = fx_funnel_r(w3, ws, S - 96);
        ry = ws;
    } else {
        rx = ry = ws;
    }
    return (int64_t)(((uint64_t)ry << 32) | rx);
}

// 64-bit right shift with the PTX semantics for amounts >= 64 (the result
// is 0): unsigned; and arithmetic (sign fill).
FX_HD uint64_t fx_shr_u(uint64_t v, uint32_t s) {
#if defined(__CUDA_ARCH__)
    uint64_t r;
    asm("shr.b64 %0, %1, %2;" : "=l"(r) : "l"(v), "r"(s));
    return r;
#else
    return s >= 64 ? 0 : v >> s;
#endif
}
FX_HD int64_t fx_sar(int64_t v, uint32_t s) {
#if defined(__CUDA_ARCH__)
    int64_t r;
    asm("shr.s64 %0, %1, %2;" : "=l"(r) : "l"(v), "r"(s));
    return r;
#else
    return s >= 64 ? (v < 0 ? -1 : 0) : v >> s;
#endif
}

// trunc(|u| 2^(56-E)) with the sign of u, for a finite u with |u| < 2^E and
// E >= -958 (so that zeros and subnormals shift out to 0).
FX_HD int64_t fx_from_f64_fast(uint32_t hi, uint32_t lo, int E) {
    // significand << 3, i.e. (2^52 + frac) << 3, built from the words
    const uint32_t h3 = (((hi << 3) | (lo >> 29)) & 0x7FFFFFu) | 0x800000u;
    const uint64_t m3 = ((uint64_t)h3 << 32) | (uint64_t)(lo << 3);
    const uint64_t v = fx_shr_u(m3, (uint32_t)(1022 + E - fx_expfield(hi)));
    const int64_t sm = (int64_t)(int32_t)hi >> 31;   // 0 or -1
    return ((int64_t)v ^ sm) - sm;
}

// R (Gh + Gl) f1 f2 in FP32, for an integer R (|R| < 2^63), Gh + Gl a
// float-float factor (Gh an integer below 2^24, |Gl| <= 1, together a 53-bit
// mantissa to 2^-48) and f1, f2 powers of two in the normal range.  R is split
// exactly into hi 2^32 + lo (lo the signed low word), both halves are
// converted with one rounding each and recombined with one FMA, so
// v = R (1 + d) with |d| <= 5 2^-25 (|d| <= 2^-24 when |R| < 2^31); the
// product with Gh + Gl adds one rounding (2^-24) and the powers of two are
// exact: the result is within 7 2^-25 relative of R (Gh + Gl) f1 f2 (under 4
// ulp of FP32) while it stays in the normal range.
FX_HD float fx_to_f32_pair(int64_t R, float Gh, float Gl, float f1, float f2) {
    const int32_t lo = (int32_t)(uint32_t)(uint64_t)R;
    const int32_t hi = (int32_t)(uint32_t)((uint64_t)R >> 32) - (lo >> 31);   // R = hi 2^32 + lo
#if defined(__CUDA_ARCH__)
    const float v = __fmaf_rn(__int2float_rn(hi), 4294967296.0f, __int2float_rn(lo));
    return __fmul_rn(__fmul_rn(__fmaf_rn(v, Gh, __fmul_rn(v, Gl)), f1), f2);
#else
    const float v = fmaf((float)hi, 4294967296.0f, (float)lo);
    return fmaf(v, Gh, v * Gl) * f1 * f2;
#endif
}

// Float-float mantissa of a positive normal double g given its bits:
// g = (Gh + Gl) 2^(e - 1046), e the biased exponent field, Gh the top 24
// bits of the 53-bit significand (an integer in [2^23, 2^24)) and Gl the
// remaining 29 bits / 2^29 rounded to FP32 (|Gl| < 1, error <= 2^-25).
FX_HD void fx_split_f64(uint64_t gbits, float& Gh, float& Gl, int& e) {
    e = (int)((gbits >> 52) & 0x7FF);
    const uint64_t m = (gbits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    Gh = (float)(uint32_t)(m >> 29);
    Gl = (float)(uint32_t)(m & 0x1FFFFFFFu) * (1.0f / 536870912.0f);
}

}  // namespace pint
