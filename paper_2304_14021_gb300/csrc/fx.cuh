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
// term's bound, finer than the rounding of the same sums in FP64.
//
// All helpers are __host__ __device__ so that their arithmetic can be checked
// on the CPU against 128-bit integer and long double references.
#pragma once

#include <stdint.h>

#if defined(__CUDACC__)
#define FX_HD __host__ __device__ __forceinline__
#else
#define FX_HD inline
#endif

namespace pint {

// |c| = m * 2^q with m = mh * 2^32 + ml in [2^52, 2^53) (c's mantissa), neg = sign; c = 0: m = 0.
struct FxCoef {
    uint32_t mh, ml;
    int q, neg;
};

FX_HD uint32_t fx_umulhi(uint32_t a, uint32_t b) {
#if defined(__CUDA_ARCH__)
    return __umulhi(a, b);
#else
    return (uint32_t)(((uint64_t)a * b) >> 32);
#endif
}

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

// trunc(|u| 2^(56-E)) with the sign of u, for a finite u with |u| < 2^E.
// The result has magnitude < 2^56.  Zeros and subnormals give 0.
FX_HD int64_t fx_from_f64(uint32_t hi, uint32_t lo, int E) {
    const int ex = fx_expfield(hi);
    const uint64_t m = ((uint64_t)((hi & 0xFFFFFu) | 0x100000u) << 32) | lo;   // 53-bit significand
    // |u| = m 2^(ex-1075), in units 2^(E-56): m 2^(ex-1019-E); ex <= E+1022, so the left shift is at most 3
    int s = 1022 + E - ex;       // right shift of m << 3
    s = s < 0 ? 0 : (s > 63 ? 63 : s);
    uint64_t v = (m << 3) >> s;
    if (ex == 0) v = 0;
    const int64_t r = (int64_t)v;
    return (hi >> 31) ? -r : r;
}

// floor(|L| m / 2^55) with the sign of L, for |L| < 2^62 and m < 2^53 (so the
// result is below 2^60 in magnitude).  Exact: |L| m = A 2^64 + (B + C) 2^32 + al ml,
// and the dropped low word of al ml cannot carry across the 2^23 boundary of
// the integer B + C + hi(al ml).
FX_HD int64_t fx_mul(int64_t L, const FxCoef& c) {
    const uint64_t a = (uint64_t)(L < 0 ? -L : L);
    const uint32_t ah = (uint32_t)(a >> 32), al = (uint32_t)a;
    const uint64_t A = (uint64_t)ah * c.mh;
    const uint64_t B = (uint64_t)ah * c.ml;
    const uint64_t C = (uint64_t)al * c.mh;
    const uint64_t mid = B + C + fx_umulhi(al, c.ml);
    const uint64_t P = (A << 9) + (mid >> 23);
    return L < 0 ? -(int64_t)P : (int64_t)P;
}

// floor(L M / 2^55) (to within one unit) for |L| < 2^62 and 0 <= M < 2^53,
// M = mh 2^31 + ml (mh < 2^22, ml < 2^31): signed 32x32 products only, so no
// absolute value or negation is needed.  L M = Lh mh 2^63 + (Lh ml 2^32 +
// Ll mh 2^31 + Ll ml) with L = Lh 2^32 + Ll (Lh signed, Ll unsigned); the low
// word of Ll ml is dropped before the final floor, which can lower the result
// by one unit.  |result| < 2^60.
FX_HD int64_t fx_mul_s(int64_t L, int32_t mh, int32_t ml) {
    const int32_t Lh = (int32_t)(L >> 32);
    const uint32_t Ll = (uint32_t)L;
    const int64_t top = (int64_t)Lh * mh;                          // < 2^52
    const int64_t W = (int64_t)Lh * ml;                            // |W| < 2^61
    const uint64_t V = (uint64_t)Ll * (uint32_t)mh;                // < 2^54
    const uint64_t Zh = fx_umulhi(Ll, (uint32_t)ml);               // floor(Ll ml / 2^32) < 2^31
    // (Lh ml 2^32 + Ll mh 2^31 + Ll ml) / 2^55 = (2W + V + Ll ml / 2^31) / 2^24
    const int64_t mid = 2 * W + (int64_t)V + (int64_t)(Zh << 1);
    return (top << 8) + (mid >> 24);
}

// Bits S .. S+63 of the exact 128-bit product L M (L signed, 0 <= M < 2^63), i.e.
// floor(L M / 2^S), for 0 <= S <= 63 when that quotient fits in 64 bits.  S is
// the same for every thread of a block (a uniform branch picks the word pair).
FX_HD int64_t fx_mul_shr(int64_t L, int64_t M, int S) {
#if defined(__CUDA_ARCH__)
    const uint64_t lo = (uint64_t)L * (uint64_t)M;
    const int64_t hi = __mul64hi(L, M);
    const uint32_t w0 = (uint32_t)lo, w1 = (uint32_t)(lo >> 32), w2 = (uint32_t)hi, w3 = (uint32_t)((uint64_t)hi >> 32);
    uint32_t rx, ry;
    if (S < 32) {
        rx = __funnelshift_r(w0, w1, S);
        ry = __funnelshift_r(w1, w2, S);
    } else {
        rx = __funnelshift_r(w1, w2, S - 32);
        ry = __funnelshift_r(w2, w3, S - 32);
    }
    return (int64_t)(((uint64_t)ry << 32) | rx);
#else
    const __int128 p = (__int128)L * (__int128)M;
    return (int64_t)(p >> S);
#endif
}

// Significant bits of |v| (0 for v = 0).
FX_HD int fx_bits(int64_t v) { return 64 - fx_clz64((uint64_t)(v < 0 ? -v : v)); }

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

// Nearest float to R 2^X g, g = (gh 2^32 + gl) 2^gq with gh >= 2^31, and
// F = 2^(96 + X + gq) given as two float factors f1 f2 (each a power of two
// in the normal range).  The top 64 bits of |R| g (normalized) are formed to
// within three units and rounded once to FP32 through a 32-bit integer with a
// sticky bit (round to odd, then to nearest), so the result is the correctly
// rounded value except within 2^-40 of a tie.
FX_HD float fx_to_f32_fast(int64_t R, uint32_t gh, uint32_t gl, float f1, float f2) {
    if (R == 0) return 0.0f;
    const uint64_t a0 = (uint64_t)(R < 0 ? -R : R);
    const int lz = fx_clz64(a0);
    const uint64_t a = a0 << lz;
    const uint32_t ah = (uint32_t)(a >> 32), al = (uint32_t)a;
    const uint64_t P = (uint64_t)ah * gh + fx_umulhi(ah, gl) + fx_umulhi(al, gh);
    const uint32_t u = (uint32_t)(P >> 32) | ((uint32_t)P != 0u ? 1u : 0u);
#if defined(__CUDA_ARCH__)
    float f = __uint2float_rn(u);
    const float p2 = __int_as_float((127 - lz) << 23);
#else
    float f = (float)u;
    const uint32_t pb = (uint32_t)(127 - lz) << 23;
    float p2;
    __builtin_memcpy(&p2, &pb, 4);
#endif
    f = f * p2 * f1 * f2;
    return R < 0 ? -f : f;
}

// Arithmetic right shift by s >= 0 (floor), saturating at 63.
FX_HD int64_t fx_shr(int64_t v, int s) { return v >> (s > 63 ? 63 : s); }

// Nearest float to R 2^X g, where g = gm 2^gq with gm in [2^63, 2^64) (g's
// mantissa left-aligned).  The product R g is formed to 2^-62 relative
// before the single rounding to FP32 (round to nearest even; overflow gives
// infinity, results below the normal range give zero).
FX_HD float fx_to_f32_scaled(int64_t R, int X, uint64_t gm, int gq) {
    if (R == 0) return 0.0f;
    const uint32_t sign = R < 0 ? 0x80000000u : 0u;
    uint64_t a = (uint64_t)(R < 0 ? -R : R);
    const int lz = fx_clz64(a);
    a <<= lz;                                           // [2^63, 2^64)
    const uint32_t ah = (uint32_t)(a >> 32), al = (uint32_t)a, gh = (uint32_t)(gm >> 32), gl = (uint32_t)gm;
    // top word of a gm (al gl and the low words of the cross products dropped: < 3 units)
    const uint64_t P = (uint64_t)ah * gh + fx_umulhi(ah, gl) + fx_umulhi(al, gh);   // [2^62, 2^64)
    const int top = (P >> 63) ? 63 : 62;
    int sh = top - 23;
    uint64_t mnt = P >> sh;                              // 24 bits
    const uint64_t rem = P & ((1ull << sh) - 1), half = 1ull << (sh - 1);
    if (rem > half || (rem == half && (mnt & 1ull))) ++mnt;
    if (mnt == (1ull << 24)) {
        mnt >>= 1;
        ++sh;
    }
    // R 2^X g = a gm 2^(X - lz + gq) ~ P 2^(64 + X - lz + gq) = mnt 2^(sh + 64 + X - lz + gq)
    const int be = sh + 64 + X - lz + gq + 23 + 127;
    uint32_t bits;
    if (be >= 255) bits = sign | 0x7F800000u;
    else if (be <= 0) bits = sign;
    else bits = sign | ((uint32_t)be << 23) | ((uint32_t)mnt & 0x7FFFFFu);
#if defined(__CUDA_ARCH__)
    return __uint_as_float(bits);
#else
    float f;
    __builtin_memcpy(&f, &bits, 4);
    return f;
#endif
}

// Left-aligned mantissa and exponent of a positive finite double g given its
// bits: g = gm 2^gq, gm in [2^63, 2^64).  (g = 0 gives gm = 0.)
FX_HD void fx_align(uint64_t gbits, uint64_t& gm, int& gq) {
    const int ex = (int)((gbits >> 52) & 0x7FF);
    if (ex == 0) {
        gm = 0;
        gq = 0;
        return;
    }
    gm = ((gbits & 0xFFFFFFFFFFFFFull) | (1ull << 52)) << 11;
    gq = ex - 1075 - 11;
}

}  // namespace pint
