// ff.cuh - float-float ("double-word") arithmetic on the FP32 pipes.
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2,
// about 48 significant bits.  The building blocks are the classical
// error-free transformations:
//   two_sum(a, b)       s + e == a + b exactly           (Knuth, 6 flops)
//   fast_two_sum(a, b)  same, valid when |a| >= |b|        (Dekker, 3 flops)
//   two_prod(a, b)      p + e == a * b exactly            (one FMA)
// and the double-word sum / product algorithms built from them (analysed in
// Joldes, Muller, Popescu, "Tight and rigorous error bounds for basic building
// blocks of double-word arithmetic", ACM TOMS 2017).  The sum used here is the
// accurate variant: its result is within ~2^-47 relative of the exact sum even
// under cancellation, which is what finite-difference stencils of smooth data
// need.  Expressions are written so that no multiply is contracted into a
// following add (the products that must be exact use explicit fmaf).
#pragma once

#include <cuda_runtime.h>

namespace pint {

typedef float2 ff;  // x = hi, y = lo

__device__ __forceinline__ ff ffmk(float h, float l) { return make_float2(h, l); }

__device__ __forceinline__ ff two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return ffmk(s, e);
}
__device__ __forceinline__ ff fast_two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return ffmk(s, e);
}
__device__ __forceinline__ ff two_prod(float a, float b) {
    float p = __fmul_rn(a, b);
    float e = fmaf(a, b, -p);
    return ffmk(p, e);
}
// accurate double-word + double-word
__device__ __forceinline__ ff ff_add(ff x, ff y) {
    ff s = two_sum(x.x, y.x);
    ff t = two_sum(x.y, y.y);
    float c = __fadd_rn(s.y, t.x);
    ff v = fast_two_sum(s.x, c);
    float w = __fadd_rn(t.y, v.y);
    return fast_two_sum(v.x, w);
}
__device__ __forceinline__ ff ff_neg(ff x) { return ffmk(-x.x, -x.y); }
__device__ __forceinline__ ff ff_sub(ff x, ff y) { return ff_add(x, ff_neg(y)); }
// double-word + float
__device__ __forceinline__ ff ff_add_f(ff x, float b) {
    ff s = two_sum(x.x, b);
    float v = __fadd_rn(x.y, s.y);
    return fast_two_sum(s.x, v);
}
// double-word * float
__device__ __forceinline__ ff ff_mul_f(ff x, float c) {
    ff p = two_prod(x.x, c);
    float l = fmaf(x.y, c, p.y);
    return fast_two_sum(p.x, l);
}
// double-word * double-word
__device__ __forceinline__ ff ff_mul(ff x, ff y) {
    ff p = two_prod(x.x, y.x);
    float t = __fmul_rn(x.x, y.y);
    t = fmaf(x.y, y.x, t);
    float l = __fadd_rn(p.y, t);
    return fast_two_sum(p.x, l);
}
// multiplication by a power of two (exact)
__device__ __forceinline__ ff ff_scale2(ff x, float p2) { return ffmk(x.x * p2, x.y * p2); }

// host: split a double into hi + lo floats
__host__ __device__ inline float2 ff_from_double(double d) {
    float h = (float)d;
    float l = (float)(d - (double)h);
    return make_float2(h, l);
}

}  // namespace pint
