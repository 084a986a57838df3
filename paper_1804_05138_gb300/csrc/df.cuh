// df.cuh -- float-pair ("double-float") arithmetic for the FP32 form: a value is h + l with |l| at
// most half an ulp of h, about 44 significant bits.  Products are exact by FMA (Dekker), sums by
// Knuth's TwoSum; reciprocal, reciprocal square root and square root take one Newton step in pairs
// from the FP32 result.  Used where one SM would otherwise issue a long chain of FP64 instructions
// (FP64 issues at a small fraction of the FP32 rate on this part).
#pragma once

namespace rq {

struct df {
    float h, l;
};
__device__ __forceinline__ df df_two_sum(float a, float b)
{
    const float s = a + b;
    const float z = s - a;
    return {s, (a - (s - z)) + (b - z)};
}
__device__ __forceinline__ df df_quick(float a, float b)  // |a| >= |b|
{
    const float s = a + b;
    return {s, b - (s - a)};
}
__device__ __forceinline__ df df_add(df a, df b)
{
    const df s = df_two_sum(a.h, b.h);
    return df_quick(s.h, s.l + a.l + b.l);
}
__device__ __forceinline__ df df_neg(df a) { return {-a.h, -a.l}; }
__device__ __forceinline__ df df_mul(df a, df b)
{
    const float p = a.h * b.h;
    const float e = fmaf(a.h, b.h, -p);
    return df_quick(p, fmaf(a.h, b.l, fmaf(a.l, b.h, e)));
}
// c - a b
__device__ __forceinline__ df df_fms(df c, df a, df b) { return df_add(c, df_neg(df_mul(a, b))); }
// 1 / a: FP32 reciprocal refined by one Newton step in pairs
__device__ __forceinline__ df df_rcp(df a)
{
    const float r = 1.0f / a.h;
    const df e = df_add({1.0f, 0.0f}, df_neg(df_mul(a, {r, 0.0f})));  // 1 - a r
    return df_add({r, 0.0f}, df_mul({r, 0.0f}, e));
}
// a^{-1/2}: FP32 reciprocal square root refined by one Newton step in pairs
__device__ __forceinline__ df df_rsqrt(df a)
{
    const float y = rsqrtf(a.h);
    const float p = y * y;
    const df yy = {p, fmaf(y, y, -p)};
    const df e = df_add({1.0f, 0.0f}, df_neg(df_mul(a, yy)));  // 1 - a y^2
    return df_add({y, 0.0f}, df_mul({0.5f * y, 0.0f}, e));
}
// sqrt(a) for a > 0: y = sqrt(a.h) in FP32, then y + (a - y^2) / (2 y) with the square exact
__device__ __forceinline__ df df_sqrt(df a)
{
    if (!(a.h > 0.0f)) return {0.0f, 0.0f};
    const float y = sqrtf(a.h);
    const float p = y * y;
    const df e = df_add(a, {-p, -fmaf(y, y, -p)});  // a - y^2
    return df_quick(y, e.h / (2.0f * y));
}
__device__ __forceinline__ df df_of(double x)
{
    const float h = (float)x;
    return {h, (float)(x - (double)h)};
}
__device__ __forceinline__ double df_dbl(df a) { return (double)a.h + (double)a.l; }

// (sh, sl) += x * y with the product's rounding error (FMA) and the sum's (TwoSum) carried in sl
// (Dot2, Ogita, Rump and Oishi 2005).
__device__ __forceinline__ void dot2_add(float& sh, float& sl, float x, float y)
{
    const float p = x * y;
    const float pe = fmaf(x, y, -p);
    const df t = df_two_sum(sh, p);
    sh = t.h;
    sl += t.l + pe;
}

}  // namespace rq
