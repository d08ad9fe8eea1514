// Double-float arithmetic on the FP32 cores (FP64 issue is a small fraction
// of FP32 on this part): a value as hi + lo, two FP32 numbers; each
// multiply-add takes the product's rounding error from an FMA and the sum's
// from TwoSum (Knuth), both collected in a compensation term, which keeps
// about 2^-48 of each sum's terms.
#pragma once

namespace tl {

struct df2 {
    float hi, lo;
};
__device__ __forceinline__ df2 df_of(double x) {
    const float h = (float)x;
    return {h, (float)(x - (double)h)};
}
// (s, c) += a * b; the intrinsics keep the compiler from contracting or
// reassociating the error terms
__device__ __forceinline__ void df_mac(float& s, float& c, df2 a, df2 b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    const float t = __fadd_rn(s, p);
    const float bp = __fsub_rn(t, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp));
    s = t;
    c = __fadd_rn(c, __fadd_rn(err, e));
}
// a * b rounded to a double-float (the lo * lo term, 2^-48 of the
// product, dropped)
__device__ __forceinline__ df2 df_mul(df2 a, df2 b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    const float h = __fadd_rn(p, e);
    return {h, __fsub_rn(e, __fsub_rn(h, p))};
}
__device__ __forceinline__ df2 df_norm(float s, float c) {
    const float h = __fadd_rn(s, c);
    return {h, __fsub_rn(c, __fsub_rn(h, s))};
}

}  // namespace tl
