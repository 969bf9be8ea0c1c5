// Double-float ("df") arithmetic on the FP32 pipe: a value is hi + lo with two
// floats, |lo| <= ulp(hi)/2, about 48 significant bits.  On GB300 FP64 FMA
// throughput is about 1/62 of FP32 (measured 1.20 against 74.8 TFLOP/s), so
// the mixed form evaluates the entropy functional (a log per node) in df
// instead of float64.
//
// Error-free transformations: TwoSum (Knuth), FastTwoSum (Dekker), TwoProd
// via FMA.  Logarithm: table-driven reduction in the manner of Tang (1990,
// "Table-driven implementation of the logarithm function in IEEE
// floating-point arithmetic"): x = 2^k m, m in [1,2), F = 1 + j/128 nearest
// to m, r = (m - F)/F with |r| <= 2^-8, log x = k log 2 + log F + log1p(r),
// log1p(r) = r - r^2/2 + r^2 c with c = r/3 - r^2/4 + r^3/5 - r^4/6: r and
// r^2/2 in df, the term r^2 c (below 2^-25) in float, whose rounding (about
// 2^-49) and the series' truncation (r^7/7, below 2^-58) stay under the df
// rounding of the sum.  log F and 1/F come from a host-built table (long
// double, split into float pairs).
#pragma once

#include <cstdint>

namespace perrk {

struct df {
    float hi, lo;
};

struct DfConst {
    df ln2, gm1, gam;   // log 2, gamma - 1, gamma as float pairs
};

__device__ __forceinline__ df df_two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return df{s, (a - (s - bb)) + (b - bb)};
}

__device__ __forceinline__ df df_fast(float a, float b) {  // |a| >= |b|
    const float s = a + b;
    return df{s, b - (s - a)};
}

__device__ __forceinline__ df df_add(df x, df y) {
    df s = df_two_sum(x.hi, y.hi);
    df t = df_two_sum(x.lo, y.lo);
    float e = s.lo + t.hi;
    s = df_fast(s.hi, e);
    e = s.lo + t.lo;
    return df_fast(s.hi, e);
}

__device__ __forceinline__ df df_neg(df x) { return df{-x.hi, -x.lo}; }

__device__ __forceinline__ df df_sub(df x, df y) { return df_add(x, df_neg(y)); }

__device__ __forceinline__ df df_mul(df x, df y) {
    const float p = x.hi * y.hi;
    float e = fmaf(x.hi, y.hi, -p);
    e = fmaf(x.hi, y.lo, e);
    e = fmaf(x.lo, y.hi, e);
    return df_fast(p, e);
}

__device__ __forceinline__ df df_mul_f(df x, float f) {
    const float p = x.hi * f;
    float e = fmaf(x.hi, f, -p);
    e = fmaf(x.lo, f, e);
    return df_fast(p, e);
}

// 1 / x for a df x: the MUFU reciprocal of x.hi refined by one Newton step in
// float (about 0.5 ulp), then corrected by the df residual t = 1 - x r
// (products exact in the FMAs): r (1 + t), relative error about 2^-46.
__device__ __forceinline__ df df_rcp(df x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x.hi));
    r = fmaf(r, fmaf(-x.hi, r, 1.0f), r);
    float t = fmaf(-x.hi, r, 1.0f);
    t = fmaf(-x.lo, r, t);
    return df_fast(r, r * t);
}

// x + y f (df plus df times float), the step of the direction sums
// d = sum_i b_i K_i: the product is left unnormalised (ph + pl, its FMA error
// and y.lo f in pl), and only the high parts are added by TwoSum; the three
// low-order terms are summed in float.  Error about 2^-46 of the larger
// operand, far below the FP32 rounding that the K_i themselves carry; 14
// FP32 operations against 26 for df_add(x, df_mul_f(y, f)).
__device__ __forceinline__ df df_fma_f(df x, df y, float f) {
    const float ph = y.hi * f;
    const float pl = fmaf(y.lo, f, fmaf(y.hi, f, -ph));
    const df s = df_two_sum(x.hi, ph);
    return df_fast(s.hi, s.lo + (x.lo + pl));
}

// x + f (df plus float)
__device__ __forceinline__ df df_add_f(df x, float f) {
    const df s = df_two_sum(x.hi, f);
    return df_fast(s.hi, s.lo + x.lo);
}

// float64 -> df (one FP64 subtraction) and back (one FP64 addition).
__device__ __forceinline__ df df_from(double d) {
    const float hi = __double2float_rn(d);
    return df{hi, __double2float_rn(d - (double)hi)};
}

__device__ __forceinline__ double df_to(df x) { return (double)x.hi + (double)x.lo; }

// log(x) for x > 0 (x.hi a normal float).  tab[j] = (log F_j hi, lo, 1/F_j hi, lo).
__device__ __forceinline__ df df_log(df x, const float4 *__restrict__ tab, const DfConst &K) {
    const uint32_t bits = __float_as_uint(x.hi);
    const int k = (int)((bits >> 23) & 0xffu) - 127;
    const float mh = __uint_as_float((bits & 0x7fffffu) | 0x3f800000u);   // hi / 2^k in [1, 2)
    const float ml = x.lo * __uint_as_float((uint32_t)(127 - k) << 23);   // lo / 2^k
    const int j = __float2int_rn((mh - 1.0f) * 128.0f);
    const float F = 1.0f + (float)j * 0.0078125f;
    const float4 t = __ldg(tab + j);
    // r = (m - F) / F: m_hi - F is exact (Sterbenz), then times 1/F in df
    const df d = df_two_sum(mh - F, ml);
    const df r = df_mul(d, df{t.z, t.w});
    const float rh = r.hi;
    const float c = rh * fmaf(rh, fmaf(rh, fmaf(rh, -1.0f / 6.0f, 0.2f), -0.25f), 1.0f / 3.0f);
    const df r2 = df_mul(r, r);
    const df l1p = df_add_f(df_add(r, df{-0.5f * r2.hi, -0.5f * r2.lo}), r2.hi * c);   // r - r^2/2 + r^2 c
    const df kl = df_mul_f(K.ln2, (float)k);
    return df_add(df_add(kl, df{t.x, t.y}), l1p);
}

}  // namespace perrk
