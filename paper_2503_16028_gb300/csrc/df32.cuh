// Double-float ("df32") arithmetic: a value is the unevaluated sum hi + lo of
// two FP32 numbers with |lo| <= ulp(hi)/2, about 48 significant bits.  The
// error-free transformations are Knuth's TwoSum (The Art of Computer
// Programming, vol. 2, 4.2.2), Dekker's FastTwoSum and the FMA form of
// Dekker's product (T. J. Dekker, "A floating-point technique for extending
// the available precision", Numer. Math. 18, 1971).  On GB300 FP32 runs ~58x
// faster than FP64, so the FP64-accurate coefficient set-up and residual of
// the mixed-precision refinement run in df32 on the FP32 pipes.  Nothing here
// may be reassociated or contracted: sums and products use the _rn intrinsics,
// and products that must be exact use explicit fmaf.
#pragma once
#include <cuda_runtime.h>

namespace smcgm {

struct df32 {
    float hi, lo;
};

// s + e = a + b exactly (any magnitudes).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// s + e = a + b exactly, given |a| >= |b| or a == 0.
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

// a + b with the lower parts added in plain FP32 (relative error ~2^-46
// unless the two values cancel to far below their own size).
__device__ __forceinline__ df32 df_add(df32 a, df32 b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    df32 r;
    fast_two_sum(s, e, r.hi, r.lo);
    return r;
}

__device__ __forceinline__ df32 df_neg(df32 a) { return df32{-a.hi, -a.lo}; }

// a - b with both the high and the low parts subtracted error-free and the
// four pieces renormalised (the accurate double-double addition of Bailey's
// QD library): relative error ~2^-46 of the result even when a and b cancel.
__device__ __forceinline__ df32 df_sub_acc(df32 a, df32 b) {
    float s1, e1, s2, e2;
    two_sum(a.hi, -b.hi, s1, e1);
    two_sum(a.lo, -b.lo, s2, e2);
    e1 = __fadd_rn(e1, s2);
    fast_two_sum(s1, e1, s1, e1);
    e1 = __fadd_rn(e1, e2);
    df32 r;
    fast_two_sum(s1, e1, r.hi, r.lo);
    return r;
}

// p + e = a * b exactly (FMA form of Dekker's product).
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
    p = __fmul_rn(a, b);
    e = fmaf(a, b, -p);
}

// a * b (relative error ~2^-46).
__device__ __forceinline__ df32 df_mul(df32 a, df32 b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);                 // exact low part of hi * hi
    e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
    df32 r;
    fast_two_sum(p, e, r.hi, r.lo);
    return r;
}

// a + x for a single float x.
__device__ __forceinline__ df32 df_add_f(df32 a, float x) {
    float s, e;
    two_sum(a.hi, x, s, e);
    e = __fadd_rn(e, a.lo);
    df32 r;
    fast_two_sum(s, e, r.hi, r.lo);
    return r;
}

// A double as df32 by bit manipulation, no FP64 instruction: hi keeps the
// top 24 significant bits (truncated) and lo the next 24 of the remaining 29,
// so hi + lo = v to ~2^-48 relative.  Zero for |v| < 2^-126; the caller
// keeps |v| far below the FP32 overflow.
__device__ __forceinline__ df32 df_from_double_bits(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const unsigned hw = (unsigned)(b >> 32), lw = (unsigned)b;
    const int e = (int)((hw >> 20) & 0x7ffu);                 // biased FP64 exponent
    if (e < 1023 - 126) return df32{0.f, 0.f};
    const unsigned sign = hw & 0x80000000u;
    const float hi = __uint_as_float(sign | ((unsigned)(e - 1023 + 127) << 23) | ((hw & 0xfffffu) << 3) | (lw >> 29));
    const int pe = e - 1075 + 127;                            // biased FP32 exponent of 2^(e - 1075)
    float lo = pe > 0 ? __fmul_rn(__uint2float_rn(lw & 0x1fffffffu), __uint_as_float((unsigned)pe << 23)) : 0.f;
    if (sign) lo = -lo;
    df32 r;
    fast_two_sum(hi, lo, r.hi, r.lo);
    return r;
}

// Constants of df_exp: ln2/64 = c1 + c2 + c3 (c1 with 11 significant bits, so
// k c1 is exact for |k| < 2^13) and the table 2^(j/64) = thi[j] + tlo[j].
struct ExpConsts {
    float c1, c2, c3;
};

// e^x for a df32 x with |x| < 64, by Tang's table-driven method (P. T. P.
// Tang, "Table-driven implementation of the exponential function in IEEE
// floating-point arithmetic", ACM TOMS 15(2), 1989): x = (64 m + j) ln2/64 + r
// with |r| <= ln2/128, e^x = 2^m 2^(j/64) e^r, and e^r - 1 = r + r^2 t with
// t = 1/2 + r/6 + r^2/24 + r^3/120 (the first omitted term, r^6/720, is below
// 4e-17).  The reduction is exact up to ~2^-53 |x| from the three-part ln2/64,
// and the result has a relative error ~1e-14.  `tab` holds the 64 table pairs.
__device__ __forceinline__ df32 df_exp(df32 x, const float2* tab, const ExpConsts& C) {
    const float kf = rintf(__fmul_rn(x.hi, 92.332482616893657f));   // 64 / ln2
    const int k = (int)kf;
    const int j = k & 63, m = k >> 6;                               // k = 64 m + j
    const float r1 = fmaf(-kf, C.c1, x.hi);                         // exact
    df32 r;
    two_sum(r1, x.lo, r.hi, r.lo);
    float p2, e2;
    two_prod(kf, C.c2, p2, e2);
    r = df_sub_acc(r, df32{p2, e2});
    r = df_add_f(r, -__fmul_rn(kf, C.c3));
    const float s = __fmul_rn(r.hi, fmaf(r.hi, fmaf(r.hi, 1.f / 120.f, 1.f / 24.f), 1.f / 6.f));
    df32 t;
    fast_two_sum(0.5f, s, t.hi, t.lo);
    const df32 em1 = df_add(r, df_mul(df_mul(r, r), t));
    const float2 tj = tab[j];
    const df32 T{tj.x, tj.y};
    const df32 y = df_add(T, df_mul(T, em1));
    const float sc = __uint_as_float((unsigned)(m + 127) << 23);   // 2^m, |m| < 127
    return df32{__fmul_rn(y.hi, sc), __fmul_rn(y.lo, sc)};
}

// 2 / d for a positive df32 d: one Newton step from the FP32 reciprocal,
// 2/d = y0 + y0 (2 - d y0) / 2 with the residual 2 - d y0 formed by FMA.
__device__ __forceinline__ df32 df_two_over(df32 d) {
    const float y0 = __fmul_rn(2.f, __frcp_rn(d.hi));
    const float rho = fmaf(-d.lo, y0, fmaf(-d.hi, y0, 2.f));
    df32 r;
    fast_two_sum(y0, __fmul_rn(__fmul_rn(rho, y0), 0.5f), r.hi, r.lo);
    return r;
}

}  // namespace smcgm
