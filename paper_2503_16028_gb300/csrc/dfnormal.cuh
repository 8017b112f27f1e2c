// Box-Muller normals in double-float arithmetic on the FP32 pipes.
//
// The proposal needs d standard normals per particle and step; in FP64 the
// logarithm and sin/cos of the Box-Muller transform make the proposal kernel
// FP64-bound on GB300.  Here both are evaluated in df32 from the exact integer
// form of the Philox uniforms, to ~1e-14 relative, and only the final
// products go back to FP64:
//   U1 = (2 a + 1) 2^-54, R = sqrt(-2 log U1),  t = 2 U2 = (2 b + 1) 2^-53,
//   z0 = R cos(pi t), z1 = R sin(pi t).
// log: U1 = 2^m y with y in [1, 2); F = 1 + j/64 the nearest table point;
// log y = log F + log1p(s), s = (y - F)/F, |s| <= 2^-7, log1p by its series
// (the terms from s^4 on in FP32).  For F >= 1.5 the table holds log(F/2) and
// m grows by one, so that log U1 never forms a difference of two large terms.
// sin/cos: t = q/2 + r, |r| <= 1/4, Taylor series of sin and cos of pi r (the
// terms from the 11th / 10th power on in FP32), and the quarter-turn symmetry.
#pragma once
#include "df32.cuh"

namespace smcgm {

// Host-computed constants (df32 pairs as float2: x = hi, y = lo).
struct NormalConsts {
    float ln2a, ln2b, ln2c;   // ln 2 = a + b + c, a with 16 significant bits (m a exact for |m| < 256)
    float2 pi;                // pi
    float2 s3, s5, s7, s9;    // 1/3!, 1/5!, 1/7!, 1/9!
    float2 c2, c4, c6, c8;    // 1/2!, 1/4!, 1/6!, 1/8!
    float2 third;             // 1/3
};

// Table of the logarithm: for j = 0..64, F_j = 1 + j/64,
// tab[j] = (log F_j or, for j >= 32, log(F_j / 2), as df32), tab[65 + j] = 1/F_j.
constexpr int NORMAL_TAB = 130;

// v 2^e2 as df32, v < 2^55 (hi: the top 24 significant bits, lo: the rest rounded).
__device__ __forceinline__ df32 df_from_i64(long long v, int e2) {
    const bool neg = v < 0;
    unsigned long long a = (unsigned long long)(neg ? -v : v);
    if (a == 0) return df32{0.f, 0.f};
    const int L = 63 - __clzll((long long)a);
    float hi, lo;
    if (L <= 23) {
        hi = __uint2float_rn((unsigned)a);
        lo = 0.f;
    } else {
        const int sh = L - 23;
        const unsigned long long ah = a >> sh;
        hi = __fmul_rn(__uint2float_rn((unsigned)ah), __uint_as_float((unsigned)(127 + sh) << 23));
        lo = __uint2float_rn((unsigned)(a - (ah << sh)));
    }
    const float sc = __uint_as_float((unsigned)(127 + e2) << 23);   // 2^e2, |e2| < 127
    df32 r;
    fast_two_sum(__fmul_rn(hi, sc), __fmul_rn(lo, sc), r.hi, r.lo);
    if (neg) r = df_neg(r);
    return r;
}

__device__ __forceinline__ df32 dfc(float2 c) { return df32{c.x, c.y}; }

// sqrt of a positive df32 (one correction of the FP32 square root: y + (x - y^2) / (2 y)).
__device__ __forceinline__ df32 df_sqrt(df32 x) {
    const float y = __fsqrt_rn(x.hi);
    float p, pe;
    two_prod(y, y, p, pe);
    const float e = __fadd_rn(__fadd_rn(__fsub_rn(x.hi, p), -pe), x.lo);
    df32 r;
    fast_two_sum(y, __fdiv_rn(e, __fmul_rn(2.f, y)), r.hi, r.lo);
    return r;
}

// log U for U = (2 a + 1) 2^-54, a < 2^53.
__device__ __forceinline__ df32 df_log_u54(unsigned long long a, const float2* tab, const NormalConsts& C) {
    const unsigned long long v = 2ull * a + 1ull;                    // odd, < 2^54
    const int L = 63 - __clzll((long long)v);                          // msb
    const unsigned long long vv = v << (53 - L);                       // msb at bit 53: y = vv 2^-53
    const int j = (int)((((vv >> 46) & 127ull) + 1ull) >> 1);          // nearest F_j = 1 + j/64
    const long long d = (long long)vv - ((long long)(64 + j) << 47);   // (y - F_j) 2^53, |d| <= 2^46
    const int m = (L - 54) + (j >= 32 ? 1 : 0);
    const df32 s = df_mul(df_from_i64(d, -53), dfc(tab[65 + j]));     // (y - F) / F
    // log1p(s) = s - s^2/2 + s^3/3 - s^4 (1/4 - s/5 + s^2/6 - s^3/7 + s^4/8 - s^5/9)
    const float sh = s.hi;
    const float q = fmaf(sh, fmaf(sh, fmaf(sh, fmaf(sh, fmaf(sh, -1.f / 9.f, 1.f / 8.f), -1.f / 7.f), 1.f / 6.f), -1.f / 5.f), 0.25f);
    const df32 s2 = df_mul(s, s);
    const df32 s3 = df_mul(s2, s);
    const float t4 = __fmul_rn(__fmul_rn(s2.hi, s2.hi), q);
    df32 l = df_add(s, df32{-0.5f * s2.hi, -0.5f * s2.lo});
    l = df_add(l, df_mul(s3, dfc(C.third)));
    l = df_add_f(l, -t4);
    // + m ln2 + tab[j]
    const float mf = (float)m;
    float p2, e2;
    two_prod(mf, C.ln2b, p2, e2);
    df32 ml;
    fast_two_sum(__fmul_rn(mf, C.ln2a), p2, ml.hi, ml.lo);             // m a is exact; |m a| >= |m b|
    ml.lo = __fadd_rn(ml.lo, fmaf(mf, C.ln2c, e2));
    fast_two_sum(ml.hi, ml.lo, ml.hi, ml.lo);
    return df_add(df_add(ml, dfc(tab[j])), l);
}

// sin(pi t) and cos(pi t) for t = (2 b + 1) 2^-53, b < 2^52 (so 0 < t < 1... 2).
__device__ __forceinline__ void df_sincospi_u53(unsigned long long b, const NormalConsts& C, df32& sn, df32& cs) {
    const long long V = (long long)(2ull * b + 1ull);                   // t = V 2^-53 in (0, 2)
    const int q = (int)((V + (1ll << 51)) >> 52);                      // nearest multiple of 1/2, 0..4
    const long long D = V - ((long long)q << 52);                      // r = D 2^-53, |r| <= 1/4
    const df32 x = df_mul(df_from_i64(D, -53), dfc(C.pi));             // pi r, |x| <= pi/4
    const df32 u = df_mul(x, x);
    const float y = u.hi;
    // sin x = x (1 - u/3! + u^2/5! - u^3/7! + u^4/9! - u^5 S), S = 1/11! - u/13! + u^2/15! - u^3/17!
    const float S = fmaf(y, fmaf(y, fmaf(y, -1.f / 355687428096000.f, 1.f / 1307674368000.f), -1.f / 6227020800.f), 1.f / 39916800.f);
    df32 ps = df_sub_acc(dfc(C.s9), df_mul(u, df32{S, 0.f}));
    ps = df_sub_acc(dfc(C.s7), df_mul(u, ps));
    ps = df_sub_acc(dfc(C.s5), df_mul(u, ps));
    ps = df_sub_acc(dfc(C.s3), df_mul(u, ps));
    ps = df_sub_acc(df32{1.f, 0.f}, df_mul(u, ps));
    const df32 sx = df_mul(x, ps);
    // cos x = 1 - u/2! + u^2/4! - u^3/6! + u^4/8! - u^5 Cc, Cc = 1/10! - u/12! + u^2/14! - u^3/16!
    const float Cc = fmaf(y, fmaf(y, fmaf(y, -1.f / 20922789888000.f, 1.f / 87178291200.f), -1.f / 479001600.f), 1.f / 3628800.f);
    df32 pc = df_sub_acc(dfc(C.c8), df_mul(u, df32{Cc, 0.f}));
    pc = df_sub_acc(dfc(C.c6), df_mul(u, pc));
    pc = df_sub_acc(dfc(C.c4), df_mul(u, pc));
    pc = df_sub_acc(dfc(C.c2), df_mul(u, pc));
    const df32 cx = df_sub_acc(df32{1.f, 0.f}, df_mul(u, pc));
    // pi t = q pi/2 + x
    switch (q & 3) {
        case 0: sn = sx; cs = cx; break;
        case 1: sn = cx; cs = df_neg(sx); break;
        case 2: sn = df_neg(sx); cs = df_neg(cx); break;
        default: sn = df_neg(cx); cs = sx; break;
    }
}

}  // namespace smcgm
