// Double-float elementary functions and the saturation of q0 (appendix) for
// the FP32-mixed q0 steps, plain and spin-polarised:
//  * sums of positive terms use the sloppy double-float addition (exact
//    two-sum of the high parts); sums that may cancel use the full one;
//  * reciprocals: FP32 reciprocal plus one correction with the exact remainder;
//  * ln x = e ln2 + ln c_i + ln(1 + r), x = 2^e m, m = c_i (1 + r), c_i from
//    a 64-entry table (c_0 = 1), |r| <= 1/64, ln(1+r) to r^8;
//  * exp(-S) = 2^(-k/64) exp(-r), |r| <= ln2/128, 2^(-j/64) from a table;
//  * saturation: with t = q_raw / q_cut and S = sum_{m<=12} t^m/m, for t < 0.4
//    the identity S = -ln(1 - t) - R, R = sum_{m>=13} t^m/m, gives
//    1 - e^-S = t - (1 - t) expm1(R) and h'(x) = e^R (1 - t^12) without
//    cancellation; for 0.4 <= t <= 1.5 S and e^-S are formed directly; for
//    t > 1.5, S > 40 and q0 = q_cut to double precision.
#pragma once
#include "dfloat.cuh"

namespace vdwgb {

// the ln and exp tables (shared memory, filled by the whole block):
// lnt[i] = {1/c_i in FP32, ln c_i hi, ln c_i lo, 0}, ex2[j] = 2^(-j/64) hi, lo
__device__ __forceinline__ void load_df_tables(float4 *lnt, float2 *ex2) {
    for (int i = threadIdx.x; i < 64; i += blockDim.x) {
        const double c = i == 0 ? 1.0 : 1.0 + (i + 0.5) / 64.0;
        const float inv = (float)(1.0 / c);
        const double lc = -log((double)inv);          // ln of 1 / inv exactly
        const float lh = (float)lc;
        lnt[i] = make_float4(inv, lh, (float)(lc - (double)lh), 0.f);
        const double v = exp2(-(double)i / 64.0);
        const float vh = (float)v;
        ex2[i] = make_float2(vh, (float)(v - (double)vh));
    }
}

// a + b for a, b of one sign (sloppy addition: exact two-sum of the high parts)
__device__ __forceinline__ dfl df_add_pos(dfl a, dfl b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    e += a.lo + b.lo;
    return df_quick(s, e);
}

__device__ __forceinline__ dfl df_rcp_fast(dfl b) {
    const float r = __frcp_rn(b.hi);
    float e = fmaf(-b.hi, r, 1.0f);      // exact remainder of the rounded reciprocal
    e = fmaf(-b.lo, r, e);
    return df_quick(r, r * e);
}

// ln(1 + r) for |r| <= 1/64 in double-float: r - r^2/2 + r^3/3 in
// double-float plus the FP32 tail r^4 (-1/4 + r/5 - r^2/6 + r^3/7 - r^4/8)
__device__ __forceinline__ dfl df_ln1p_small(float rh, float rl) {
    const float p2 = rh * rh;
    const float e2 = fmaf(rh, rh, -p2) + 2.f * rh * rl;
    const float p3 = p2 * rh;
    const float e3 = fmaf(p2, rh, -p3) + e2 * rh;
    const dfl c3 = df_mul(dfl{p3, e3}, DF(1.0 / 3.0));
    float tail = fmaf(rh, -0.125f, 0.14285715f);
    tail = fmaf(rh, tail, -0.16666667f);
    tail = fmaf(rh, tail, 0.2f);
    tail = fmaf(rh, tail, -0.25f);
    tail *= p2 * p2;
    // |r^2/2| <= |r|/128 and |r^3/3| << |r - r^2/2|: fast two-sums
    const float s = rh - 0.5f * p2;
    float se = ((rh - s) - 0.5f * p2) + (rl - 0.5f * e2);
    const float s2 = s + c3.hi;
    se += ((s - s2) + c3.hi) + c3.lo + tail;
    return df_quick(s2, se);
}

// ln(1 + u), u >= 0: the series on u itself below 1/64 (no rounding of 1 + u),
// else x = 1 + u = 2^e m, m = c_i (1 + r), ln x = e ln2 + ln c_i + ln(1 + r)
__device__ __forceinline__ dfl df_log1p(dfl u, const float4 *lnt) {
    if (u.hi < 0.015625f) return df_ln1p_small(u.hi, u.lo);
    const dfl x = df_add_pos(DF(1.0), u);
    const int bits = __float_as_int(x.hi);
    const int e = ((bits >> 23) & 0xff) - 127;
    const int i = (bits >> 17) & 63;
    const float sc = __int_as_float((127 - e) << 23);     // 2^-e
    const float mh = x.hi * sc, ml = x.lo * sc;
    const float4 T = lnt[i];
    const float p = mh * T.x;
    const float pe = fmaf(mh, T.x, -p);
    float rh, rl;
    two_sum(p - 1.0f, fmaf(ml, T.x, pe), rh, rl);         // r = m / c_i - 1 (p - 1 exact)
    const dfl l1p = df_ln1p_small(rh, rl);
    const dfl el = df_mulf(DF(0.69314718055994530942), (float)e);
    return df_add(df_add_pos(el, dfl{T.y, T.z}), l1p);
}

// exp(-S), S >= 0
__device__ __forceinline__ dfl df_exp_neg2(dfl S, const float2 *ex2) {
    const float kf = rintf(S.hi * 92.332482616893656f);   // 64 / ln2
    const int k = (int)kf;
    // ln2/64 = C1 + C2 + C3, C1 with 11 significant bits (k * C1 exact for k < 8192)
    const float C1 = 0.010833740234375f, C2 = -3.3155381516e-6f, C3 = 2.5727683872e-14f;
    const float a = S.hi - kf * C1;
    const float bh = kf * C2;
    const float bl = fmaf(kf, C2, -bh);
    float rh, rl;
    two_sum(a, -bh, rh, rl);
    rl += S.lo - bl - kf * C3;
    const dfl r = df_quick(rh, rl);
    // exp(-r) = 1 - r + r^2/2 - r^3/6 + r^4/24 - r^5/120
    float oh, ol;
    two_sum(1.0f, -r.hi, oh, ol);
    ol -= r.lo;
    const float p2 = r.hi * r.hi;
    const float e2 = fmaf(r.hi, r.hi, -p2) + 2.f * r.hi * r.lo;
    float tail = fmaf(r.hi, -8.3333333e-3f, 4.1666668e-2f);
    tail = fmaf(r.hi, tail, -0.16666667f);
    tail *= p2 * r.hi;
    dfl E = df_add_pos(df_quick(oh, ol), dfl{0.5f * p2, 0.5f * e2});
    E.lo += tail;
    const float2 Tj = ex2[k & 63];
    const dfl v = df_mul(dfl{Tj.x, Tj.y}, E);
    const float sc = __int_as_float((127 - (k >> 6)) << 23);
    return dfl{v.hi * sc, v.lo * sc};
}

// h_a(x) / a = 1 - exp(-sum_{m=1}^{12} t^m / m), t = x / a, times qcut = a,
// and h'(x) (FP32, 0 where q0 = q_cut)
__device__ __forceinline__ dfl df_saturate(dfl t, float qcut, const float2 *ex2, float &dh) {
    dfl q0;
    dh = 0.f;
    if (t.hi > 1.5f) {
        q0 = dfl{qcut, 0.f};
    } else if (t.hi < 0.4f) {
        const float th = t.hi;
        float R = 1.f / 30.f;
#pragma unroll
        for (int m = 29; m >= 13; --m) R = fmaf(R, th, 1.f / (float)m);
        const float t2 = th * th, t4 = t2 * t2, t12 = t4 * t4 * t4;
        R *= t12 * th;
        const float E = fmaf(0.5f * R, R, R);                 // expm1(R)
        float omh, oml;
        two_sum(1.0f, -t.hi, omh, oml);
        oml -= t.lo;
        const dfl w = df_mulf(df_quick(omh, oml), E);         // (1 - t) expm1(R)
        const float h = t.hi - w.hi;                          // |w| << t: fast two-sum
        const float he = ((t.hi - h) - w.hi) + t.lo - w.lo;
        q0 = df_mulf(df_quick(h, he), qcut);
        dh = (1.f + E) * (1.f - t12);
    } else {
        dfl S = DF(1.0 / 12.0);
#pragma unroll
        for (int m = 11; m >= 1; --m) S = df_add_pos(df_mul(S, t), DF(1.0 / (double)m));
        S = df_mul(S, t);
        const dfl ex = df_exp_neg2(S, ex2);
        const float h = 1.0f - ex.hi;                         // ex <= e^-0.46: fast two-sum
        const float he = ((1.0f - h) - ex.hi) - ex.lo;
        q0 = df_mulf(df_quick(h, he), qcut);
        float dS = 1.f;
#pragma unroll
        for (int m = 0; m < 11; ++m) dS = fmaf(dS, t.hi, 1.f);   // sum_{m=0}^{11} t^m
        dh = ex.hi * dS;
    }
    return q0;
}

}  // namespace vdwgb
