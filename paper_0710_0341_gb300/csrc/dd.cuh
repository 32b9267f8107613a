// Double-float real numbers for the stencil template of dslash_site.cuh.
//
// A dd is the unevaluated sum hi + lo of two FP32 numbers (|lo| <= ulp(hi)),
// about 48 significant bits. Instantiating the stencil with T = dd runs the
// FP64 mode's arithmetic on the FP32 pipes, which GB300 issues at 64 times
// its FP64 rate; the loads and stores stay FP64 (double2), so the memory
// traffic and its indexing are those of the FP64 kernel.
//
// Arithmetic by the error-free transformations of Dekker (1971) and Knuth
// (TAOCP vol. 2): two_sum (a + b = s + e exactly), fast_two_sum (the same
// when |a| >= |b|), and the FMA form of two_prod (a * b = p + e exactly).
// Sums and products keep the low-order terms in FP32, so each operation has
// a relative error of a few units of 2^-47 of its operands' size.
//
// FP64 <-> dd conversions avoid the FP64 pipe: a double is cut into hi (its
// sign, exponent and leading 24 significant bits, truncated) and lo (the next
// 23 bits, as an exact FP32 integer scaled by a power of two) with integer
// operations only; the 6 trailing bits of the 52-bit mantissa are dropped
// (relative error below 2^-46). Values below 2^-80 in magnitude keep only hi,
// values below 2^-126 become 0, magnitudes of 2^128 or more become infinite
// and a NaN stays a NaN.
#pragma once

#include <stdint.h>
#include <string.h>

#include "df.cuh"
#include "dslash_site.cuh"

namespace ovl_stencil {

// IEEE single operations that the compiler must neither fuse nor reorder
OVL_HD float f_add(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fadd_rn(a, b);
#else
    return a + b;
#endif
}
OVL_HD float f_sub(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fsub_rn(a, b);
#else
    return a - b;
#endif
}
OVL_HD float f_mul(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fmul_rn(a, b);
#else
    return a * b;
#endif
}
OVL_HD float f_fma(float a, float b, float c) {
#ifdef __CUDA_ARCH__
    return __fmaf_rn(a, b, c);
#else
    return std::fmaf(a, b, c);
#endif
}
OVL_HD float u32_as_f32(uint32_t u) {
#ifdef __CUDA_ARCH__
    return __uint_as_float(u);
#else
    float f;
    memcpy(&f, &u, 4);
    return f;
#endif
}
OVL_HD uint64_t f64_bits(double x) {
#ifdef __CUDA_ARCH__
    return (uint64_t)__double_as_longlong(x);
#else
    uint64_t u;
    memcpy(&u, &x, 8);
    return u;
#endif
}

OVL_HD void dd_two_sum(float a, float b, float& s, float& e) {
    s = f_add(a, b);
    const float bb = f_sub(s, a);
    e = f_add(f_sub(a, f_sub(s, bb)), f_sub(b, bb));
}
OVL_HD void dd_fast_two_sum(float a, float b, float& s, float& e) {
    s = f_add(a, b);
    e = f_sub(b, f_sub(s, a));
}

struct dd {
    float hi, lo;
    dd() = default;
    OVL_HD dd(int v) : hi((float)v), lo(0.f) {}
    OVL_HD dd(float h, float l) : hi(h), lo(l) {}
    // cut a double into hi + lo with integer operations (see the file header)
    OVL_HD dd(double x) {
        const uint64_t b = f64_bits(x);
        const uint32_t w1 = (uint32_t)(b >> 32), w0 = (uint32_t)b;
        const uint32_t sgn = w1 & 0x80000000u;
        const int e = (int)((w1 >> 20) & 0x7ffu);  // biased FP64 exponent
        hi = 0.f;
        lo = 0.f;
        if (e >= 1151) {  // |x| >= 2^128, inf or NaN: inf or NaN (a NaN stays a NaN)
            const bool nan = e == 2047 && ((w1 & 0xfffffu) | w0);
            hi = u32_as_f32(sgn | 0x7f800000u | (nan ? 0x400000u : 0u));
        } else if (e >= 897) {  // |x| >= 2^-126: hi keeps the leading 24 bits (23 stored)
            const uint32_t m23 = ((w1 & 0xfffffu) << 3) | (w0 >> 29);
            hi = u32_as_f32(sgn | ((uint32_t)(e - 896) << 23) | m23);
            const uint32_t rem = (w0 & 0x1fffffffu) >> 6;  // next 23 bits
            if (e >= 943 && rem) {                            // 2^(e-1069) is a normal FP32
                const float r = f_sub(u32_as_f32(0x4b000000u | rem), 8388608.0f);  // exactly rem
                const float l = f_mul(r, u32_as_f32((uint32_t)(e - 942) << 23));
                lo = sgn ? -l : l;
            }
        }
    }
    OVL_HD explicit operator double() const { return (double)hi + (double)lo; }
};

OVL_HD dd operator-(dd a) { return dd(-a.hi, -a.lo); }
OVL_HD dd operator+(dd a, dd b) {
    float s, e;
    dd_two_sum(a.hi, b.hi, s, e);
    e = f_add(e, f_add(a.lo, b.lo));
    dd_fast_two_sum(s, e, s, e);
    return dd(s, e);
}
OVL_HD dd operator-(dd a, dd b) { return a + (-b); }
OVL_HD dd operator*(dd a, dd b) {
    const float p = f_mul(a.hi, b.hi);
    float e = f_fma(a.hi, b.hi, -p);  // the rounding error of p, exactly
    e = f_fma(a.hi, b.lo, e);
    e = f_fma(a.lo, b.hi, e);
    float s, t;
    dd_fast_two_sum(p, e, s, t);
    return dd(s, t);
}
// a * b + c
OVL_HD dd ffma(dd a, dd b, dd c) {
    const float p = f_mul(a.hi, b.hi);
    float e = f_fma(a.hi, b.hi, -p);
    e = f_fma(a.hi, b.lo, e);
    e = f_fma(a.lo, b.hi, e);
    float s, t;
    dd_two_sum(p, c.hi, s, t);
    t = f_add(t, f_add(e, c.lo));
    dd_fast_two_sum(s, t, s, t);
    return dd(s, t);
}

// The link multiplication in double-float: each output is one accumulation of
// three complex products (dfacc_mac of df.cuh: exact hi products, two_sum of
// the hi parts, low-order terms in FP32), renormalised once at the end.
template <>
struct LinkMul<dd> {
    template <bool FWD>
    static OVL_HD void run(const C<dd> (&u)[9], const C<dd> (&h)[6], C<dd> (&g)[6]) {
#pragma unroll
        for (int s = 0; s < 2; s++) {
#pragma unroll
            for (int ai = 0; ai < 3; ai++) {
                dfacc acc;
                dfacc_zero(acc);
#pragma unroll
                for (int b = 0; b < 3; b++) {
                    const C<dd> w = FWD ? u[3 * ai + b] : u[3 * b + ai];
                    const C<dd> x = h[3 * s + b];
                    // U h, or conj(U) h for U^dag h
                    const float wih = FWD ? w.i.hi : -w.i.hi, wil = FWD ? w.i.lo : -w.i.lo;
                    dfacc_mac(acc, make_float2(w.r.hi, wih), make_float2(w.r.lo, wil), make_float2(x.r.hi, x.i.hi),
                              make_float2(x.r.lo, x.i.lo));
                }
                float rs, rt, is, it;
                dd_two_sum(acc.s.x, acc.t.x, rs, rt);
                dd_two_sum(acc.s.y, acc.t.y, is, it);
                g[3 * s + ai] = C<dd>{dd(rs, rt), dd(is, it)};
            }
        }
    }
};

}  // namespace ovl_stencil
