// Double-float ("df") arithmetic: a value is an unevaluated sum hi + lo of two
// FP32 numbers (about 48 significant bits). GB300 issues FP32 at 64 times its
// FP64 rate, so FP64-class accumulations here run on the FP32 pipes with the
// error-free transformations of Dekker (1971) and Knuth (TAOCP vol. 2):
//   two_sum(a, b)  : s + e == a + b exactly      (6 flops, no ordering needed)
//   fast_two_sum   : same when |a| >= |b|        (3 flops)
//   two_prod(a, b) : p + e == a * b exactly      (1 mul + 1 fma)
// The *_rn intrinsics stop the compiler from contracting these steps into
// fused operations, which would break exactness.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

// Every function here is __host__ __device__ (a host build checks the
// arithmetic on the CPU); on the device the single-precision steps use the
// *_rn intrinsics, on the host plain IEEE operations (built without FP
// contraction) with the same results.
#define DF_HD __host__ __device__ __forceinline__
#ifdef __CUDA_ARCH__
#define DF_ADD(a, b) __fadd_rn(a, b)
#define DF_SUB(a, b) __fsub_rn(a, b)
#define DF_MUL(a, b) __fmul_rn(a, b)
#define DF_FMA(a, b, c) __fmaf_rn(a, b, c)
#define DF_DIV(a, b) __fdiv_rn(a, b)
#else
#define DF_ADD(a, b) ((float)(a) + (float)(b))
#define DF_SUB(a, b) ((float)(a) - (float)(b))
#define DF_MUL(a, b) ((float)(a) * (float)(b))
#define DF_FMA(a, b, c) fmaf(a, b, c)
#define DF_DIV(a, b) ((float)(a) / (float)(b))
#endif

struct dfc {  // complex df: (re_hi, im_hi) + (re_lo, im_lo)
    float2 hi, lo;
};

DF_HD void two_sum(float a, float b, float& s, float& e) {
    s = DF_ADD(a, b);
    float bb = DF_SUB(s, a);
    e = DF_ADD(DF_SUB(a, DF_SUB(s, bb)), DF_SUB(b, bb));
}
DF_HD void fast_two_sum(float a, float b, float& s, float& e) {
    s = DF_ADD(a, b);
    e = DF_SUB(b, DF_SUB(s, a));
}
DF_HD void two_prod(float a, float b, float& p, float& e) {
    p = DF_MUL(a, b);
    e = DF_FMA(a, b, -p);
}

// split an FP64 value into hi + lo FP32 (exact to 48 bits)
DF_HD float2 split_d(double x) {
    float h = (float)x;
    float l = (float)(x - (double)h);
    return make_float2(h, l);
}
DF_HD dfc dfc_from(double2 z) {
    float2 a = split_d(z.x), b = split_d(z.y);
    dfc r;
    r.hi = make_float2(a.x, b.x);
    r.lo = make_float2(a.y, b.y);
    return r;
}
DF_HD double2 dfc_to(const dfc& z) {
    return make_double2((double)z.hi.x + (double)z.lo.x, (double)z.hi.y + (double)z.lo.y);
}

// Accumulator for sum_k q_k * g_k with q, g df complex.
// hi parts are carried with two_sum; every rounding error and every cross
// term (hi*lo, lo*hi) goes into the lo accumulator with plain FP32 FMAs
// (their relative size is 2^-24, so FP32 rounding of them costs 2^-48).
struct dfacc {
    float2 s;  // hi sum
    float2 t;  // low-order terms
};
DF_HD void dfacc_zero(dfacc& a) {
    a.s = make_float2(0.f, 0.f);
    a.t = make_float2(0.f, 0.f);
}
// Paired FP32 operations: the real and imaginary parts of a complex
// accumulation travel as one float2. On the device these are Blackwell's
// paired instructions (one instruction, two independent IEEE operations with
// round-to-nearest, never contracted); on the host the two scalar operations.
// Either way each component gets exactly the scalar operation's result.
#ifdef __CUDA_ARCH__
#define F2_ADD(a, b) __fadd2_rn(a, b)
#define F2_MUL(a, b) __fmul2_rn(a, b)
#define F2_FMA(a, b, c) __ffma2_rn(a, b, c)
#else
#define F2_ADD(a, b) make_float2(DF_ADD((a).x, (b).x), DF_ADD((a).y, (b).y))
#define F2_MUL(a, b) make_float2(DF_MUL((a).x, (b).x), DF_MUL((a).y, (b).y))
#define F2_FMA(a, b, c) make_float2(DF_FMA((a).x, (b).x, (c).x), DF_FMA((a).y, (b).y, (c).y))
#endif
DF_HD float2 f2_neg(float2 a) { return make_float2(-a.x, -a.y); }
// two_sum on both components
DF_HD void two_sum2(float2 a, float2 b, float2& s, float2& e) {
    s = F2_ADD(a, b);
    const float2 bb = F2_ADD(s, f2_neg(a));
    e = F2_ADD(F2_ADD(a, f2_neg(F2_ADD(s, f2_neg(bb)))), F2_ADD(b, f2_neg(bb)));
}

// a += q * g (complex), q = qh + ql, g = gh + gl. The real part is
// qh.x gh.x - qh.y gh.y and the imaginary part qh.x gh.y + qh.y gh.x: as pairs,
// (qh.x, qh.x) * (gh.x, gh.y) and (qh.y, qh.y) * (-gh.y, gh.x), each product
// exact as two_prod (p + e), the p's summed into s by two_sum, every rounding
// error and cross term (hi * lo, lo * hi) into t -- the operations and their
// order per component are those of the scalar formulation.
DF_HD void dfacc_mac(dfacc& a, float2 qh, float2 ql, float2 gh, float2 gl) {
    const float2 qx = make_float2(qh.x, qh.x), qy = make_float2(qh.y, qh.y);
    const float2 gr = make_float2(-gh.y, gh.x);  // i * gh
    float2 p, e, s, err;
    p = F2_MUL(qx, gh);
    e = F2_FMA(qx, gh, f2_neg(p));
    two_sum2(a.s, p, s, err);
    a.s = s;
    a.t = F2_ADD(a.t, F2_ADD(err, e));
    p = F2_MUL(qy, gr);
    e = F2_FMA(qy, gr, f2_neg(p));
    two_sum2(a.s, p, s, err);
    a.s = s;
    a.t = F2_ADD(a.t, F2_ADD(err, e));
    a.t = F2_FMA(qx, gl, a.t);
    a.t = F2_FMA(qy, make_float2(-gl.y, gl.x), a.t);
    a.t = F2_FMA(make_float2(ql.x, ql.x), gh, a.t);
    a.t = F2_FMA(make_float2(ql.y, ql.y), gr, a.t);
}
// merge b into a (both accumulators)
DF_HD void dfacc_add(dfacc& a, const dfacc& b) {
    float s, err;
    two_sum(a.s.x, b.s.x, s, err);
    a.s.x = s;
    a.t.x = DF_ADD(a.t.x, DF_ADD(err, b.t.x));
    two_sum(a.s.y, b.s.y, s, err);
    a.s.y = s;
    a.t.y = DF_ADD(a.t.y, DF_ADD(err, b.t.y));
}
DF_HD double2 dfacc_value(const dfacc& a) {
    return make_double2((double)a.s.x + (double)a.t.x, (double)a.s.y + (double)a.t.y);
}

// ---- complex df values (Newton sign): hi + lo, each a complex FP32 -------
DF_HD dfc dfc_make(float2 hi, float2 lo) {
    dfc r;
    r.hi = hi;
    r.lo = lo;
    return r;
}
DF_HD float4 dfc_pack(const dfc& a) { return make_float4(a.hi.x, a.hi.y, a.lo.x, a.lo.y); }
DF_HD dfc dfc_unpack(float4 v) { return dfc_make(make_float2(v.x, v.y), make_float2(v.z, v.w)); }
// renormalise a real df pair (s, t) so that |t| <= ulp(s)/2
DF_HD void df_norm(float& s, float& t) {
    float a, b;
    fast_two_sum(s, t, a, b);
    s = a;
    t = b;
}
// c - a * b  (all complex df), error about 2^-46 relative to |a||b| + |c|
DF_HD dfc dfc_fms(const dfc& c, const dfc& a, const dfc& b) {
    float p, e, s, err;
    dfc r;
    // real: c.re - (a.re b.re - a.im b.im)
    float sr = c.hi.x, tr = c.lo.x;
    two_prod(a.hi.x, b.hi.x, p, e);
    two_sum(sr, -p, s, err);
    sr = s;
    tr = DF_ADD(tr, DF_SUB(err, e));
    two_prod(a.hi.y, b.hi.y, p, e);
    two_sum(sr, p, s, err);
    sr = s;
    tr = DF_ADD(tr, DF_ADD(err, e));
    tr = fmaf(-a.hi.x, b.lo.x, tr);
    tr = fmaf(-a.lo.x, b.hi.x, tr);
    tr = fmaf(a.hi.y, b.lo.y, tr);
    tr = fmaf(a.lo.y, b.hi.y, tr);
    df_norm(sr, tr);
    // imag: c.im - (a.re b.im + a.im b.re)
    float si = c.hi.y, ti = c.lo.y;
    two_prod(a.hi.x, b.hi.y, p, e);
    two_sum(si, -p, s, err);
    si = s;
    ti = DF_ADD(ti, DF_SUB(err, e));
    two_prod(a.hi.y, b.hi.x, p, e);
    two_sum(si, -p, s, err);
    si = s;
    ti = DF_ADD(ti, DF_SUB(err, e));
    ti = fmaf(-a.hi.x, b.lo.y, ti);
    ti = fmaf(-a.lo.x, b.hi.y, ti);
    ti = fmaf(-a.hi.y, b.lo.x, ti);
    ti = fmaf(-a.lo.y, b.hi.x, ti);
    df_norm(si, ti);
    r.hi = make_float2(sr, si);
    r.lo = make_float2(tr, ti);
    return r;
}
DF_HD dfc dfc_zero() { return dfc_make(make_float2(0.f, 0.f), make_float2(0.f, 0.f)); }
DF_HD dfc dfc_mul(const dfc& a, const dfc& b) { return dfc_fms(dfc_zero(), dfc_make(make_float2(-a.hi.x, -a.hi.y), make_float2(-a.lo.x, -a.lo.y)), b); }
// s * a + t * b for real FP64 scalars s, t (via FP64 on the two parts: used once per element per iteration)
DF_HD dfc dfc_axpby(double s, const dfc& a, double t, const dfc& b) {
    double2 x = dfc_to(a), y = dfc_to(b);
    return dfc_from(make_double2(s * x.x + t * y.x, s * x.y + t * y.y));
}

// 1 / z for a complex df value: conj(z) * (1 / |z|^2), the real reciprocal
// refined by one Newton step in df (error about 2^-46 relative)
DF_HD dfc dfc_inv(const dfc& z) {
    float p1, e1, p2, e2, s, e;
    two_prod(z.hi.x, z.hi.x, p1, e1);
    two_prod(z.hi.y, z.hi.y, p2, e2);
    two_sum(p1, p2, s, e);
    float t = DF_ADD(DF_ADD(e, e1), e2);
    t = fmaf(2.f * z.hi.x, z.lo.x, t);
    t = fmaf(2.f * z.hi.y, z.lo.y, t);
    df_norm(s, t);  // |z|^2 = s + t
    const float r0 = DF_DIV(1.f, s);
    float pr, pe;
    two_prod(s, r0, pr, pe);
    // residual 1 - (s + t) r0; 1 - pr is exact (pr is within an ulp of 1)
    const float res = DF_SUB(DF_SUB(DF_SUB(1.f, pr), pe), DF_MUL(t, r0));
    float rh, rl;
    fast_two_sum(r0, DF_MUL(r0, res), rh, rl);
    const dfc zc = dfc_make(make_float2(z.hi.x, -z.hi.y), make_float2(z.lo.x, -z.lo.y));
    return dfc_mul(zc, dfc_make(make_float2(rh, 0.f), make_float2(rl, 0.f)));
}
