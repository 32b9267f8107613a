// Host build of the double-float accumulation of paper_0710_0341_gb300/csrc/
// df.cuh (pass B, the projections, the recombination and the Newton-Schulz
// products accumulate with it), so that the CPU tests can hold it to exact
// arithmetic. No GPU and no CUDA runtime call is involved.
#include "../../paper_0710_0341_gb300/csrc/df.cuh"

// out = sum_k q_k g_k (complex; q = qh + ql, g = gh + gl as interleaved re, im)
extern "C" void host_dfacc_dot(const float* qh, const float* ql, const float* gh, const float* gl, int n,
                               double* out) {
    dfacc a;
    dfacc_zero(a);
    for (int k = 0; k < n; k++)
        dfacc_mac(a, make_float2(qh[2 * k], qh[2 * k + 1]), make_float2(ql[2 * k], ql[2 * k + 1]),
                  make_float2(gh[2 * k], gh[2 * k + 1]), make_float2(gl[2 * k], gl[2 * k + 1]));
    const double2 v = dfacc_value(a);
    out[0] = v.x;
    out[1] = v.y;
}

// out = c - a b for complex df values given as (re_hi, im_hi, re_lo, im_lo)
extern "C" void host_dfc_fms(const float* c, const float* a, const float* b, float* out) {
    const dfc r = dfc_fms(dfc_unpack(make_float4(c[0], c[1], c[2], c[3])), dfc_unpack(make_float4(a[0], a[1], a[2], a[3])),
                          dfc_unpack(make_float4(b[0], b[1], b[2], b[3])));
    const float4 p = dfc_pack(r);
    out[0] = p.x;
    out[1] = p.y;
    out[2] = p.z;
    out[3] = p.w;
}

// split an FP64 value into hi + lo FP32
extern "C" void host_split_d(const double* x, float* out, int n) {
    for (int i = 0; i < n; i++) {
        const float2 s = split_d(x[i]);
        out[2 * i] = s.x;
        out[2 * i + 1] = s.y;
    }
}

// out = 1 / z for a complex df value (re_hi, im_hi, re_lo, im_lo): the pivot
// reciprocal of the Gauss-Jordan Newton kernels
extern "C" void host_dfc_inv(const float* z, float* out) {
    const float4 p = dfc_pack(dfc_inv(dfc_unpack(make_float4(z[0], z[1], z[2], z[3]))));
    out[0] = p.x;
    out[1] = p.y;
    out[2] = p.z;
    out[3] = p.w;
}
