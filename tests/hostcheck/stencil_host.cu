// Host build of the stencil's site arithmetic (paper_0710_0341_gb300/csrc/
// dslash_site.cuh and dd.cuh), so that the CPU tests can check it against the
// oracle: the same templates the kernels instantiate, run over all sites on
// the host. No GPU and no CUDA runtime call is involved.
#include <math.h>

#include "../../paper_0710_0341_gb300/csrc/dd.cuh"
#include "../../paper_0710_0341_gb300/csrc/dslash_site.cuh"

using namespace ovl_stencil;

template <typename T, typename VT, int LINKS>
static void apply(const KArgs& a, const void* in, void* out, double mu) {
    const T wp = (T)exp(mu), wm = (T)exp(-mu);
    for (size_t s = 0; s < a.V; s++) site_compute<T, VT, LINKS>(a, (const VT*)in, (VT*)out, s, wp, wm);
}

// mode 0: FP64 spinors and links, FP64 arithmetic; 1: the same data, double-float
// arithmetic; 2: FP32 spinors, 18-real FP32 links; 3: FP32 spinors, 12-real links.
// links_a / links_b in the device layouts (links_b: the ninth entries, mode 2 only).
extern "C" int host_apply_hw(const int* dims, int apbc, double mu, double kappa, int mode, const void* links_a,
                             const void* links_b, const void* in, void* out) {
    KArgs a;
    memset(&a, 0, sizeof a);
    a.Lx = dims[0];
    a.Ly = dims[1];
    a.Lz = dims[2];
    a.Lt = dims[3];
    a.V = (size_t)dims[0] * dims[1] * dims[2] * dims[3];
    a.kappa = kappa;
    a.apbc = apbc;
    switch (mode) {
        case 0:
            a.u64 = (const double2*)links_a;
            apply<double, double2, OVL_LINKS_F64>(a, in, out, mu);
            return 0;
        case 1:
            a.u64 = (const double2*)links_a;
            apply<dd, double2, OVL_LINKS_F64>(a, in, out, mu);
            return 0;
        case 2:
            a.u32q = (const float4*)links_a;
            a.u32r = (const float2*)links_b;
            apply<float, float2, OVL_LINKS_F32>(a, in, out, mu);
            return 0;
        case 3:
            a.u12 = (const float4*)links_a;
            apply<float, float2, OVL_LINKS_R12>(a, in, out, mu);
            return 0;
        default:
            return 1;
    }
}

// dd conversions and operations on n values: out = [double(dd(x)), a+b, a-b, a*b, a*b+c] per element
extern "C" void host_dd_ops(const double* x, const double* a, const double* b, const double* c, double* out, int n) {
    for (int i = 0; i < n; i++) {
        const dd X(x[i]), A(a[i]), B(b[i]), Cc(c[i]);
        out[5 * i + 0] = (double)X;
        out[5 * i + 1] = (double)(A + B);
        out[5 * i + 2] = (double)(A - B);
        out[5 * i + 3] = (double)(A * B);
        out[5 * i + 4] = (double)ffma(A, B, Cc);
    }
}
