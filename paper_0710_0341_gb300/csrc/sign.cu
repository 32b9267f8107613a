// Deflation data and the batched sign-function driver (Secs. 2-4).
//
// ovl_sign_apply runs, for every solve of a batch, on the device:
//   deflation projection  Schur: x_perp = (1 - S S^dag) b (twice)      (Sec. 3)
//                         LR:    g = L^dag b, x_minus = b - R g        (Eq. 21)
//   start vector          beta = |x|, v_1 = x / beta                   (Eq. 7)
//   k Arnoldi steps       stencil + two Gram-Schmidt passes per step   (Eqs. 7, 14)
//   small sign            F = sgn(H) by scaled Newton                  (Eqs. 11, 16-17, 22)
//   recombination         Schur: y = (S V_k) F (S^dag b; beta e_1)     (Eq. 16 = Eq. 19)
//                         LR:    y = R sgn(Lambda) g + beta V_k F e_1  (Eq. 22)
// The host only sizes buffers, launches kernels and reads back three small
// arrays (the projection coefficients, the solve descriptors and the
// Newton status); every arithmetic step runs in the kernels of this library.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <utility>

#include "df.cuh"
#include "krylov.cuh"
#include "newton.cuh"
#include "sylvester.cuh"

// Newton-Schulz takes over from the scaled Newton iteration once a step is
// below NS_SWITCH (relative, Frobenius); at most NS_MAX_ITER products steps
static constexpr double NS_SWITCH = 3e-2;  // measured: 1e-2 one more Newton step, 1e-1 worse
static constexpr int NS_MAX_ITER = 40;

namespace {

__global__ void k_split_planes(const double2* __restrict__ x, float2* __restrict__ hi, float2* __restrict__ lo,
                               size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        double2 v = x[i];
        float2 a = split_d(v.x), b = split_d(v.y);
        hi[i] = make_float2(a.x, b.x);
        lo[i] = make_float2(a.y, b.y);
    }
}

__global__ void k_join_planes(const float2* __restrict__ hi, const float2* __restrict__ lo, double2* __restrict__ x,
                              size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        float2 a = hi[i], b = lo[i];
        x[i] = make_double2((double)a.x + (double)b.x, (double)a.y + (double)b.y);
    }
}

__global__ void k_h_to_h32(const double2* __restrict__ H, float2* __restrict__ H32, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        H32[i] = make_float2((float)H[i].x, (float)H[i].y);
}

struct Carve {
    char* base;
    size_t off = 0;
    template <class T>
    T* take(size_t n) {
        off = (off + 255) & ~(size_t)255;
        T* p = (T*)(base + off);
        off += n * sizeof(T);
        return p;
    }
};

unsigned grid_for(size_t n, int sms) {
    size_t b = (n + 255) / 256;
    size_t cap = (size_t)sms * 8;
    return (unsigned)std::max<size_t>(1, std::min(b, cap));
}

}  // namespace

// ---------------------------------------------------------------------------
// deflation data
// ---------------------------------------------------------------------------
static int upload_vectors(ovl_lattice lat, const double* canon, int m, float2** hi, float2** lo, double2** f64) {
    size_t N = lat->N;
    size_t vb = N * sizeof(double2) * (size_t)m;
    if (cudaMalloc(hi, N * sizeof(float2) * m) != cudaSuccess || cudaMalloc(lo, N * sizeof(float2) * m) != cudaSuccess) {
        cudaGetLastError();
        return ovl_fail(lat, OVL_ENOMEM, "deflation vectors: allocation failed");
    }
    // canonical (host or device) -> packed FP64 (scratch) -> hi/lo planes
    void* s;
    if (int rc = ovl_scratch(lat, 2 * vb, &s)) return rc;
    const double* src = canon;
    if (!ovl_is_device_ptr(canon)) {
        OVL_CUDA_TRY(lat, cudaMemcpyAsync(s, canon, vb, cudaMemcpyHostToDevice, lat->stream));
        src = (const double*)s;
    }
    double2* packed = (double2*)((char*)s + vb);
    if (int rc = ovl_pack_impl(lat, src, packed, m, OVL_VEC_F64, lat->stream)) return rc;
    k_split_planes<<<grid_for(N * m, lat->num_sms), 256, 0, lat->stream>>>(packed, *hi, *lo, N * m);
    OVL_LAUNCH_CHECK(lat);
    if (cudaMalloc(f64, vb) != cudaSuccess) {
        cudaGetLastError();
        return ovl_fail(lat, OVL_ENOMEM, "deflation vectors: allocation failed");
    }
    OVL_CUDA_TRY(lat, cudaMemcpyAsync(*f64, packed, vb, cudaMemcpyDeviceToDevice, lat->stream));
    OVL_CUDA_TRY(lat, cudaStreamSynchronize(lat->stream));
    return OVL_OK;
}

// complex128 copies of the deflation vectors for the plain FP64 form, joined
// from the hi + lo planes when the object has none yet (computed or adjoint data)
static int defl_fp64(ovl_lattice lat, ovl_deflation d) {
    const size_t N = lat->N, n = N * (size_t)d->m;
    for (int which = 0; which < 2; which++) {
        double2** dst = which ? &d->L64 : &d->S64;
        const float2* hi = which ? d->L_hi : d->S_hi;
        const float2* lo = which ? d->L_lo : d->S_lo;
        if (*dst || !hi) continue;
        if (cudaMalloc(dst, n * sizeof(double2)) != cudaSuccess) {
            cudaGetLastError();
            return ovl_fail(lat, OVL_ENOMEM, "deflation vectors: FP64 copy does not fit");
        }
        k_join_planes<<<grid_for(n, lat->num_sms), 256, 0, lat->stream>>>(hi, lo, *dst, n);
        OVL_LAUNCH_CHECK(lat);
    }
    return OVL_OK;
}

extern "C" int ovl_destroy_deflation(ovl_deflation d) {
    if (!d) return OVL_OK;
    if (d->lat) cudaStreamSynchronize(d->lat->stream);
    cudaFree(d->S_hi);
    cudaFree(d->S_lo);
    cudaFree(d->L_hi);
    cudaFree(d->L_lo);
    cudaFree(d->S64);
    cudaFree(d->L64);
    cudaFree(d->T);
    delete d;
    return OVL_OK;
}

extern "C" int ovl_set_deflation(ovl_lattice lat, double mu, double m_w, int scheme, int m, const double* S_or_R,
                                 const double* T, const double* L, ovl_deflation* out) {
    if (!lat || !out || !S_or_R || !T) return ovl_fail(lat, OVL_EINVAL, "ovl_set_deflation: null argument");
    if (scheme != OVL_DEFL_SCHUR && scheme != OVL_DEFL_LR)
        return ovl_fail(lat, OVL_EINVAL, "ovl_set_deflation: scheme %d is not Schur or LR", scheme);
    if (m < 1 || (size_t)m >= lat->N || m > 200) return ovl_fail(lat, OVL_EINVAL, "ovl_set_deflation: m=%d (1..200)", m);
    if (scheme == OVL_DEFL_LR && !L) return ovl_fail(lat, OVL_EINVAL, "ovl_set_deflation: LR needs L");
    if (scheme == OVL_DEFL_SCHUR && L) return ovl_fail(lat, OVL_EINVAL, "ovl_set_deflation: Schur takes no L");
    ovl_deflation d = new ovl_deflation_s();
    d->lat = lat;
    d->scheme = scheme;
    d->m = m;
    d->mu = mu;
    d->m_w = m_w;
    int rc = upload_vectors(lat, S_or_R, m, &d->S_hi, &d->S_lo, &d->S64);
    if (!rc && scheme == OVL_DEFL_LR) rc = upload_vectors(lat, L, m, &d->L_hi, &d->L_lo, &d->L64);
    if (rc) {
        ovl_destroy_deflation(d);
        return rc;
    }
    size_t tn = scheme == OVL_DEFL_SCHUR ? (size_t)m * m : (size_t)m;
    d->T_host.resize(2 * tn);
    if (ovl_is_device_ptr(T)) {
        if (cudaMemcpy(d->T_host.data(), T, tn * sizeof(double2), cudaMemcpyDeviceToHost) != cudaSuccess) {
            ovl_destroy_deflation(d);
            return ovl_fail(lat, OVL_ECUDA, "ovl_set_deflation: copying T failed");
        }
    } else {
        memcpy(d->T_host.data(), T, tn * sizeof(double2));
    }
    for (double v : d->T_host)
        if (!(v == v)) {
            ovl_destroy_deflation(d);
            return ovl_fail(lat, OVL_EINVAL, "ovl_set_deflation: T/Lambda has NaN");
        }
    if (cudaMalloc(&d->T, tn * sizeof(double2)) != cudaSuccess ||
        cudaMemcpy(d->T, d->T_host.data(), tn * sizeof(double2), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        ovl_destroy_deflation(d);
        return ovl_fail(lat, OVL_ENOMEM, "ovl_set_deflation: T allocation failed");
    }
    *out = d;
    return OVL_OK;
}

// packed vectors -> canonical (host or device); from the exact complex128
// copy when the object has one, else from the hi + lo planes (48-bit)
static int download_vectors(ovl_lattice lat, const float2* hi, const float2* lo, const double2* f64, int m,
                            double* canon) {
    size_t N = lat->N;
    size_t vb = N * sizeof(double2) * (size_t)m;
    void* s;
    if (int rc = ovl_scratch(lat, 2 * vb, &s)) return rc;
    double2* packed = (double2*)s;
    double2* cdev = (double2*)((char*)s + vb);
    if (f64) {
        OVL_CUDA_TRY(lat, cudaMemcpyAsync(packed, f64, vb, cudaMemcpyDeviceToDevice, lat->stream));
    } else {
        k_join_planes<<<grid_for(N * m, lat->num_sms), 256, 0, lat->stream>>>(hi, lo, packed, N * m);
        OVL_LAUNCH_CHECK(lat);
    }
    bool dev = ovl_is_device_ptr(canon);
    if (int rc = ovl_unpack_impl(lat, packed, dev ? canon : (double*)cdev, m, OVL_VEC_F64, lat->stream)) return rc;
    if (!dev) OVL_CUDA_TRY(lat, cudaMemcpyAsync(canon, cdev, vb, cudaMemcpyDeviceToHost, lat->stream));
    OVL_CUDA_TRY(lat, cudaStreamSynchronize(lat->stream));
    return OVL_OK;
}

extern "C" int ovl_get_deflation(ovl_deflation d, int* scheme, int* m, double* S_or_R, double* T, double* L) {
    if (!d) return ovl_fail(nullptr, OVL_EINVAL, "ovl_get_deflation: null handle");
    ovl_lattice lat = d->lat;
    if (scheme) *scheme = d->scheme;
    if (m) *m = d->m;
    if (S_or_R)
        if (int rc = download_vectors(lat, d->S_hi, d->S_lo, d->S64, d->m, S_or_R)) return rc;
    if (L && d->scheme == OVL_DEFL_LR)
        if (int rc = download_vectors(lat, d->L_hi, d->L_lo, d->L64, d->m, L)) return rc;
    if (T) {
        size_t tb = d->T_host.size() * sizeof(double);
        if (ovl_is_device_ptr(T))
            OVL_CUDA_TRY(lat, cudaMemcpy(T, d->T_host.data(), tb, cudaMemcpyHostToDevice));
        else
            memcpy(T, d->T_host.data(), tb);
    }
    return OVL_OK;
}

// ---------------------------------------------------------------------------
// the sign function
// ---------------------------------------------------------------------------
namespace {

struct SolvePlan {
    int m_q = 0, m_defl = 0, scheme = OVL_DEFL_NONE, k = 0, ldH = 0, nmax = 0;
    int adapt = 0, k_first = 0;   // adaptive depth: check interval and first check
    double tol = 1e-8, err_est = 0.0;
    std::vector<double2> g_prev;  // coefficients at the previous check
    double2 *H_est = nullptr, *g_est = nullptr;
    float2* H32_est = nullptr;
    ovl_deflation d = nullptr;
    // device pieces
    float2 *Vhi = nullptr, *Vlo = nullptr;
    double2 *u = nullptr, *w = nullptr, *H = nullptr;
    float2* H32 = nullptr;
    double2 *dots = nullptr, *dvec = nullptr;
    float2 *ap = nullptr, *gh = nullptr, *gl = nullptr;
    double* scal = nullptr;
    double2 *ap64 = nullptr, *g64 = nullptr;
    // Sylvester route (Schur, Eqs. 18-19): sgn(H_k) copy, R, Y, work, sgn(T) S^dag b
    double2 *syFH = nullptr, *syR = nullptr, *syY = nullptr, *syW = nullptr, *syr = nullptr, *sygT = nullptr;
    const float2** qhi = nullptr;
    const float2** qlo = nullptr;
    double2 *X = nullptr, *W = nullptr, *Yns = nullptr;
    double* nsacc = nullptr;
    int* handoff = nullptr;
    float4* crow = nullptr;
    double *cand_val = nullptr, *red = nullptr;
    int* cand_row = nullptr;
    unsigned* bar = nullptr;
    int *nstat = nullptr, *iters = nullptr;
    double2 *cvec = nullptr, *gcomb = nullptr;
    double2 *pout1 = nullptr, *pout2 = nullptr, *pout3 = nullptr;
    const float2 **pc_hi = nullptr, **pc_lo = nullptr;   // projection columns (dot)
    const float2 **pu_hi = nullptr, **pu_lo = nullptr;   // projection columns (update)
    const float2 **gc_hi = nullptr, **gc_lo = nullptr;   // recombination columns
};

}  // namespace

// size_only != null: validate and return the workspace bytes the batch needs
static int sign_apply_impl(ovl_lattice lat, int nsolve, const ovl_sign_params* params, const ovl_deflation* defl,
                           const double* b, double* y, ovl_sign_info* info, size_t* size_only) {
    if (!lat || nsolve < 1 || !params || (!size_only && (!b || !y)))
        return ovl_fail(lat, OVL_EINVAL, "ovl_sign_apply: bad argument");
    if (!lat->have_links) return ovl_fail(lat, OVL_EINVAL, "ovl_sign_apply: links not set");
    if (nsolve > 4096) return ovl_fail(lat, OVL_EINVAL, "ovl_sign_apply: nsolve=%d too large", nsolve);
    const size_t N = lat->N;
    const int prec = params[0].prec;
    const double m_w = params[0].m_w;
    if (prec < OVL_PREC_FP64 || prec > OVL_PREC_DF40)
        return ovl_fail(lat, OVL_EINVAL, "ovl_sign_apply: precision %d unknown", prec);
    const bool lo16 = prec == OVL_PREC_DF40;  // BF16 low planes of the Krylov columns
    const bool df = prec == OVL_PREC_FP64 || prec == OVL_PREC_FP64_DFSTENCIL || lo16;  // hi + lo basis
    const bool f64 = prec == OVL_PREC_FP64_PLAIN;                              // complex128 basis
    // the plain FP64 form takes the FP64 Gauss-Jordan Newton whatever newton_fp64 says
    const int nmode = f64 ? 1 : params[0].newton_fp64;
    const bool syl = params[0].schur_route == 1;  // Schur solves by Eqs. 18-19
    std::vector<SolvePlan> P(nsolve);
    int kmax = 0, ldmax = 0, mdef_max = 0;
    for (int i = 0; i < nsolve; i++) {
        const ovl_sign_params& q = params[i];
        if (q.prec != prec) return ovl_fail(lat, OVL_EINVAL, "ovl_sign_apply: mixed precisions in one batch");
        if (q.m_w != m_w) return ovl_fail(lat, OVL_EINVAL, "ovl_sign_apply: one m_w per batch");
        if (q.schur_route != params[0].schur_route || q.schur_route < 0 || q.schur_route > 1)
            return ovl_fail(lat, OVL_EINVAL, "ovl_sign_apply: solve %d: schur_route=%d (0 or 1, one per batch)", i,
                            q.schur_route);
        if (q.newton_fp64 != params[0].newton_fp64 || q.newton_fp64 < 0 || q.newton_fp64 > 4)
            return ovl_fail(lat, OVL_EINVAL, "ovl_sign_apply: solve %d: newton_fp64=%d (0..4, one per batch)", i,
                            q.newton_fp64);
        if (!(q.m_w > -4.0 + 1e-12) || !(q.mu == q.mu) || fabs(q.mu) > 50.0)
            return ovl_fail(lat, OVL_EINVAL, "ovl_sign_apply: solve %d: bad mu/m_w", i);
        if (q.k < 1) return ovl_fail(lat, OVL_EINVAL, "ovl_sign_apply: solve %d: k=%d < 1", i, q.k);
        if (q.adapt_every < 0 || (q.adapt_every > 0 && q.k_max < q.k))
            return ovl_fail(lat, OVL_EINVAL, "ovl_sign_apply: solve %d: adaptive needs k_max >= k", i);
        SolvePlan& p = P[i];
        p.k = q.adapt_every > 0 ? q.k_max : q.k;
        p.adapt = q.adapt_every;
        p.k_first = q.k;
        p.tol = q.tol > 0 ? q.tol : 1e-8;
        if (defl && defl[i]) {
            ovl_deflation d = defl[i];
            if (d->lat != lat) return ovl_fail(lat, OVL_EINVAL, "solve %d: deflation of another lattice", i);
            if (fabs(d->mu - q.mu) > 1e-12 || fabs(d->m_w - q.m_w) > 1e-12)
                return ovl_fail(lat, OVL_EINVAL, "solve %d: deflation built for mu=%g m_w=%g, solve has mu=%g m_w=%g", i,
                                d->mu, d->m_w, q.mu, q.m_w);
            p.d = d;
            p.scheme = d->scheme;
            p.m_defl = d->m;
            p.m_q = d->scheme == OVL_DEFL_SCHUR ? d->m : 0;
        }
        p.ldH = p.m_q + p.k + 1;
        p.nmax = p.m_q + p.k;
        if (p.ldH > OVL_MAXCOL || p.nmax > OVL_NEWTON_MAXN)
            return ovl_fail(lat, OVL_EINVAL, "solve %d: m+k+1=%d exceeds the build limit %d", i, p.ldH, OVL_MAXCOL);
        if ((size_t)p.k > N) return ovl_fail(lat, OVL_EINVAL, "solve %d: k=%d exceeds N", i, p.k);
        kmax = std::max(kmax, p.k);
        ldmax = std::max(ldmax, p.ldH);
        mdef_max = std::max(mdef_max, p.m_defl);
    }
    const int G = ovl_gs_grid(lat);
    const int pstride = std::max(2 * ldmax + 3, mdef_max + 1);
    // ---- sizes and one allocation ----
    auto plan_bytes = [&](bool carve, char* base) -> size_t {
        Carve c{base};
        for (int i = 0; i < nsolve; i++) {
            SolvePlan& p = P[i];
            size_t ld = p.ldH, nm = p.nmax, md = std::max(1, p.m_defl);
            auto t = [&](auto*& ptr, size_t n) {
                using T = std::remove_reference_t<decltype(*ptr)>;
                T* q = c.take<std::remove_const_t<T>>(n);
                if (carve) ptr = q;
            };
            t(p.Vhi, N * (p.k + 1) * (f64 ? 2 : 1));  // complex128 columns take two float2 slots
            if (df) t(p.Vlo, lo16 ? (N * (p.k + 1) + 1) / 2 : N * (p.k + 1));  // BF16 pairs: 4 bytes per entry
            t(p.u, N);
            t(p.w, N);
            t(p.H, ld * ld);
            t(p.H32, ld * ld);
            t(p.dots, 2 * ld + 3);
            t(p.dvec, ld + 1);
            t(p.ap, ld);
            t(p.gh, ld);
            t(p.gl, ld);
            t(p.scal, 8);
            if (f64) {
                t(p.ap64, ld);
                t(p.g64, ld);
            }
            if (syl && p.m_q) {
                const size_t kk = (size_t)p.k, mm = (size_t)p.m_q;
                t(p.syFH, kk * kk);
                t(p.syR, mm * kk);
                t(p.syY, mm * kk);
                t(p.syW, kk * kk);
                t(p.syr, kk);
                t(p.sygT, mm);
            }
            t(p.qhi, ld);
            t(p.qlo, ld);
            t(p.X, nm * nm);
            t(p.W, nm * nm + 64 * nm);
            t(p.Yns, nm * nm);
            t(p.nsacc, OVL_NS_ACC);
            t(p.handoff, 1);
            t(p.crow, 2 * 64 * nm);
            t(p.cand_val, 128);
            t(p.cand_row, 128);
            t(p.red, 128);
            t(p.bar, 1);
            t(p.nstat, 1);
            t(p.iters, 1);
            t(p.cvec, nm + md);
            t(p.gcomb, nm + md);
            t(p.pout1, md + 1);
            t(p.pout2, md + 1);
            t(p.pout3, md + 1);
            t(p.pc_hi, md);
            t(p.pc_lo, md);
            t(p.pu_hi, md);
            t(p.pu_lo, md);
            t(p.gc_hi, nm + md);
            t(p.gc_lo, nm + md);
            if (p.adapt) {
                t(p.H_est, ld * ld);
                t(p.H32_est, ld * ld);
                t(p.g_est, nm + md);
            }
        }
        c.take<char>(0);
        return c.off;
    };
    size_t per = plan_bytes(false, nullptr);
    // batch-wide pieces after the per-solve ones: one routine sizes and carves
    struct BatchPtrs {
        SolveDev *sd = nullptr, *sd_est = nullptr;
        NewtonDev* nd = nullptr;
        NsDev* ns = nullptr;
        SylDev* sy = nullptr;
        ProjDev* pd = nullptr;
        GemvDev* gd = nullptr;
        double2* part = nullptr;
        double* mu = nullptr;
        void** ptrs = nullptr;
        double2* canon = nullptr;  // canonical staging for host b / y
    };
    auto carve_batch = [&](char* at) -> std::pair<BatchPtrs, size_t> {
        Carve cb{at};
        cb.off = per;
        BatchPtrs q;
        q.sd = cb.take<SolveDev>(nsolve);
        q.sd_est = cb.take<SolveDev>(nsolve);
        q.nd = cb.take<NewtonDev>(nsolve);
        q.ns = cb.take<NsDev>(nsolve);
        q.sy = cb.take<SylDev>(nsolve);
        q.pd = cb.take<ProjDev>(nsolve);
        q.gd = cb.take<GemvDev>(nsolve);
        q.part = cb.take<double2>((size_t)nsolve * G * pstride);
        q.mu = cb.take<double>(nsolve);
        q.ptrs = cb.take<void*>(2 * (size_t)nsolve);
        q.canon = cb.take<double2>(N * nsolve);
        cb.take<char>(0);
        return {q, cb.off};
    };
    const size_t batch_off = carve_batch(nullptr).second;
    if (size_only) {
        *size_only = batch_off;
        return OVL_OK;
    }
    if (batch_off > lat->ws_bytes) {
        cudaStreamSynchronize(lat->stream);
        if (lat->graph_exec) {  // its kernels point into the old workspace
            cudaGraphExecDestroy(lat->graph_exec);
            lat->graph_exec = nullptr;
            lat->graph_key = lat->graph_seen = 0;
        }
        cudaFree(lat->ws);
        lat->ws = nullptr;
        lat->ws_bytes = 0;
        if (cudaMalloc(&lat->ws, batch_off) != cudaSuccess) {
            cudaGetLastError();
            return ovl_fail(lat, OVL_ENOMEM, "ovl_sign_apply: workspace of %.3f GB does not fit", batch_off / 1e9);
        }
        lat->ws_bytes = batch_off;
    }
    char* base = (char*)lat->ws;
    plan_bytes(true, base);
    const BatchPtrs bp = carve_batch(base).first;
    SolveDev* d_sd = bp.sd;
    SolveDev* d_sd_est = bp.sd_est;
    NewtonDev* d_nd = bp.nd;
    NsDev* d_ns = bp.ns;
    ProjDev* d_pd = bp.pd;
    GemvDev* d_gd = bp.gd;
    double2* d_part = bp.part;
    double* d_mu = bp.mu;
    void** d_ptrs = bp.ptrs;
    double2* d_canon = bp.canon;
    cudaStream_t st = lat->stream;

    // ---- inputs ----
    const double* bsrc = b;
    if (!ovl_is_device_ptr(b)) {
        OVL_CUDA_TRY(lat, cudaMemcpyAsync(d_canon, b, N * sizeof(double2) * nsolve, cudaMemcpyHostToDevice, st));
        bsrc = (const double*)d_canon;
    }
    for (int i = 0; i < nsolve; i++)
        if (int rc = ovl_pack_impl(lat, bsrc + 2 * N * i, P[i].u, 1, OVL_VEC_F64, st)) return rc;

    if (f64)
        for (int i = 0; i < nsolve; i++)
            if (P[i].d)
                if (int rc = defl_fp64(lat, P[i].d)) return rc;

    // ---- column pointers, descriptors ----
    std::vector<SolveDev> hs(nsolve);
    std::vector<const float2*> tmp_hi, tmp_lo;
    for (int i = 0; i < nsolve; i++) {
        SolvePlan& p = P[i];
        tmp_hi.assign(p.ldH, nullptr);
        tmp_lo.assign(p.ldH, nullptr);
        for (int cidx = 0; cidx < p.m_q; cidx++) {
            tmp_hi[cidx] = f64 ? (const float2*)(p.d->S64 + N * cidx) : p.d->S_hi + N * cidx;
            tmp_lo[cidx] = f64 ? nullptr : p.d->S_lo + N * cidx;
        }
        for (int cidx = p.m_q; cidx < p.ldH; cidx++) {
            tmp_hi[cidx] = f64 ? (const float2*)((double2*)p.Vhi + N * (cidx - p.m_q)) : p.Vhi + N * (cidx - p.m_q);
            tmp_lo[cidx] = !df ? nullptr
                           : lo16 ? (const float2*)((const char*)p.Vlo + (size_t)4 * N * (cidx - p.m_q))
                                  : p.Vlo + N * (cidx - p.m_q);
        }
        OVL_CUDA_TRY(lat, cudaMemcpyAsync(p.qhi, tmp_hi.data(), p.ldH * sizeof(void*), cudaMemcpyHostToDevice, st));
        OVL_CUDA_TRY(lat, cudaMemcpyAsync(p.qlo, tmp_lo.data(), p.ldH * sizeof(void*), cudaMemcpyHostToDevice, st));
        OVL_CUDA_TRY(lat, cudaStreamSynchronize(st));  // tmp vectors are reused
        SolveDev& s = hs[i];
        s.qhi = p.qhi;
        s.qlo = df ? p.qlo : nullptr;
        s.vhi = p.Vhi;
        s.vlo = df ? p.Vlo : nullptr;
        s.nptr = p.m_q;
        s.u = p.u;
        s.w = p.w;
        s.H = p.H;
        s.H32 = p.H32;
        s.dots = p.dots;
        s.dvec = p.dvec;
        s.ap = p.ap;
        s.gh = p.gh;
        s.gl = p.gl;
        s.scal = p.scal;
        s.ap64 = f64 ? p.ap64 : nullptr;
        s.g64 = f64 ? p.g64 : nullptr;
        s.m_q = p.m_q;
        s.k = p.k;
        s.ldH = p.ldH;
        s.active = 1;
        s.k_used = p.k;
        s.status = 0;
        s.fin = 1;
        OVL_CUDA_TRY(lat, cudaMemsetAsync(p.H, 0, (size_t)p.ldH * p.ldH * sizeof(double2), st));
        if (p.m_q)
            OVL_CUDA_TRY(lat, cudaMemcpy2DAsync(p.H, p.ldH * sizeof(double2), p.d->T, p.m_q * sizeof(double2),
                                                p.m_q * sizeof(double2), p.m_q, cudaMemcpyDeviceToDevice, st));
        k_h_to_h32<<<grid_for((size_t)p.ldH * p.ldH, lat->num_sms), 256, 0, st>>>(p.H, p.H32,
                                                                                  (size_t)p.ldH * p.ldH);
        OVL_LAUNCH_CHECK(lat);
    }
    OVL_CUDA_TRY(lat, cudaMemcpyAsync(d_sd, hs.data(), nsolve * sizeof(SolveDev), cudaMemcpyHostToDevice, st));

    // ---- deflation projection and |x|^2 ----
    auto run_proj = [&](int which) -> int {
        // which 0: first dot (S or L), 1: second dot (Schur only), 2: norm only
        std::vector<ProjDev> pd(nsolve);
        int maxcol = 0;
        for (int i = 0; i < nsolve; i++) {
            SolvePlan& p = P[i];
            ProjDev& q = pd[i];
            q.x = p.u;
            q.ncol = (which == 2 || p.scheme == OVL_DEFL_NONE || (which == 1 && p.scheme != OVL_DEFL_SCHUR)) ? 0 : p.m_defl;
            q.out = which == 0 ? p.pout1 : which == 1 ? p.pout2 : p.pout3;
            q.qhi = p.pc_hi;
            q.qlo = f64 ? nullptr : p.pc_lo;
            q.coef = q.out;
            q.f64 = f64;
            maxcol = std::max(maxcol, q.ncol);
        }
        OVL_CUDA_TRY(lat, cudaMemcpyAsync(d_pd, pd.data(), nsolve * sizeof(ProjDev), cudaMemcpyHostToDevice, st));
        if (int rc = ovl_proj_dot(lat, d_pd, nsolve, maxcol, d_part, G, st, f64)) return rc;
        if (which == 2 || maxcol == 0) {
            OVL_CUDA_TRY(lat, cudaStreamSynchronize(st));
            return OVL_OK;
        }
        // update x -= Q coef with the update columns (S for Schur, R for LR)
        for (int i = 0; i < nsolve; i++) {
            pd[i].qhi = P[i].pu_hi;
            pd[i].qlo = f64 ? nullptr : P[i].pu_lo;
        }
        OVL_CUDA_TRY(lat, cudaMemcpyAsync(d_pd, pd.data(), nsolve * sizeof(ProjDev), cudaMemcpyHostToDevice, st));
        if (int rc = ovl_proj_update(lat, d_pd, nsolve, maxcol, st, f64)) return rc;
        OVL_CUDA_TRY(lat, cudaStreamSynchronize(st));
        return OVL_OK;
    };
    for (int i = 0; i < nsolve; i++) {
        SolvePlan& p = P[i];
        if (!p.m_defl) continue;
        std::vector<const float2*> dh(p.m_defl), dl(p.m_defl), uh(p.m_defl), ul(p.m_defl);
        for (int cidx = 0; cidx < p.m_defl; cidx++) {
            bool lr = p.scheme == OVL_DEFL_LR;
            if (f64) {
                dh[cidx] = (const float2*)((lr ? p.d->L64 : p.d->S64) + N * cidx);
                uh[cidx] = (const float2*)(p.d->S64 + N * cidx);
                dl[cidx] = ul[cidx] = nullptr;
                continue;
            }
            dh[cidx] = (lr ? p.d->L_hi : p.d->S_hi) + N * cidx;
            dl[cidx] = (lr ? p.d->L_lo : p.d->S_lo) + N * cidx;
            uh[cidx] = p.d->S_hi + N * cidx;
            ul[cidx] = p.d->S_lo + N * cidx;
        }
        OVL_CUDA_TRY(lat, cudaMemcpyAsync(p.pc_hi, dh.data(), p.m_defl * sizeof(void*), cudaMemcpyHostToDevice, st));
        OVL_CUDA_TRY(lat, cudaMemcpyAsync(p.pc_lo, dl.data(), p.m_defl * sizeof(void*), cudaMemcpyHostToDevice, st));
        OVL_CUDA_TRY(lat, cudaMemcpyAsync(p.pu_hi, uh.data(), p.m_defl * sizeof(void*), cudaMemcpyHostToDevice, st));
        OVL_CUDA_TRY(lat, cudaMemcpyAsync(p.pu_lo, ul.data(), p.m_defl * sizeof(void*), cudaMemcpyHostToDevice, st));
        OVL_CUDA_TRY(lat, cudaStreamSynchronize(st));
    }
    {
        double pb = 0.0;
        for (int i = 0; i < nsolve; i++) pb += (double)N * 16.0 * (2.0 * P[i].m_defl * (P[i].scheme == OVL_DEFL_SCHUR ? 2 : 1) + 6.0);
        ProfScope ps(lat, 6, pb, st);
        if (int rc = run_proj(0)) return rc;
        if (int rc = run_proj(1)) return rc;
        if (int rc = run_proj(2)) return rc;
        ps.end(st);
    }
    // projection coefficients back to the host (m + 1 numbers per solve)
    std::vector<std::vector<double2>> c1(nsolve), c2(nsolve), nrm(nsolve);
    std::vector<double> beta(nsolve);
    for (int i = 0; i < nsolve; i++) {
        SolvePlan& p = P[i];
        int m = p.m_defl;
        c1[i].resize(m + 1);
        c2[i].resize(m + 1);
        nrm[i].resize(1);
        if (m) OVL_CUDA_TRY(lat, cudaMemcpy(c1[i].data(), p.pout1, m * sizeof(double2), cudaMemcpyDeviceToHost));
        if (m && p.scheme == OVL_DEFL_SCHUR)
            OVL_CUDA_TRY(lat, cudaMemcpy(c2[i].data(), p.pout2, m * sizeof(double2), cudaMemcpyDeviceToHost));
        OVL_CUDA_TRY(lat, cudaMemcpy(nrm[i].data(), p.pout3, sizeof(double2), cudaMemcpyDeviceToHost));
        beta[i] = sqrt(nrm[i][0].x);
    }

    // ---- start vectors ----
    BatchDev bd = {};
    bd.sd = d_sd;
    bd.nsolve = nsolve;
    bd.N = N;
    bd.part = d_part;
    bd.G = G;
    bd.pstride = pstride;
    bd.df = df;
    bd.f64 = f64;
    bd.lo16 = lo16;
    bd.bulk16 = N % 4 == 0;  // the basis is carved at 256-byte offsets, the Schur vectors are cudaMalloc'd
    bd.pmax = 0;
    // beta^2 sits in .x of pout3[0]; pass it through a per-solve array
    {
        std::vector<double> b2(nsolve);
        for (int i = 0; i < nsolve; i++) b2[i] = nrm[i][0].x;
        OVL_CUDA_TRY(lat, cudaMemcpyAsync(d_mu, b2.data(), nsolve * sizeof(double), cudaMemcpyHostToDevice, st));
        if (int rc = ovl_start_vector(lat, bd, d_mu, 1, st)) return rc;
    }
    // ---- Arnoldi loop ----
    std::vector<double> mus(nsolve);
    std::vector<void*> ptrs(2 * nsolve);
    for (int i = 0; i < nsolve; i++) {
        mus[i] = params[i].mu;
        ptrs[i] = P[i].u;
        ptrs[nsolve + i] = P[i].w;
    }
    OVL_CUDA_TRY(lat, cudaMemcpyAsync(d_mu, mus.data(), nsolve * sizeof(double), cudaMemcpyHostToDevice, st));
    OVL_CUDA_TRY(lat, cudaMemcpyAsync(d_ptrs, ptrs.data(), 2 * nsolve * sizeof(void*), cudaMemcpyHostToDevice, st));
    DslashArgs da;
    da.in = (const void* const*)d_ptrs;
    da.out = (void* const*)(d_ptrs + nsolve);
    da.mu = d_mu;
    da.active = &d_sd[0].active;
    da.klim = &d_sd[0].k;
    da.stride = (int)(sizeof(SolveDev) / sizeof(int));
    da.nrhs = nsolve;
    da.kappa = 1.0 / (8.0 + 2.0 * m_w);
    const int links = (prec == OVL_PREC_FP64 || f64 || lo16) ? OVL_LINKS_F64
                      : prec == OVL_PREC_FP64_DFSTENCIL ? OVL_LINKS_F64DF
                      : prec == OVL_PREC_MIXED          ? OVL_LINKS_F32
                                                        : OVL_LINKS_R12;
    const double site_bytes =
        2.0 * 12 * 16 + 4.0 * ((links == OVL_LINKS_F64 || links == OVL_LINKS_F64DF) ? 144 : links == OVL_LINKS_F32 ? 72 : 48);
    const double qbytes = lo16 ? 12.0 : (df || f64) ? 16.0 : 8.0;
    bool any_adapt = false;
    for (int i = 0; i < nsolve; i++) any_adapt = any_adapt || P[i].adapt > 0;
    // accurate Galerkin correction of the last column (FP64 projection of u)
    // for the solves whose descriptor in sdev has fin set; H as in sdev
    auto final_pass = [&](SolveDev* sdev, const std::vector<int>& ncol) -> int {
        std::vector<ProjDev> pd(nsolve);
        int maxcol = 0;
        for (int i = 0; i < nsolve; i++) {
            ProjDev& q = pd[i];
            q.qhi = P[i].qhi;
            q.qlo = df ? P[i].qlo : nullptr;
            q.x = P[i].u;
            q.out = P[i].dots;
            q.coef = nullptr;
            q.ncol = ncol[i];
            q.f64 = f64;
            q.lo16_from = lo16 ? P[i].m_q : 0;  // the Krylov columns
            q.lo16_to = lo16 ? ncol[i] : 0;
            maxcol = std::max(maxcol, q.ncol);
        }
        OVL_CUDA_TRY(lat, cudaMemcpyAsync(d_pd, pd.data(), nsolve * sizeof(ProjDev), cudaMemcpyHostToDevice, st));
        BatchDev b2 = bd;
        b2.sd = sdev;
        b2.pmax = maxcol;
        double fb = 0.0;
        for (int i = 0; i < nsolve; i++) fb += (double)pd[i].ncol * N * 16.0 + N * 16.0;
        ProfScope pf(lat, 6, fb, st);
        if (int rc = ovl_gs_final(lat, b2, d_pd, maxcol, st)) return rc;
        pf.end(st);
        OVL_CUDA_TRY(lat, cudaStreamSynchronize(st));  // pd must outlive the copy
        return OVL_OK;
    };
    // scaled Newton on H[0:n, 0:n] of each solve with n[i] > 0; g = F c
    std::vector<NewtonDev> nd(nsolve);
    // cvo (optional): per-solve coefficient vectors c replacing the default
    // (S^dag b; beta e_1) or beta e_1 (used by the Sylvester route)
    auto newton = [&](const std::vector<const double2*>& Hs, const std::vector<int>& nn,
                      const std::vector<double2*>& gout,
                      const std::vector<std::vector<double2>>* cvo = nullptr) -> int {
        int nmax_run = 0, any_run = 0;
        for (int i = 0; i < nsolve; i++) {
            SolvePlan& p = P[i];
            NewtonDev& q = nd[i];
            int n = nn[i];
            q = NewtonDev();
            q.H = Hs[i];
            q.ldH = p.ldH;
            q.n = n;
            q.run = n > 0 ? 1 : 0;
            q.max_iter = params[i].newton_max_iter > 0 ? params[i].newton_max_iter : 100;
            q.tol = params[i].newton_tol > 0 ? params[i].newton_tol : 1e-13;
            q.X = p.X;
            q.W = p.W;
            q.cand_val = p.cand_val;
            q.cand_row = p.cand_row;
            q.red = p.red;
            q.bar = p.bar;
            q.status = p.nstat;
            q.iters = p.iters;
            q.cvec = p.cvec;
            q.gout = gout[i];
            q.df = nmode == 1 ? 0 : 1;
            q.crow = p.crow;
            q.Wg = (float4*)p.W;
            q.ns_switch = (nmode == 0 || nmode == 4) ? NS_SWITCH : 0.0;
            q.resume = 0;
            q.handoff = p.handoff;
            if (q.run) {
                any_run = 1;
                nmax_run = std::max(nmax_run, n);
            }
            // coefficient vector: Schur (S^dag b; beta e_1), otherwise beta e_1
            std::vector<double2> cv(std::max(1, n), make_double2(0.0, 0.0));
            if (cvo && !(*cvo)[i].empty()) {
                for (int t = 0; t < n && t < (int)(*cvo)[i].size(); t++) cv[t] = (*cvo)[i][t];
            } else {
                if (p.scheme == OVL_DEFL_SCHUR)
                    for (int t = 0; t < p.m_q && t < n; t++)
                        cv[t] = make_double2(c1[i][t].x + c2[i][t].x, c1[i][t].y + c2[i][t].y);
                if (n > p.m_q) cv[p.m_q] = make_double2(beta[i], 0.0);
            }
            OVL_CUDA_TRY(lat,
                         cudaMemcpyAsync(p.cvec, cv.data(), std::max(1, n) * sizeof(double2), cudaMemcpyHostToDevice, st));
            OVL_CUDA_TRY(lat, cudaMemsetAsync(p.bar, 0, sizeof(unsigned), st));
            OVL_CUDA_TRY(lat, cudaMemsetAsync(p.nstat, 0, sizeof(int), st));
            OVL_CUDA_TRY(lat, cudaMemsetAsync(p.iters, 0, sizeof(int), st));
            OVL_CUDA_TRY(lat, cudaMemsetAsync(p.handoff, 0, sizeof(int), st));
            OVL_CUDA_TRY(lat, cudaStreamSynchronize(st));
        }
        OVL_CUDA_TRY(lat, cudaMemcpyAsync(d_nd, nd.data(), nsolve * sizeof(NewtonDev), cudaMemcpyHostToDevice, st));
        if (any_run) {
            int cpm_run = ovl_newton_cpm(lat, nsolve, nmax_run);
            ProfScope pn(lat, 5, 0.0, st);
            // 0: cluster (else cooperative) double-float Gauss-Jordan, Newton-Schulz finish;
            // 1: FP64 Gauss-Jordan; 2: cooperative double-float only; 3: cluster (else
            // cooperative) double-float only; 4: as 0 with every Newton-Schulz step
            // declined (the return to Gauss-Jordan)
            const int mode = nmode;
            int cl_size = 0, cl_nrs = 0, cl_l2 = 0, cpm_df = 1, smem_rows = 0;
            size_t cl_smem = 0;
            if (mode == 0 || mode == 3 || mode == 4)
                ovl_newton_cl_plan(lat, nsolve, nmax_run, &cl_size, &cl_smem, &cl_nrs, &cl_l2);
            if (mode != 1 && cl_size == 0) ovl_newton_df_plan(lat, nsolve, nmax_run, &cpm_df, &smem_rows);
            auto launch_gj = [&]() -> int {
                if (mode == 1) return ovl_newton_launch(lat, d_nd, nsolve, cpm_run, st);
                if (cl_size > 0) return ovl_newton_cl_launch(lat, d_nd, nsolve, cl_size, cl_smem, cl_nrs, cl_l2, st);
                return ovl_newton_df_launch(lat, d_nd, nsolve, nmax_run, cpm_df, smem_rows, st);
            };
            if (int rc = launch_gj()) return rc;
            if (mode == 0 || mode == 4) {
                std::vector<int> hf(nsolve, 0), it_gj(nsolve, 0);
                for (int i = 0; i < nsolve; i++) {
                    if (!nd[i].run) continue;
                    OVL_CUDA_TRY(lat, cudaMemcpyAsync(&hf[i], P[i].handoff, sizeof(int), cudaMemcpyDeviceToHost, st));
                    OVL_CUDA_TRY(lat, cudaMemcpyAsync(&it_gj[i], P[i].iters, sizeof(int), cudaMemcpyDeviceToHost, st));
                }
                OVL_CUDA_TRY(lat, cudaStreamSynchronize(st));
                std::vector<NsDev> hn(nsolve);
                bool any_ns = false;
                for (int i = 0; i < nsolve; i++) {
                    NsDev& z = hn[i];
                    memset(&z, 0, sizeof z);
                    z.X = (float4*)P[i].X;
                    z.W = (float4*)P[i].W;
                    z.Y = (float4*)P[i].Yns;
                    z.acc = P[i].nsacc;
                    z.n = nd[i].n;
                    z.on = nd[i].run && hf[i];
                    z.tol = nd[i].tol;
                    z.prev = 1e300;
                    z.region = mode == 4 ? 0.0 : 0.25;
                    any_ns = any_ns || z.on;
                }
                if (any_ns) {
                    if (int rc = ovl_newton_schulz(lat, d_ns, hn.data(), nsolve, nmax_run, NS_MAX_ITER, st)) return rc;
                    // matrices that left the Newton-Schulz region go back to Gauss-Jordan
                    std::vector<int> run0(nsolve), tot(nsolve);
                    bool any_fb = false;
                    for (int i = 0; i < nsolve; i++) {
                        run0[i] = nd[i].run;
                        tot[i] = it_gj[i] + hn[i].iters;
                        nd[i].run = run0[i] && hf[i] && hn[i].fallback;
                        nd[i].resume = 1;
                        nd[i].ns_switch = 0.0;
                        any_fb = any_fb || nd[i].run;
                    }
                    if (any_fb) {
                        for (int i = 0; i < nsolve; i++)  // the cooperative kernel's barrier starts at zero
                            if (nd[i].run) OVL_CUDA_TRY(lat, cudaMemsetAsync(P[i].bar, 0, sizeof(unsigned), st));
                        OVL_CUDA_TRY(lat, cudaMemcpyAsync(d_nd, nd.data(), nsolve * sizeof(NewtonDev),
                                                          cudaMemcpyHostToDevice, st));
                        if (int rc = launch_gj()) return rc;
                        std::vector<int> it2(nsolve, 0);
                        for (int i = 0; i < nsolve; i++)
                            if (nd[i].run)
                                OVL_CUDA_TRY(lat, cudaMemcpyAsync(&it2[i], P[i].iters, sizeof(int),
                                                                  cudaMemcpyDeviceToHost, st));
                        OVL_CUDA_TRY(lat, cudaStreamSynchronize(st));
                        for (int i = 0; i < nsolve; i++) tot[i] += it2[i];
                    }
                    for (int i = 0; i < nsolve; i++) {
                        nd[i].run = run0[i];
                        if (run0[i] && hf[i])
                            OVL_CUDA_TRY(lat, cudaMemcpyAsync(P[i].iters, &tot[i], sizeof(int), cudaMemcpyHostToDevice, st));
                    }
                    OVL_CUDA_TRY(lat, cudaMemcpyAsync(d_nd, nd.data(), nsolve * sizeof(NewtonDev),
                                                      cudaMemcpyHostToDevice, st));
                    OVL_CUDA_TRY(lat, cudaStreamSynchronize(st));  // tot, nd must outlive the copies
                }
            }
            if (int rc = ovl_fmatvec_launch(lat, d_nd, nsolve, nmax_run, st)) return rc;
            pn.end(st);
        }
        OVL_CUDA_TRY(lat, cudaStreamSynchronize(st));
        return OVL_OK;
    };
    // adaptive depth: estimate from the coefficients of the approximation at
    // depth j (H snapshot, accurate last-column correction on the copy, Newton)
    auto adaptive_check = [&](int j) -> int {
        OVL_CUDA_TRY(lat, cudaMemcpyAsync(hs.data(), d_sd, nsolve * sizeof(SolveDev), cudaMemcpyDeviceToHost, st));
        OVL_CUDA_TRY(lat, cudaStreamSynchronize(st));
        std::vector<SolveDev> he = hs;
        std::vector<int> ncol(nsolve, 0), nn(nsolve, 0);
        std::vector<const double2*> Hs(nsolve, nullptr);
        std::vector<double2*> go(nsolve, nullptr);
        bool any = false;
        for (int i = 0; i < nsolve; i++) {
            SolvePlan& p = P[i];
            bool on = p.adapt && hs[i].active && j <= p.k && j >= p.k_first && (j - p.k_first) % p.adapt == 0;
            he[i].fin = on ? 1 : 0;
            he[i].active = 0;
            if (!on) continue;
            any = true;
            size_t hb = (size_t)p.ldH * p.ldH;
            OVL_CUDA_TRY(lat, cudaMemcpyAsync(p.H_est, p.H, hb * sizeof(double2), cudaMemcpyDeviceToDevice, st));
            OVL_CUDA_TRY(lat, cudaMemcpyAsync(p.H32_est, p.H32, hb * sizeof(float2), cudaMemcpyDeviceToDevice, st));
            he[i].H = p.H_est;
            he[i].H32 = p.H32_est;
            he[i].k_used = j;
            ncol[i] = p.m_q + j;
            nn[i] = p.m_q + j;
            Hs[i] = p.H_est;
            go[i] = p.g_est;
        }
        if (!any) return OVL_OK;
        OVL_CUDA_TRY(lat, cudaMemcpyAsync(d_sd_est, he.data(), nsolve * sizeof(SolveDev), cudaMemcpyHostToDevice, st));
        if (int rc = final_pass(d_sd_est, ncol)) return rc;
        if (int rc = newton(Hs, nn, go)) return rc;
        bool changed = false;
        for (int i = 0; i < nsolve; i++) {
            if (!nn[i]) continue;
            SolvePlan& p = P[i];
            std::vector<double2> g(nn[i]);
            OVL_CUDA_TRY(lat, cudaMemcpy(g.data(), p.g_est, nn[i] * sizeof(double2), cudaMemcpyDeviceToHost));
            int st_n = 0;
            OVL_CUDA_TRY(lat, cudaMemcpy(&st_n, p.nstat, sizeof(int), cudaMemcpyDeviceToHost));
            if (st_n) continue;  // no estimate from a failed small sign; keep going
            if (!p.g_prev.empty()) {
                double dn = 0.0, gn = 0.0;
                for (size_t t = 0; t < g.size(); t++) {
                    double2 a = g[t], b = t < p.g_prev.size() ? p.g_prev[t] : make_double2(0.0, 0.0);
                    dn += (a.x - b.x) * (a.x - b.x) + (a.y - b.y) * (a.y - b.y);
                    gn += a.x * a.x + a.y * a.y;
                }
                p.err_est = gn > 0 ? sqrt(dn / gn) : 0.0;
                if (p.err_est <= 0.1 * p.tol) {
                    p.k = j;  // converged: stop this solve here
                    hs[i].k = j;
                    changed = true;
                }
            }
            p.g_prev = g;
        }
        if (changed)
            for (int i = 0; i < nsolve; i++)
                OVL_CUDA_TRY(lat, cudaMemcpyAsync(&d_sd[i].k, &P[i].k, sizeof(int), cudaMemcpyHostToDevice, st));
        OVL_CUDA_TRY(lat, cudaStreamSynchronize(st));
        return OVL_OK;
    };
    // The fixed-depth Arnoldi loop launches the same kernels with the same
    // arguments whenever a batch of the same shape runs on the same workspace:
    // with graphs enabled (ovl_set_graphs) the second such call captures the
    // loop into a CUDA graph and every later one replays it (one launch for
    // 5 k kernels). Not with adaptive depth (host decisions inside the loop)
    // or per-class profiling (events inside the loop).
    const bool graph_ok = lat->graphs && !any_adapt && !lat->prof;
    uint64_t gkey = 0;
    if (graph_ok) {
        auto mix = [&](uint64_t v) { gkey = (gkey ^ v) * 0x100000001b3ull; };
        gkey = 0xcbf29ce484222325ull;
        mix((uint64_t)(uintptr_t)lat->ws);
        mix((uint64_t)nsolve);
        mix((uint64_t)prec);
        mix((uint64_t)kmax);
        mix((uint64_t)links);
        for (int i = 0; i < nsolve; i++) {
            mix((uint64_t)P[i].k);
            mix((uint64_t)P[i].m_q);
            mix((uint64_t)(uintptr_t)(P[i].d ? P[i].d->S_hi : nullptr));
        }
        for (double v : mus) {
            uint64_t u;
            memcpy(&u, &v, sizeof u);
            mix(u);
        }
        uint64_t u;
        memcpy(&u, &da.kappa, sizeof u);  // baked into the stencil launches
        mix(u);
    }
    // a failure inside a capture ends the capture (discarding the graph) before returning
    auto end_capture = [&](int rc) -> int {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (lat->cap_stream && cudaStreamIsCapturing(lat->cap_stream, &cs) == cudaSuccess &&
            cs != cudaStreamCaptureStatusNone) {
            cudaGraph_t g = nullptr;
            cudaStreamEndCapture(lat->cap_stream, &g);
            if (g) cudaGraphDestroy(g);
        }
        cudaGetLastError();
        return rc;
    };
    bool replay = graph_ok && lat->graph_exec && lat->graph_key == gkey;
    bool capture = graph_ok && !replay && lat->graph_seen == gkey;
    if (graph_ok && !replay && !capture) lat->graph_seen = gkey;  // first call of this shape runs eagerly
    if (replay) {
        OVL_CUDA_TRY(lat, cudaGraphLaunch(lat->graph_exec, st));
        lat->launches += lat->graph_kernels;
        lat->graph_replays++;
    }
    const long long launches_before = lat->launches;
    // the loop's stream: the lattice's, or while capturing a private one (the
    // lattice's stream may be the legacy default stream, which cannot be
    // captured); a captured loop only records, the graph then runs on st
    cudaStream_t lst = st;
    if (capture) {
        if (lat->graph_exec) {
            cudaGraphExecDestroy(lat->graph_exec);
            lat->graph_exec = nullptr;
        }
        if (!lat->cap_stream) OVL_CUDA_TRY(lat, cudaStreamCreateWithFlags(&lat->cap_stream, cudaStreamNonBlocking));
        OVL_CUDA_TRY(lat, cudaStreamSynchronize(st));
        OVL_CUDA_TRY(lat, cudaStreamBeginCapture(lat->cap_stream, cudaStreamCaptureModeThreadLocal));
        lst = lat->cap_stream;
    }
    for (int j = 1; j <= kmax && !replay; j++) {
        int pmax = 0, nact = 0;
        double colsum = 0.0, colsum_s = 0.0;  // basis columns; of them Schur columns
        for (int i = 0; i < nsolve; i++)
            if (j <= P[i].k) {
                pmax = std::max(pmax, P[i].m_q + j - 1);
                nact++;
                colsum += P[i].m_q + j - 1;
                colsum_s += P[i].m_q;
            }
        if (!nact) break;
        bd.pmax = pmax;
        da.j = j;
        // algorithmic bytes: stencil 960 B/site (FP64); pass A reads the FP32 high
        // plane and u, w; pass B reads the full basis, u, w and writes u and q
        ProfScope p0(lat, 0, nact * (double)lat->V * site_bytes, lst);
        if (int rc = ovl_dslash_launch(lat, da, OVL_VEC_F64, links, lst)) return end_capture(rc);
        p0.end(lst);
        ProfScope p1(lat, 1, colsum * N * 8.0 + nact * 2.0 * N * 16.0, lst);
        if (int rc = ovl_gs_dot(lat, bd, j, lst)) return end_capture(rc);
        p1.end(lst);
        ProfScope p2(lat, 2, 0.0, lst);
        if (int rc = ovl_gs_reduce(lat, bd, j, lst)) return end_capture(rc);
        p2.end(lst);
        ProfScope p3(lat, 3, 0.0, lst);
        if (int rc = ovl_gs_small(lat, bd, j, lst)) return end_capture(rc);
        p3.end(lst);
        // the Schur columns keep FP32 low planes (16 B) in the 40-bit form
        const double bbytes = lo16 ? (colsum - colsum_s) * N * qbytes + colsum_s * N * 16.0 : colsum * N * qbytes;
        ProfScope p4(lat, 4, bbytes + nact * (3.0 * N * 16.0 + N * qbytes), lst);
        if (int rc = ovl_gs_update(lat, bd, j, lst)) return end_capture(rc);
        p4.end(lst);
        if (any_adapt)
            if (int rc = adaptive_check(j)) return rc;
    }
    if (capture) {
        cudaGraph_t g = nullptr;
        OVL_CUDA_TRY(lat, cudaStreamEndCapture(lat->cap_stream, &g));
        const cudaError_t e = cudaGraphInstantiate(&lat->graph_exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            lat->graph_exec = nullptr;
            return ovl_fail(lat, OVL_ECUDA, "ovl_sign_apply: graph instantiation failed: %s", cudaGetErrorString(e));
        }
        lat->graph_key = gkey;
        lat->graph_kernels = lat->launches - launches_before;
        OVL_CUDA_TRY(lat, cudaGraphLaunch(lat->graph_exec, st));
    }
    OVL_CUDA_TRY(lat, cudaMemcpyAsync(hs.data(), d_sd, nsolve * sizeof(SolveDev), cudaMemcpyDeviceToHost, st));
    OVL_CUDA_TRY(lat, cudaStreamSynchronize(st));
    {
        std::vector<int> ncol(nsolve);
        for (int i = 0; i < nsolve; i++) ncol[i] = hs[i].fin ? P[i].m_q + std::min(hs[i].k_used, P[i].k) : 0;
        // a solve stopped by the adaptive check: its depth is k (the loop stopped there)
        for (int i = 0; i < nsolve; i++)
            if (hs[i].fin && P[i].k < hs[i].k_used) {
                hs[i].k_used = P[i].k;
                OVL_CUDA_TRY(lat, cudaMemcpyAsync(&d_sd[i].k_used, &P[i].k, sizeof(int), cudaMemcpyHostToDevice, st));
            }
        if (int rc = final_pass(d_sd, ncol)) return rc;
    }
    OVL_CUDA_TRY(lat, cudaMemcpyAsync(hs.data(), d_sd, nsolve * sizeof(SolveDev), cudaMemcpyDeviceToHost, st));
    OVL_CUDA_TRY(lat, cudaStreamSynchronize(st));

    // ---- small sign by Newton ----
    std::vector<int> syl_on(nsolve, 0), nit_extra(nsolve, 0);
    std::vector<int> nstat(nsolve, 0), nit(nsolve, 0);
    {
        std::vector<const double2*> Hs(nsolve);
        std::vector<int> nn(nsolve);
        std::vector<double2*> go(nsolve);
        std::vector<std::vector<double2>> cvo(nsolve);
        for (int i = 0; i < nsolve; i++) {
            SolvePlan& p = P[i];
            const int ku = hs[i].status == 0 ? hs[i].k_used : 0;
            syl_on[i] = syl && p.m_q > 0 && ku > 0;
            if (syl_on[i]) {  // sgn(H_k) beta e_1 on the Krylov block alone (Eq. 19)
                Hs[i] = p.H + (size_t)p.m_q * (p.ldH + 1);
                nn[i] = ku;
                go[i] = p.gcomb + p.m_q;
                cvo[i].assign(1, make_double2(beta[i], 0.0));
            } else {
                Hs[i] = p.H;
                nn[i] = hs[i].status == 0 ? p.m_q + ku : 0;
                go[i] = p.gcomb;
            }
        }
        if (int rc = newton(Hs, nn, go, &cvo)) return rc;
        for (int i = 0; i < nsolve; i++) {  // status and iterations of this run (a second run resets them)
            OVL_CUDA_TRY(lat, cudaMemcpyAsync(&nstat[i], P[i].nstat, sizeof(int), cudaMemcpyDeviceToHost, st));
            OVL_CUDA_TRY(lat, cudaMemcpyAsync(&nit[i], P[i].iters, sizeof(int), cudaMemcpyDeviceToHost, st));
        }
        OVL_CUDA_TRY(lat, cudaStreamSynchronize(st));
        bool any_syl = false;
        for (int i = 0; i < nsolve; i++) any_syl = any_syl || syl_on[i];
        if (any_syl) {
            // keep sgn(H_k), then sgn(T) S^dag b from the Newton kernels on T
            const std::vector<NewtonDev> nd_first = nd;
            for (int i = 0; i < nsolve; i++) {
                if (!syl_on[i]) continue;
                const size_t kk = (size_t)hs[i].k_used;
                OVL_CUDA_TRY(lat, cudaMemcpyAsync(P[i].syFH, P[i].X, kk * kk * sizeof(double2),
                                                  cudaMemcpyDeviceToDevice, st));
            }
            int nst = 0;
            for (int i = 0; i < nsolve; i++)
                if (syl_on[i] && nstat[i]) nst = nstat[i];
            for (int i = 0; i < nsolve; i++) {
                Hs[i] = P[i].H;
                nn[i] = syl_on[i] ? P[i].m_q : 0;
                go[i] = P[i].sygT;
                cvo[i].clear();
                if (syl_on[i])
                    for (int t = 0; t < P[i].m_q; t++)
                        cvo[i].push_back(make_double2(c1[i][t].x + c2[i][t].x, c1[i][t].y + c2[i][t].y));
            }
            if (!nst) {
                if (int rc = newton(Hs, nn, go, &cvo)) return rc;
                std::vector<SylDev> sy(nsolve);
                int mmax = 0;
                for (int i = 0; i < nsolve; i++) {
                    SylDev& z = sy[i];
                    memset(&z, 0, sizeof z);
                    if (!syl_on[i]) continue;
                    SolvePlan& p = P[i];
                    z.H = p.H;
                    z.ldH = p.ldH;
                    z.m = p.m_q;
                    z.k = hs[i].k_used;
                    z.on = 1;
                    z.df = nmode == 1 ? 0 : 1;
                    z.FT = p.X;
                    z.FH = p.syFH;
                    z.R = p.syR;
                    z.Y = p.syY;
                    z.W = p.syW;
                    z.r = p.syr;
                    z.gT = p.sygT;
                    z.gS = p.gcomb;
                    z.beta = beta[i];
                    mmax = std::max(mmax, p.m_q);
                }
                OVL_CUDA_TRY(lat, cudaMemcpyAsync(bp.sy, sy.data(), nsolve * sizeof(SylDev), cudaMemcpyHostToDevice, st));
                ProfScope py(lat, 5, 0.0, st);
                if (int rc = ovl_sylvester_launch(lat, bp.sy, nsolve, mmax, st)) return rc;
                py.end(st);
                OVL_CUDA_TRY(lat, cudaStreamSynchronize(st));  // sy must outlive the copy
                for (int i = 0; i < nsolve; i++) {
                    if (!syl_on[i]) continue;
                    int s2 = 0, i2 = 0;
                    OVL_CUDA_TRY(lat, cudaMemcpy(&s2, P[i].nstat, sizeof(int), cudaMemcpyDeviceToHost));
                    OVL_CUDA_TRY(lat, cudaMemcpy(&i2, P[i].iters, sizeof(int), cudaMemcpyDeviceToHost));
                    if (!nstat[i]) nstat[i] = s2;
                    nit_extra[i] = i2;  // iterations on T, added to those on H_k
                }
            }
            // the recombination below runs over the m + k columns of each solve
            nd = nd_first;
            for (int i = 0; i < nsolve; i++)
                if (syl_on[i]) nd[i].n = P[i].m_q + hs[i].k_used;
        }
    }
    for (int i = 0; i < nsolve; i++)
        if (syl_on[i]) nit[i] += nit_extra[i];  // iterations on H_k plus those on T

    // ---- recombination ----
    std::vector<GemvDev> gd(nsolve);
    int gmax = 0;
    for (int i = 0; i < nsolve; i++) {
        SolvePlan& p = P[i];
        int n = nd[i].run ? nd[i].n : 0;
        std::vector<const float2*> ch, cl;
        std::vector<double2> extra;
        for (int cidx = 0; cidx < n; cidx++) {
            if (f64) {
                ch.push_back(cidx < p.m_q ? (const float2*)(p.d->S64 + N * cidx)
                                          : (const float2*)((double2*)p.Vhi + N * (cidx - p.m_q)));
                cl.push_back(nullptr);
            } else if (cidx < p.m_q) {
                ch.push_back(p.d->S_hi + N * cidx);
                cl.push_back(p.d->S_lo + N * cidx);
            } else {
                ch.push_back(p.Vhi + N * (cidx - p.m_q));
                cl.push_back(!df ? nullptr
                             : lo16 ? (const float2*)((const char*)p.Vlo + (size_t)4 * N * (cidx - p.m_q))
                                    : p.Vlo + N * (cidx - p.m_q));
            }
        }
        if (p.scheme == OVL_DEFL_LR) {
            // R sgn(Lambda) L^dag b  (Eq. 22, f = sgn on the diagonal)
            for (int t = 0; t < p.m_defl; t++) {
                ch.push_back(f64 ? (const float2*)(p.d->S64 + N * t) : p.d->S_hi + N * t);
                cl.push_back(f64 ? nullptr : p.d->S_lo + N * t);
                double lre = p.d->T_host[2 * t];
                double sg = lre > 0 ? 1.0 : (lre < 0 ? -1.0 : 0.0);
                extra.push_back(make_double2(sg * c1[i][t].x, sg * c1[i][t].y));
            }
        }
        if (!extra.empty())
            OVL_CUDA_TRY(lat, cudaMemcpyAsync(p.gcomb + n, extra.data(), extra.size() * sizeof(double2),
                                              cudaMemcpyHostToDevice, st));
        OVL_CUDA_TRY(lat, cudaMemcpyAsync(p.gc_hi, ch.data(), ch.size() * sizeof(void*), cudaMemcpyHostToDevice, st));
        OVL_CUDA_TRY(lat, cudaMemcpyAsync(p.gc_lo, cl.data(), cl.size() * sizeof(void*), cudaMemcpyHostToDevice, st));
        OVL_CUDA_TRY(lat, cudaStreamSynchronize(st));
        gd[i].qhi = p.gc_hi;
        gd[i].qlo = p.gc_lo;
        gd[i].g = p.gcomb;
        gd[i].y = p.w;
        gd[i].ncol = (int)ch.size();
        gd[i].f64 = f64;
        gd[i].lo16_from = lo16 ? p.m_q : 0;  // the Krylov columns; Schur and LR columns keep FP32 low planes
        gd[i].lo16_to = lo16 ? n : 0;
        gmax = std::max(gmax, gd[i].ncol);
    }
    OVL_CUDA_TRY(lat, cudaMemcpyAsync(d_gd, gd.data(), nsolve * sizeof(GemvDev), cudaMemcpyHostToDevice, st));
    double gb = 0.0;
    for (int i = 0; i < nsolve; i++) gb += (double)gd[i].ncol * N * 16.0 + N * 16.0;
    ProfScope pg(lat, 7, gb, st);
    if (int rc = ovl_gemv_df(lat, d_gd, nsolve, gmax, st, f64)) return rc;
    pg.end(st);
    // ---- outputs ----
    bool ydev = ovl_is_device_ptr(y);
    for (int i = 0; i < nsolve; i++) {
        double* dst = ydev ? y + 2 * N * i : (double*)(d_canon + N * i);
        if (int rc = ovl_unpack_impl(lat, P[i].w, dst, 1, OVL_VEC_F64, st)) return rc;
    }
    if (!ydev)
        OVL_CUDA_TRY(lat, cudaMemcpyAsync(y, d_canon, N * sizeof(double2) * nsolve, cudaMemcpyDeviceToHost, st));
    OVL_CUDA_TRY(lat, cudaStreamSynchronize(st));
    int first_bad = OVL_OK;
    for (int i = 0; i < nsolve; i++) {
        int stt = hs[i].status ? hs[i].status : nstat[i];
        if (stt && !first_bad) first_bad = stt;
        if (info) {
            info[i].status = stt;
            info[i].k_used = hs[i].k_used;
            info[i].m_used = P[i].m_defl;
            info[i].newton_iters = nit[i];
            info[i].beta = beta[i];
            double bk = 0.0;
            cudaMemcpy(&bk, P[i].scal + 4, sizeof(double), cudaMemcpyDeviceToHost);
            info[i].beta_k = bk;
            info[i].err_est = P[i].err_est;
        }
    }
    ovl_prof_flush(lat);
    if (first_bad) return ovl_fail(lat, first_bad, "ovl_sign_apply: a solve failed (first status %d)", first_bad);
    return OVL_OK;
}

extern "C" int ovl_sign_apply(ovl_lattice lat, int nsolve, const ovl_sign_params* params, const ovl_deflation* defl,
                              const double* b, double* y, ovl_sign_info* info) {
    return sign_apply_impl(lat, nsolve, params, defl, b, y, info, nullptr);
}

extern "C" int ovl_sign_workspace_bytes(ovl_lattice lat, int nsolve, const ovl_sign_params* params,
                                        const ovl_deflation* defl, double* bytes) {
    if (!bytes) return ovl_fail(lat, OVL_EINVAL, "ovl_sign_workspace_bytes: null argument");
    size_t n = 0;
    if (int rc = sign_apply_impl(lat, nsolve, params, defl, nullptr, nullptr, nullptr, &n)) return rc;
    *bytes = (double)n;
    return OVL_OK;
}

extern "C" int ovl_deflation_stats(ovl_deflation d, int* restarts, int* matvecs) {
    if (!d) return ovl_fail(nullptr, OVL_EINVAL, "ovl_deflation_stats: null handle");
    if (restarts) *restarts = d->setup_restarts;
    if (matvecs) *matvecs = d->setup_matvecs;
    return OVL_OK;
}

extern "C" int ovl_set_graphs(ovl_lattice lat, int enable, long long* replays) {
    if (!lat) return ovl_fail(lat, OVL_EINVAL, "ovl_set_graphs: null handle");
    if (enable == 0 || enable == 1) {
        lat->graphs = enable != 0;
        if (!enable && lat->graph_exec) {
            cudaStreamSynchronize(lat->stream);
            cudaGraphExecDestroy(lat->graph_exec);
            lat->graph_exec = nullptr;
            lat->graph_key = lat->graph_seen = 0;
        }
    } else if (enable != -1) {
        return ovl_fail(lat, OVL_EINVAL, "ovl_set_graphs: enable=%d (0, 1, or -1 to query)", enable);
    }
    if (replays) *replays = lat->graph_replays;
    return OVL_OK;
}
