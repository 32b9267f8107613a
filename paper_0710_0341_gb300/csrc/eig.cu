// Deflation setup: the m critical eigenpairs of A = H_w(mu) (Secs. 3-5).
//
// The eigenvalues closest to the imaginary axis (smallest |Re lambda|) are
// interior points of the spectrum, where Krylov methods converge slowly. The
// map lambda -> lambda^2 sends them to the left end of the spectrum of A^2
// (Re lambda^2 = (Re lambda)^2 - (Im lambda)^2), where they are extremal. So
// the setup runs restarted Arnoldi (Krylov-Schur: Stewart, SIAM J. Matrix
// Anal. Appl. 23 (2001) 601) on B = A^2 for the nev = m + extra Ritz values
// of smallest real part, then a Rayleigh-Ritz step with A itself on the
// converged invariant subspace of B, and keeps the m eigenpairs of A with
// smallest |Re lambda| (ties: |Im lambda|).
//
// Polynomial filter: the wanted eigenvalues of B = A^2 sit at the left end
// of its spectrum, close to each other compared with the spread of the rest,
// so plain restarted Arnoldi on B converges slowly. After one unfiltered
// expansion gives the spread [Re theta_0, |theta|_max] of the Ritz values,
// the solver restarts on C = T_d(l(B)), a Chebyshev polynomial of degree d in
// the affine map l that sends the damped interval [a, b] (a: a Ritz value well
// above the wanted ones, b: above the largest) to [-1, 1]; eigenvalues of B
// left of a map to |T_d| > 1 and grow like exp(d acosh l), the rest stay in
// [-1, 1] (Saad, Numerical Methods for Large Eigenvalue Problems, 2nd ed.,
// Sec. 7.4; Zhou and Saad, J. Comput. Phys. 219 (2006) 172). C has the
// eigenvectors of B, so the final Rayleigh-Ritz step with A is unchanged.
// Each application of C is d applications of B by the three-term recurrence
// y_{i+1} = 2 l(B) y_i - y_{i-1}.
//
// Work split: every O(N) operation (stencil, Gram-Schmidt, restart
// combinations V Z, projections) runs in this library's kernels on the GPU;
// the O(p^3) projected eigenproblems (p = basis size, at most a few hundred)
// run on the host CPU in the library's own small dense code (smallla.h),
// because GB300 issues FP64 at about 2 FMA per clock per SM and a serial
// p^3 Schur iteration on one SM would take longer than on one Grace core.
//
// Schur deflation gets S_m (orthonormal) and upper triangular T_m with
// A S_m = S_m T_m (Eq. 13); LR deflation also runs the solver on
// A^dag = H_w(-mu) for the left eigenvectors, pairs them by
// lambda_left = conj(lambda_right) and scales them to L^dag R = I (Eq. 20).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <random>

#include "df.cuh"
#include "krylov.cuh"
#include "smallla.h"

using sla::cd;
using sla::Mat;

namespace {

__global__ void k_join(const float2* __restrict__ hi, const float2* __restrict__ lo, double2* __restrict__ x,
                       size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        float2 a = hi[i], b = lo[i];
        x[i] = make_double2((double)a.x + (double)b.x, (double)a.y + (double)b.y);
    }
}
__global__ void k_split_scale(const double2* __restrict__ x, double s, float2* __restrict__ hi,
                              float2* __restrict__ lo, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        double2 v = x[i];
        float2 a = split_d(v.x * s), b = split_d(v.y * s);
        hi[i] = make_float2(a.x, b.x);
        lo[i] = make_float2(a.y, b.y);
    }
}

// out = sy*y + sz*z + syp*yp (yp may be null): one step of the Chebyshev
// recurrence with z = B y
// (out may be yp: each element is read before it is written)
__global__ void k_cheb(double2* out, const double2* __restrict__ z, const double2* __restrict__ y, const double2* yp,
                       double sy, double sz, double syp, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        double2 a = y[i], b = z[i];
        double2 r = make_double2(sy * a.x + sz * b.x, sy * a.y + sz * b.y);
        if (yp) {
            double2 c = yp[i];
            r.x += syp * c.x;
            r.y += syp * c.y;
        }
        out[i] = r;
    }
}

unsigned nblk(ovl_lattice lat, size_t n) {
    size_t b = (n + 255) / 256, cap = (size_t)lat->num_sms * 8;
    return (unsigned)std::max<size_t>(1, std::min(b, cap));
}

struct Dev {
    ovl_lattice lat;
    std::vector<void*> allocs;
    ~Dev() {
        for (void* p : allocs) cudaFree(p);
    }
    template <class T>
    T* get(size_t n) {
        void* p = nullptr;
        if (cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T)) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        allocs.push_back(p);
        return (T*)p;
    }
};

#define TRYP(ptr)                                                                                   \
    do {                                                                                            \
        if (!(ptr)) return ovl_fail(lat, OVL_ENOMEM, "deflation setup: device allocation failed"); \
    } while (0)

struct EigResult {
    std::vector<cd> lam;  // m eigenvalues of A
    Mat Ccoef;            // nev x m coefficients of the vectors in the basis Vf
    double resmax = 0.0;
};

// One restarted-Arnoldi run on B = A(mu)^2; on success the nev basis vectors
// (FP64, packed) are in Vf and the Rayleigh-Ritz data of A on them in G, M.
class Solver {
   public:
    ovl_lattice lat;
    cudaStream_t st;
    size_t N;
    int p, nev;
    double mu, kappa;
    Dev mem;
    float2 *Va_hi = nullptr, *Va_lo, *Vb_hi, *Vb_lo;
    double2 *u, *w, *tmp, *H, *dots, *dvec, *part, *Vf, *Wf, *gcoef;
    float2 *H32, *ap, *gh, *gl;
    double* scal;
    const float2 **qhi, **qlo;
    SolveDev* d_sd;
    ProjDev* d_pd;
    GemvDev* d_gd;
    const float2** gptr;  // gemv column pointer arrays (hi, lo)
    void** dsl;           // dslash pointer arrays
    double* d_mu;
    int G, pstride;
    int restarts = 0, matvecs = 0;
    int power = 2;            // operator B = A^power
    // Chebyshev filter C = T_d(l(B)), l(z) = (cheb_c - z) / cheb_e; off while cheb_deg == 0.
    // poly < 0: chosen after the first expansion; 0: never; > 0: that degree
    int poly = -1, cheb_deg = 0;
    double cheb_c = 0.0, cheb_e = 1.0, cheb_a = 0.0, cheb_b = 0.0;
    double2 *cb0 = nullptr, *cb1 = nullptr, *cz = nullptr;
    void** dslc = nullptr;    // device pointer table {u, tmp, w, cb0, cb1, cz}
    bool start_given = false; // u already holds the start vector (packed FP64)
    bool single = false;      // one expansion only: H of the k-step Arnoldi in Hsingle
    Mat Hsingle;

    Solver(ovl_lattice L, double mu_, double m_w, int p_, int nev_)
        : lat(L), st(L->stream), N(L->N), p(p_), nev(nev_), mu(mu_), kappa(1.0 / (8.0 + 2.0 * m_w)), mem{L} {}

    int alloc() {
        size_t cols = (size_t)p + 1;
        TRYP(Va_hi = mem.get<float2>(N * cols));
        TRYP(Va_lo = mem.get<float2>(N * cols));
        TRYP(Vb_hi = mem.get<float2>(N * cols));
        TRYP(Vb_lo = mem.get<float2>(N * cols));
        TRYP(u = mem.get<double2>(N));
        TRYP(w = mem.get<double2>(N));
        TRYP(tmp = mem.get<double2>(N));
        size_t ld = cols;
        TRYP(H = mem.get<double2>(ld * ld));
        TRYP(H32 = mem.get<float2>(ld * ld));
        TRYP(dots = mem.get<double2>(2 * ld + 3));
        TRYP(dvec = mem.get<double2>(ld + 1));
        TRYP(ap = mem.get<float2>(ld));
        TRYP(gh = mem.get<float2>(ld));
        TRYP(gl = mem.get<float2>(ld));
        TRYP(scal = mem.get<double>(8));
        TRYP(qhi = mem.get<const float2*>(ld));
        TRYP(qlo = mem.get<const float2*>(ld));
        G = ovl_gs_grid(lat);
        pstride = 2 * (int)ld + 3;
        TRYP(part = mem.get<double2>((size_t)std::max(G * pstride, G * (int)(ld + 1) * 1) * (size_t)std::max(1, nev)));
        TRYP(d_sd = mem.get<SolveDev>(1));
        TRYP(d_pd = mem.get<ProjDev>(ld));
        TRYP(d_gd = mem.get<GemvDev>(ld));
        TRYP(gptr = mem.get<const float2*>(2 * ld * ld));
        TRYP(gcoef = mem.get<double2>(ld * ld));
        TRYP(dsl = mem.get<void*>(8));
        TRYP(d_mu = mem.get<double>(2));
        TRYP(Vf = mem.get<double2>(N * (size_t)nev));
        TRYP(Wf = mem.get<double2>(N * (size_t)nev));
        void* hp[4] = {u, tmp, tmp, w};
        OVL_CUDA_TRY(lat, cudaMemcpyAsync(dsl, hp, sizeof hp, cudaMemcpyHostToDevice, st));
        if (poly != 0 && power == 2) {
            TRYP(cb0 = mem.get<double2>(N));
            TRYP(cb1 = mem.get<double2>(N));
            TRYP(cz = mem.get<double2>(N));
            TRYP(dslc = mem.get<void*>(6));
            void* tp[6] = {u, tmp, w, cb0, cb1, cz};
            OVL_CUDA_TRY(lat, cudaMemcpyAsync(dslc, tp, sizeof tp, cudaMemcpyHostToDevice, st));
        }
        OVL_CUDA_TRY(lat, cudaMemcpyAsync(d_mu, &mu, sizeof(double), cudaMemcpyHostToDevice, st));
        return OVL_OK;
    }

    // dst = A (A src) through tmp; indices into dslc {0 u, 1 tmp, 2 w, 3 cb0, 4 cb1, 5 cz}
    int apply_A2(int src, int dst) {
        DslashArgs a;
        a.in = (const void* const*)(dslc + src);
        a.out = (void* const*)(dslc + 1);
        a.mu = d_mu;
        a.nrhs = 1;
        a.kappa = kappa;
        if (int rc = ovl_dslash_launch(lat, a, OVL_VEC_F64, OVL_LINKS_F64, st)) return rc;
        a.in = (const void* const*)(dslc + 1);
        a.out = (void* const*)(dslc + dst);
        matvecs++;
        return ovl_dslash_launch(lat, a, OVL_VEC_F64, OVL_LINKS_F64, st);
    }

    // w = T_d(l(B)) u by the Chebyshev recurrence (y_0 = u, y_1 = l(B) u,
    // y_{i+1} = 2 l(B) y_i - y_{i-1}); the iterates rotate through cb0, cb1
    // (an update may overwrite y_{i-1} in place), B y_i goes to cz
    int apply_filter() {
        double2* vec[6] = {u, tmp, w, cb0, cb1, cz};
        const double ie = 1.0 / cheb_e;
        int prev = 0, cur = 0;
        for (int i = 0; i < cheb_deg; i++) {
            if (int rc = apply_A2(cur, 5)) return rc;
            const int nxt = (i == cheb_deg - 1) ? 2 : (i == 0 ? 3 : (prev == 0 ? 4 : prev));
            if (i == 0)
                k_cheb<<<nblk(lat, N), 256, 0, st>>>(vec[nxt], cz, u, nullptr, cheb_c * ie, -ie, 0.0, N);
            else
                k_cheb<<<nblk(lat, N), 256, 0, st>>>(vec[nxt], cz, vec[cur], vec[prev], 2.0 * cheb_c * ie, -2.0 * ie,
                                                     -1.0, N);
            OVL_LAUNCH_CHECK(lat);
            prev = cur;
            cur = nxt;
        }
        return OVL_OK;
    }

    // Interval [a, b] and degree of the filter from the Ritz values theta of B
    // of one unfiltered expansion (ascending real parts): b above the largest
    // |theta|, a at a Ritz value with 2 nev or more below it (for Hermitian B
    // the i-th Ritz value from the left bounds the i-th eigenvalue from above,
    // so at least that many eigenvalues lie left of a), d so that
    // |T_d| reaches about 1e4 at the leftmost Ritz value. Returns false when
    // the spread gives no useful filter.
    bool choose_filter(const std::vector<double>& re, double amax) {
        const int n = (int)re.size();
        if (n < 4) return false;
        const int ia = std::min(n - 1, std::max(2 * nev, nev + 20));
        const double a = re[ia], b = 1.1 * amax, lo = re[0];
        if (!(a > lo) || !(a < 0.5 * b) || !(lo > -b)) return false;
        cheb_a = a;
        cheb_b = b;
        cheb_c = 0.5 * (a + b);
        cheb_e = 0.5 * (b - a);
        const double x0 = (cheb_c - lo) / cheb_e;  // > 1
        int d = poly > 0 ? poly : (int)ceil(acosh(1e4) / acosh(x0));
        d = std::max(5, std::min(d, 201));
        cheb_deg = d | 1;  // odd: an eigenvalue of B right of b (l < -1) gives a large negative T_d, never wanted
        return true;
    }

    // w = B u = A (A u), or A u when power == 1; the filtered operator once chosen
    int apply_B() {
        if (cheb_deg > 0 && power == 2) return apply_filter();
        DslashArgs a;
        a.in = (const void* const*)dsl;
        a.out = (void* const*)(dsl + 1);
        a.mu = d_mu;
        a.nrhs = 1;
        a.kappa = kappa;
        if (power == 1) {
            a.out = (void* const*)(dsl + 3);  // straight into w
            matvecs++;
            return ovl_dslash_launch(lat, a, OVL_VEC_F64, OVL_LINKS_F64, st);
        }
        if (int rc = ovl_dslash_launch(lat, a, OVL_VEC_F64, OVL_LINKS_F64, st)) return rc;
        a.in = (const void* const*)(dsl + 2);
        a.out = (void* const*)(dsl + 3);
        matvecs++;
        return ovl_dslash_launch(lat, a, OVL_VEC_F64, OVL_LINKS_F64, st);
    }

    int set_columns(const float2* hi, const float2* lo) {
        std::vector<const float2*> h(p + 1), l(p + 1);
        for (int c = 0; c <= p; c++) {
            h[c] = hi + N * c;
            l[c] = lo + N * c;
        }
        OVL_CUDA_TRY(lat, cudaMemcpyAsync(qhi, h.data(), (p + 1) * sizeof(void*), cudaMemcpyHostToDevice, st));
        OVL_CUDA_TRY(lat, cudaMemcpyAsync(qlo, l.data(), (p + 1) * sizeof(void*), cudaMemcpyHostToDevice, st));
        return cudaStreamSynchronize(st) == cudaSuccess ? OVL_OK : ovl_fail(lat, OVL_ECUDA, "sync failed");
    }

    // inner products P[c][i] = Q_c^dag x_i (FP64), Q columns from (hi, lo) arrays
    int dots_many(const float2* const* chi, const float2* const* clo, int ncol, const std::vector<double2*>& xs,
                  Mat& out) {
        int nx = (int)xs.size();
        std::vector<ProjDev> pd(nx);
        double2* outbuf = gcoef;  // (ncol+1) * nx <= ld*ld
        for (int i = 0; i < nx; i++) {
            pd[i].qhi = chi;
            pd[i].qlo = clo;
            pd[i].x = xs[i];
            pd[i].out = outbuf + (size_t)i * (ncol + 1);
            pd[i].coef = nullptr;
            pd[i].ncol = ncol;
        }
        OVL_CUDA_TRY(lat, cudaMemcpyAsync(d_pd, pd.data(), nx * sizeof(ProjDev), cudaMemcpyHostToDevice, st));
        if (int rc = ovl_proj_dot(lat, d_pd, nx, ncol, part, G, st)) return rc;
        std::vector<double2> h((size_t)(ncol + 1) * nx);
        OVL_CUDA_TRY(lat, cudaMemcpyAsync(h.data(), outbuf, h.size() * sizeof(double2), cudaMemcpyDeviceToHost, st));
        OVL_CUDA_TRY(lat, cudaStreamSynchronize(st));
        out = Mat(ncol + 1, nx);  // last row: |x_i|^2
        for (int i = 0; i < nx; i++)
            for (int c = 0; c <= ncol; c++) out(c, i) = cd(h[(size_t)i * (ncol + 1) + c].x, h[(size_t)i * (ncol + 1) + c].y);
        return OVL_OK;
    }

    // y_i = sum_c Q_c C(c, i) for i < nout (df accumulation), FP64 packed outputs
    int combine(const float2* hi, const float2* lo, int ncol, const Mat& C, int nout, const std::vector<double2*>& ys) {
        std::vector<const float2*> ph(ncol), pl(ncol);
        for (int c = 0; c < ncol; c++) {
            ph[c] = hi + N * c;
            pl[c] = lo + N * c;
        }
        OVL_CUDA_TRY(lat, cudaMemcpyAsync(gptr, ph.data(), ncol * sizeof(void*), cudaMemcpyHostToDevice, st));
        OVL_CUDA_TRY(lat, cudaMemcpyAsync(gptr + ncol, pl.data(), ncol * sizeof(void*), cudaMemcpyHostToDevice, st));
        std::vector<double2> co((size_t)ncol * nout);
        for (int i = 0; i < nout; i++)
            for (int c = 0; c < ncol; c++) co[(size_t)i * ncol + c] = make_double2(C(c, i).real(), C(c, i).imag());
        OVL_CUDA_TRY(lat, cudaMemcpyAsync(gcoef, co.data(), co.size() * sizeof(double2), cudaMemcpyHostToDevice, st));
        std::vector<GemvDev> gd(nout);
        for (int i = 0; i < nout; i++) {
            gd[i].qhi = gptr;
            gd[i].qlo = gptr + ncol;
            gd[i].g = gcoef + (size_t)i * ncol;
            gd[i].y = ys[i];
            gd[i].ncol = ncol;
        }
        OVL_CUDA_TRY(lat, cudaMemcpyAsync(d_gd, gd.data(), nout * sizeof(GemvDev), cudaMemcpyHostToDevice, st));
        if (int rc = ovl_gemv_df(lat, d_gd, nout, ncol, st)) return rc;
        return cudaStreamSynchronize(st) == cudaSuccess ? OVL_OK : ovl_fail(lat, OVL_ECUDA, "combine failed");
    }

    int run(double tol, int max_restarts, uint64_t seed) {
        if (!Va_hi)
            if (int rc = alloc()) return rc;
        const size_t ld = p + 1;
        // random start vector (seeded), packed order is irrelevant for it
        if (!start_given) {
            std::mt19937_64 gen(seed);
            std::normal_distribution<double> nd;
            std::vector<double2> x(N);
            for (auto& v : x) v = make_double2(nd(gen), nd(gen));
            OVL_CUDA_TRY(lat, cudaMemcpyAsync(u, x.data(), N * sizeof(double2), cudaMemcpyHostToDevice, st));
            OVL_CUDA_TRY(lat, cudaStreamSynchronize(st));
        }
        float2 *cur_hi = Va_hi, *cur_lo = Va_lo, *nxt_hi = Vb_hi, *nxt_lo = Vb_lo;
        int q = 0;            // kept columns
        Mat Tq, bq;           // kept Rayleigh quotient and coupling row
        double bnorm = 0.0;   // |B| estimate (largest Ritz value seen)
        bool first = true;
        for (restarts = 0; restarts <= max_restarts; restarts++) {
            if (int rc = set_columns(cur_hi, cur_lo)) return rc;
            // H = [[T_q, *], [b^T, *]] with zeros elsewhere
            std::vector<double2> Hh(ld * ld, make_double2(0.0, 0.0));
            for (int j = 0; j < q; j++) {
                for (int i = 0; i < q; i++) Hh[i + j * ld] = make_double2(Tq(i, j).real(), Tq(i, j).imag());
                Hh[q + j * ld] = make_double2(bq(0, j).real(), bq(0, j).imag());
            }
            OVL_CUDA_TRY(lat, cudaMemcpyAsync(H, Hh.data(), ld * ld * sizeof(double2), cudaMemcpyHostToDevice, st));
            std::vector<float2> H32h(ld * ld);
            for (size_t i = 0; i < ld * ld; i++) H32h[i] = make_float2((float)Hh[i].x, (float)Hh[i].y);
            OVL_CUDA_TRY(lat, cudaMemcpyAsync(H32, H32h.data(), ld * ld * sizeof(float2), cudaMemcpyHostToDevice, st));
            SolveDev s;
            memset(&s, 0, sizeof s);
            s.qhi = qhi;
            s.qlo = qlo;
            s.vhi = cur_hi;
            s.vlo = cur_lo;
            s.nptr = 0;
            s.u = u;
            s.w = w;
            s.H = H;
            s.H32 = H32;
            s.dots = dots;
            s.dvec = dvec;
            s.ap = ap;
            s.gh = gh;
            s.gl = gl;
            s.scal = scal;
            s.m_q = q;
            s.k = p - q;
            s.ldH = (int)ld;
            s.active = 1;
            s.k_used = p - q;
            s.fin = 1;
            OVL_CUDA_TRY(lat, cudaMemcpyAsync(d_sd, &s, sizeof s, cudaMemcpyHostToDevice, st));
            BatchDev bd = {};
            bd.sd = d_sd;
            bd.nsolve = 1;
            bd.N = N;
            bd.part = part;
            bd.G = G;
            bd.pstride = pstride;
            bd.df = 1;
            bd.bulk16 = N % 4 == 0 && (uintptr_t)cur_hi % 16 == 0 && (uintptr_t)cur_lo % 16 == 0;
            if (first) {
                // v_1 = x/|x| into column 0
                Mat nn;
                std::vector<double2*> xs{u};
                if (int rc = dots_many(qhi, qlo, 0, xs, nn)) return rc;
                double b2 = nn(0, 0).real();
                OVL_CUDA_TRY(lat, cudaMemcpyAsync(d_mu + 1, &b2, sizeof(double), cudaMemcpyHostToDevice, st));
                if (int rc = ovl_start_vector(lat, bd, d_mu + 1, 1, st)) return rc;
                first = false;
            }
            // expansion: column q holds the (normalised) start vector already
            for (int j = 1; j <= p - q; j++) {
                bd.pmax = q + j - 1;
                if (int rc = apply_B()) return rc;
                if (int rc = ovl_gs_dot(lat, bd, j, st)) return rc;
                if (int rc = ovl_gs_reduce(lat, bd, j, st)) return rc;
                if (int rc = ovl_gs_small(lat, bd, j, st)) return rc;
                if (int rc = ovl_gs_update(lat, bd, j, st)) return rc;
            }
            OVL_CUDA_TRY(lat, cudaMemcpyAsync(&s, d_sd, sizeof s, cudaMemcpyDeviceToHost, st));
            OVL_CUDA_TRY(lat, cudaStreamSynchronize(st));
            if (s.status) return ovl_fail(lat, OVL_ENOCONV, "deflation setup: Arnoldi failed (status %d)", s.status);
            int pc = q + s.k_used;  // columns reached (breakdown: invariant subspace)
            // accurate last-column correction s = Q^dag u and the residual vector
            {
                ProjDev pd = {};
                pd.qhi = qhi;
                pd.qlo = qlo;
                pd.x = u;
                pd.out = dots;
                pd.coef = dots;
                pd.ncol = pc;
                OVL_CUDA_TRY(lat, cudaMemcpyAsync(d_pd, &pd, sizeof pd, cudaMemcpyHostToDevice, st));
                bd.pmax = pc;
                if (int rc = ovl_gs_final(lat, bd, d_pd, pc, st)) return rc;
                // u <- u - Q s  (the residual direction, orthogonal to Q in FP64)
                if (int rc = ovl_proj_update(lat, d_pd, 1, pc, st)) return rc;
            }
            std::vector<double2> Hh2(ld * ld);
            OVL_CUDA_TRY(lat, cudaMemcpyAsync(Hh2.data(), H, ld * ld * sizeof(double2), cudaMemcpyDeviceToHost, st));
            OVL_CUDA_TRY(lat, cudaStreamSynchronize(st));
            Mat Hp(pc, pc);
            for (int j = 0; j < pc; j++)
                for (int i = 0; i < pc; i++) Hp(i, j) = cd(Hh2[i + j * ld].x, Hh2[i + j * ld].y);
            if (single) {
                Hsingle = Hp;
                return OVL_OK;
            }
            // residual norm beta = |u| after the correction
            Mat nn;
            std::vector<double2*> xs{u};
            if (int rc = dots_many(qhi, qlo, 0, xs, nn)) return rc;
            double beta = sqrt(std::max(0.0, nn(0, 0).real()));
            // Schur form, wanted first: the nev smallest Re(theta) of B, or the
            // nev largest Re(theta) of the filtered operator C
            const bool filt = cheb_deg > 0;
            Mat T, Z;
            if (!sla::schur(Hp, T, Z)) return ovl_fail(lat, OVL_ENOCONV, "deflation setup: small Schur failed");
            std::vector<int> idx(pc);
            for (int i = 0; i < pc; i++) idx[i] = i;
            std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) {
                return filt ? T(a, a).real() > T(b, b).real() : T(a, a).real() < T(b, b).real();
            });
            int nw = std::min(nev, pc);
            std::vector<char> want(pc, 0);
            for (int i = 0; i < nw; i++) want[idx[i]] = 1;
            double amax = 0.0;
            for (int i = 0; i < pc; i++) amax = std::max(amax, std::abs(T(i, i)));
            std::vector<double> re_sorted(pc);
            for (int i = 0; i < pc; i++) re_sorted[i] = T(idx[i], idx[i]).real();
            sla::reorder_schur(T, Z, want);
            bnorm = std::max(bnorm, amax);
            // coupling row b = beta * (last row of Z); converged leading block.
            // B: |b_i| <= tol |B|; C: |b_i| <= tol |theta_i| (the wanted values of C
            // span many orders of magnitude, the unwanted ones are at most 1)
            Mat brow(1, pc);
            for (int j = 0; j < pc; j++) brow(0, j) = beta * Z(pc - 1, j);
            int nconv = 0;
            for (int i = 0; i < nw; i++) {
                if (std::abs(brow(0, i)) <= tol * (filt ? std::abs(T(i, i)) : bnorm))
                    nconv++;
                else
                    break;
            }
            bool done = nconv >= nw || pc < p;  // pc < p: exact invariant subspace
            if (!done && !filt && poly != 0 && power == 2 && choose_filter(re_sorted, amax)) {
                // switch to C: the Krylov-Schur relation of B does not hold for C,
                // so restart explicitly from the sum of the wanted Schur vectors
                Mat Zs(pc, 1);
                for (int r = 0; r < pc; r++) {
                    cd s = 0.0;
                    for (int i = 0; i < nw; i++) s += Z(r, i);
                    Zs(r, 0) = s;
                }
                std::vector<double2*> yu{u};
                if (int rc = combine(cur_hi, cur_lo, pc, Zs, 1, yu)) return rc;
                q = 0;
                Tq = Mat();
                bq = Mat();
                bnorm = 0.0;
                first = true;
                continue;
            }
            int qn = done ? nw : std::min(p - 2, nw + std::max((p - nw) / 3, nconv));
            if (qn < 1) qn = 1;
            // new basis columns V Z[:, 0:qn] and the start vector u/beta
            std::vector<double2*> ys(qn);
            // stage FP64 combinations in Vf/Wf (up to nev) and w/tmp chunks
            for (int c0 = 0; c0 < qn; c0 += nev) {
                int cn = std::min(nev, qn - c0);
                Mat Zc(pc, cn);
                for (int i = 0; i < cn; i++)
                    for (int r = 0; r < pc; r++) Zc(r, i) = Z(r, c0 + i);
                std::vector<double2*> yy(cn);
                for (int i = 0; i < cn; i++) yy[i] = Vf + N * i;
                if (int rc = combine(cur_hi, cur_lo, pc, Zc, cn, yy)) return rc;
                for (int i = 0; i < cn; i++) {
                    k_split_scale<<<nblk(lat, N), 256, 0, st>>>(Vf + N * i, 1.0, nxt_hi + N * (c0 + i),
                                                               nxt_lo + N * (c0 + i), N);
                    OVL_LAUNCH_CHECK(lat);
                }
            }
            if (done) {
                std::swap(cur_hi, nxt_hi);
                std::swap(cur_lo, nxt_lo);
                q = qn;
                break;
            }
            if (!(beta > 0.0)) return ovl_fail(lat, OVL_ENOCONV, "deflation setup: zero residual before convergence");
            k_split_scale<<<nblk(lat, N), 256, 0, st>>>(u, 1.0 / beta, nxt_hi + N * qn, nxt_lo + N * qn, N);
            OVL_LAUNCH_CHECK(lat);
            // u for the next expansion = the stored start vector (48-bit value)
            k_join<<<nblk(lat, N), 256, 0, st>>>(nxt_hi + N * qn, nxt_lo + N * qn, u, N);
            OVL_LAUNCH_CHECK(lat);
            Tq = Mat(qn, qn);
            for (int j = 0; j < qn; j++)
                for (int i = 0; i < qn; i++) Tq(i, j) = T(i, j);
            bq = Mat(1, qn);
            for (int j = 0; j < qn; j++) bq(0, j) = brow(0, j);
            std::swap(cur_hi, nxt_hi);
            std::swap(cur_lo, nxt_lo);
            q = qn;
        }
        if (restarts > max_restarts)
            return ovl_fail(lat, OVL_ENOCONV, "deflation setup: not converged after %d restarts", max_restarts);
        // FP64 copies of the nev converged Schur vectors of B
        for (int i = 0; i < nev; i++) {
            k_join<<<nblk(lat, N), 256, 0, st>>>(cur_hi + N * i, cur_lo + N * i, Vf + N * i, N);
            OVL_LAUNCH_CHECK(lat);
        }
        fin_hi = cur_hi;
        fin_lo = cur_lo;
        return cudaStreamSynchronize(st) == cudaSuccess ? OVL_OK : ovl_fail(lat, OVL_ECUDA, "sync failed");
    }
    float2 *fin_hi = nullptr, *fin_lo = nullptr;

    // Rayleigh-Ritz of A on span(Vf): G = V^dag V, M = V^dag A V; eigenpairs of G^-1 M.
    int ritz(int m, EigResult& R, Mat& Gm, Mat& Mm) {
        // W = A V (one stencil per vector)
        for (int i = 0; i < nev; i++) {
            void* hp[2] = {Vf + N * i, Wf + N * i};
            OVL_CUDA_TRY(lat, cudaMemcpyAsync(dsl + 4, hp, sizeof hp, cudaMemcpyHostToDevice, st));
            DslashArgs a;
            a.in = (const void* const*)(dsl + 4);
            a.out = (void* const*)(dsl + 5);
            a.mu = d_mu;
            a.nrhs = 1;
            a.kappa = kappa;
            if (int rc = ovl_dslash_launch(lat, a, OVL_VEC_F64, OVL_LINKS_F64, st)) return rc;
            OVL_CUDA_TRY(lat, cudaStreamSynchronize(st));
        }
        std::vector<const float2*> h(nev), l(nev);
        for (int c = 0; c < nev; c++) {
            h[c] = fin_hi + N * c;
            l[c] = fin_lo + N * c;
        }
        OVL_CUDA_TRY(lat, cudaMemcpyAsync(qhi, h.data(), nev * sizeof(void*), cudaMemcpyHostToDevice, st));
        OVL_CUDA_TRY(lat, cudaMemcpyAsync(qlo, l.data(), nev * sizeof(void*), cudaMemcpyHostToDevice, st));
        std::vector<double2*> vx(nev), wx(nev);
        for (int i = 0; i < nev; i++) {
            vx[i] = Vf + N * i;
            wx[i] = Wf + N * i;
        }
        Mat Gx, Mx;
        if (int rc = dots_many(qhi, qlo, nev, vx, Gx)) return rc;
        if (int rc = dots_many(qhi, qlo, nev, wx, Mx)) return rc;
        Gm = Mat(nev, nev);
        Mm = Mat(nev, nev);
        for (int j = 0; j < nev; j++)
            for (int i = 0; i < nev; i++) {
                Gm(i, j) = Gx(i, j);
                Mm(i, j) = Mx(i, j);
            }
        // K = G^-1 M via Cholesky
        Mat L;
        if (!sla::cholesky(Gm, L)) return ovl_fail(lat, OVL_ENOCONV, "deflation setup: basis Gram not SPD");
        Mat Li = sla::lower_inv(L);
        Mat K = sla::mul(sla::adj(Li), sla::mul(Li, Mm));  // G^-1 = L^-dag L^-1
        Mat T, Z;
        if (!sla::schur(K, T, Z)) return ovl_fail(lat, OVL_ENOCONV, "deflation setup: Ritz Schur failed");
        Mat X = sla::tri_eigvecs(T);
        Mat Y = sla::mul(Z, X);  // eigenvectors of K
        std::vector<int> idx(nev);
        for (int i = 0; i < nev; i++) idx[i] = i;
        std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) {
            double ra = std::abs(T(a, a).real()), rb = std::abs(T(b, b).real());
            if (ra != rb) return ra < rb;
            return std::abs(T(a, a).imag()) < std::abs(T(b, b).imag());
        });
        R.lam.resize(m);
        R.Ccoef = Mat(nev, m);
        for (int k = 0; k < m; k++) {
            int c = idx[k];
            R.lam[k] = T(c, c);
            // normalise |V y| = 1 with the Gram matrix
            double nr = 0.0;
            Mat y(nev, 1);
            for (int i = 0; i < nev; i++) y(i, 0) = Y(i, c);
            Mat Gy = sla::mul(Gm, y);
            for (int i = 0; i < nev; i++) nr += (std::conj(y(i, 0)) * Gy(i, 0)).real();
            nr = sqrt(nr);
            for (int i = 0; i < nev; i++) R.Ccoef(i, k) = y(i, 0) / nr;
        }
        return OVL_OK;
    }
};

}  // namespace

extern "C" int ovl_deflation_setup(ovl_lattice lat, double mu, double m_w, int scheme, int m, double tol,
                                   int max_restarts, ovl_deflation* out) {
    return ovl_deflation_setup_ex(lat, mu, m_w, scheme, m, tol, max_restarts, -1, out);
}

extern "C" int ovl_deflation_setup_ex(ovl_lattice lat, double mu, double m_w, int scheme, int m, double tol,
                                      int max_restarts, int poly_degree, ovl_deflation* out) {
    if (!lat || !out) return ovl_fail(lat, OVL_EINVAL, "ovl_deflation_setup: null argument");
    if (!lat->have_links) return ovl_fail(lat, OVL_EINVAL, "ovl_deflation_setup: links not set");
    if (scheme != OVL_DEFL_SCHUR && scheme != OVL_DEFL_LR)
        return ovl_fail(lat, OVL_EINVAL, "ovl_deflation_setup: scheme %d", scheme);
    if (!(m_w > -4.0 + 1e-12) || !(mu == mu)) return ovl_fail(lat, OVL_EINVAL, "ovl_deflation_setup: bad mu/m_w");
    if (m < 1 || m > 200) return ovl_fail(lat, OVL_EINVAL, "ovl_deflation_setup: m=%d out of [1,200]", m);
    if (!(tol > 0.0)) tol = 1e-12;
    if (max_restarts <= 0) max_restarts = 1000;
    const size_t N = lat->N;
    int nev = m + std::max(8, m / 2);
    int p = std::max(4 * nev, nev + 60);
    if ((size_t)p + 2 > N) {
        p = (int)N - 2;
        nev = std::min(nev, p / 2);
    }
    if (p > OVL_MAXCOL - 1) p = OVL_MAXCOL - 1;
    if (nev < m) return ovl_fail(lat, OVL_EINVAL, "ovl_deflation_setup: lattice too small for m=%d", m);
    // at mu = 0, H_w is Hermitian (H_w(mu)^dag = H_w(-mu)): left = right vectors
    const bool hermitian = (mu == 0.0);
    int runs = (scheme == OVL_DEFL_LR && !hermitian) ? 2 : 1;
    EigResult res[2];
    Mat Gm[2], Mm[2];
    Solver* sv[2] = {nullptr, nullptr};
    int rc = OVL_OK;
    for (int r = 0; r < runs && !rc; r++) {
        sv[r] = new Solver(lat, r == 0 ? mu : -mu, m_w, p, nev);
        sv[r]->poly = poly_degree < 0 ? -1 : poly_degree;
        rc = sv[r]->run(tol, max_restarts, 0x9e3779b97f4a7c15ull + r);
        if (!rc) rc = sv[r]->ritz(m, res[r], Gm[r], Mm[r]);
    }
    ovl_deflation d = nullptr;
    if (!rc) {
        d = new ovl_deflation_s();
        d->lat = lat;
        d->scheme = scheme;
        d->m = m;
        d->mu = mu;
        d->m_w = m_w;
        cudaStream_t st = lat->stream;
        if (cudaMalloc(&d->S_hi, N * m * sizeof(float2)) != cudaSuccess ||
            cudaMalloc(&d->S_lo, N * m * sizeof(float2)) != cudaSuccess)
            rc = ovl_fail(lat, OVL_ENOMEM, "deflation setup: allocation failed");
        Solver& s0 = *sv[0];
        if (!rc && scheme == OVL_DEFL_SCHUR) {
            // orthonormal basis of span(R) with upper triangular T (Eq. 13):
            // C = Y L^-dag Z where Y^dag G Y = L L^dag and T0 = L^-1 Y^dag M Y L^-dag = Z T Z^dag
            Mat Y = res[0].Ccoef;
            Mat GY = sla::mul(sla::adj(Y), sla::mul(Gm[0], Y));
            Mat MY = sla::mul(sla::adj(Y), sla::mul(Mm[0], Y));
            Mat L;
            if (!sla::cholesky(GY, L)) rc = ovl_fail(lat, OVL_ENOCONV, "deflation setup: eigenvectors dependent");
            if (!rc) {
                Mat Li = sla::lower_inv(L);
                Mat T0 = sla::mul(Li, sla::mul(MY, sla::adj(Li)));
                Mat T, Z;
                if (!sla::schur(T0, T, Z)) rc = ovl_fail(lat, OVL_ENOCONV, "deflation setup: Schur of T failed");
                if (!rc) {
                    Mat C = sla::mul(Y, sla::mul(sla::adj(Li), Z));
                    std::vector<double2*> ys(m);
                    // stage in the solver's W buffer (nev >= m vectors)
                    for (int i = 0; i < m; i++) ys[i] = s0.Wf + N * i;
                    rc = s0.combine(s0.fin_hi, s0.fin_lo, s0.nev, C, m, ys);
                    for (int i = 0; i < m && !rc; i++)
                        k_split_scale<<<nblk(lat, N), 256, 0, st>>>(ys[i], 1.0, d->S_hi + N * i, d->S_lo + N * i, N);
                    d->T_host.assign(2 * (size_t)m * m, 0.0);
                    for (int j = 0; j < m; j++)
                        for (int i = 0; i < m; i++) {
                            d->T_host[2 * (i + (size_t)j * m)] = i <= j ? T(i, j).real() : 0.0;
                            d->T_host[2 * (i + (size_t)j * m) + 1] = i <= j ? T(i, j).imag() : 0.0;
                        }
                }
            }
        } else if (!rc) {
            // right vectors R, eigenvalues, and left vectors from A^dag = H_w(-mu)
            if (hermitian) {
                sv[1] = sv[0];
                res[1] = res[0];
            }
            Solver& s1 = *sv[1];
            if (cudaMalloc(&d->L_hi, N * m * sizeof(float2)) != cudaSuccess ||
                cudaMalloc(&d->L_lo, N * m * sizeof(float2)) != cudaSuccess)
                rc = ovl_fail(lat, OVL_ENOMEM, "deflation setup: allocation failed");
            // pair left eigenvalue conj(lambda_i) with right lambda_i (nearest)
            std::vector<int> pairing(m, -1);
            std::vector<char> taken(m, 0);
            for (int i = 0; i < m && !rc; i++) {
                double best = 1e300;
                int bj = -1;
                for (int j = 0; j < m; j++) {
                    if (taken[j]) continue;
                    double dd = std::abs(std::conj(res[1].lam[j]) - res[0].lam[i]);
                    if (dd < best) {
                        best = dd;
                        bj = j;
                    }
                }
                if (bj < 0 || best > 1e-6 * (1.0 + std::abs(res[0].lam[i])))
                    rc = ovl_fail(lat, OVL_ENOCONV, "deflation setup: no left eigenvalue matches lambda_%d", i);
                else {
                    pairing[i] = bj;
                    taken[bj] = 1;
                }
            }
            if (!rc) {
                std::vector<double2*> rr(m), ll(m);
                for (int i = 0; i < m; i++) {
                    rr[i] = s0.Wf + N * i;
                    ll[i] = (hermitian ? s1.Vf : s1.Wf) + N * i;  // no aliasing when s1 == s0
                }
                Mat CL(nev, m);
                for (int i = 0; i < m; i++)
                    for (int c = 0; c < nev; c++) CL(c, i) = res[1].Ccoef(c, pairing[i]);
                rc = s0.combine(s0.fin_hi, s0.fin_lo, s0.nev, res[0].Ccoef, m, rr);
                if (!rc) rc = s1.combine(s1.fin_hi, s1.fin_lo, s1.nev, CL, m, ll);
                // l_i^dag r_i: split r into planes first, then project each l_i on them
                for (int i = 0; i < m && !rc; i++)
                    k_split_scale<<<nblk(lat, N), 256, 0, st>>>(rr[i], 1.0, d->S_hi + N * i, d->S_lo + N * i, N);
                if (!rc) {
                    std::vector<const float2*> h(m), l(m);
                    for (int c = 0; c < m; c++) {
                        h[c] = d->S_hi + N * c;
                        l[c] = d->S_lo + N * c;
                    }
                    cudaMemcpyAsync(s1.qhi, h.data(), m * sizeof(void*), cudaMemcpyHostToDevice, st);
                    cudaMemcpyAsync(s1.qlo, l.data(), m * sizeof(void*), cudaMemcpyHostToDevice, st);
                    Mat RL;  // RL(c, i) = r_c^dag l_i
                    rc = s1.dots_many(s1.qhi, s1.qlo, m, ll, RL);
                    for (int i = 0; i < m && !rc; i++) {
                        cd lr = std::conj(RL(i, i));  // l_i^dag r_i
                        // l_i <- l_i / conj(l_i^dag r_i)  so that l_i^dag r_i = 1
                        cd sc = 1.0 / std::conj(lr);
                        // scale in FP64 then split (complex scale: do it on the host coefficients instead)
                        Mat c1(nev, 1);
                        for (int c = 0; c < nev; c++) c1(c, 0) = CL(c, i) * sc;
                        std::vector<double2*> one{ll[i]};
                        rc = s1.combine(s1.fin_hi, s1.fin_lo, s1.nev, c1, 1, one);
                        if (!rc)
                            k_split_scale<<<nblk(lat, N), 256, 0, st>>>(ll[i], 1.0, d->L_hi + N * i, d->L_lo + N * i,
                                                                       N);
                    }
                }
            }
            if (!rc) {
                d->T_host.assign(2 * (size_t)m, 0.0);
                for (int i = 0; i < m; i++) {
                    d->T_host[2 * i] = res[0].lam[i].real();
                    d->T_host[2 * i + 1] = res[0].lam[i].imag();
                }
            }
        }
        if (!rc) {
            size_t tb = d->T_host.size() * sizeof(double);
            if (cudaMalloc(&d->T, tb) != cudaSuccess ||
                cudaMemcpy(d->T, d->T_host.data(), tb, cudaMemcpyHostToDevice) != cudaSuccess)
                rc = ovl_fail(lat, OVL_ENOMEM, "deflation setup: T allocation failed");
        }
        if (!rc && cudaStreamSynchronize(st) != cudaSuccess) rc = ovl_fail(lat, OVL_ECUDA, "deflation setup: sync");
    }
    if (sv[1] == sv[0]) sv[1] = nullptr;  // Hermitian case shared one run
    if (d && !rc) {
        d->setup_restarts = sv[0]->restarts + (sv[1] ? sv[1]->restarts : 0);
        d->setup_matvecs = sv[0]->matvecs + (sv[1] ? sv[1]->matvecs : 0);
    }
    delete sv[0];
    delete sv[1];
    if (rc) {
        if (d) ovl_destroy_deflation(d);
        return rc;
    }
    *out = d;
    return OVL_OK;
}

// ---------------------------------------------------------------------------
// features of the (k, m) predictor
// ---------------------------------------------------------------------------
namespace {
__global__ void k_link_spread(const double2* __restrict__ u64, size_t V, double* __restrict__ part) {
    __shared__ double red[256];
    double acc = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < 4 * V; i += (size_t)gridDim.x * blockDim.x) {
        size_t nu = i / V, site = i - nu * V;
        double tr = u64[(nu * 9 + 0) * V + site].x + u64[(nu * 9 + 4) * V + site].x + u64[(nu * 9 + 8) * V + site].x;
        acc += 1.0 - tr / 3.0;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}
}  // namespace

extern "C" int ovl_link_spread(ovl_lattice lat, double* spread) {
    if (!lat || !spread) return ovl_fail(lat, OVL_EINVAL, "ovl_link_spread: null argument");
    if (!lat->have_links) return ovl_fail(lat, OVL_EINVAL, "ovl_link_spread: links not set");
    const int nb = 256;
    void* s;
    if (int rc = ovl_scratch(lat, nb * sizeof(double), &s)) return rc;
    k_link_spread<<<nb, 256, 0, lat->stream>>>(lat->links.u64, lat->V, (double*)s);
    OVL_LAUNCH_CHECK(lat);
    std::vector<double> h(nb);
    OVL_CUDA_TRY(lat, cudaMemcpyAsync(h.data(), s, nb * sizeof(double), cudaMemcpyDeviceToHost, lat->stream));
    OVL_CUDA_TRY(lat, cudaStreamSynchronize(lat->stream));
    double t = 0.0;
    for (double v : h) t += v;
    *spread = t / (4.0 * (double)lat->V);
    return OVL_OK;
}

extern "C" int ovl_ritz_values(ovl_lattice lat, double mu, double m_w, int k, const double* b, double* out) {
    if (!lat || !b || !out) return ovl_fail(lat, OVL_EINVAL, "ovl_ritz_values: null argument");
    if (!lat->have_links) return ovl_fail(lat, OVL_EINVAL, "ovl_ritz_values: links not set");
    if (k < 1 || (size_t)k + 2 > lat->N || k > OVL_MAXCOL - 2)
        return ovl_fail(lat, OVL_EINVAL, "ovl_ritz_values: k=%d out of range", k);
    Solver sv(lat, mu, m_w, k, 1);
    sv.power = 1;
    sv.single = true;
    if (int rc = sv.alloc()) return rc;
    // b (canonical, host or device) -> packed FP64 in u
    size_t cb = lat->N * sizeof(double2);
    const double* src = b;
    void* s;
    if (int rc = ovl_scratch(lat, cb, &s)) return rc;
    if (!ovl_is_device_ptr(b)) {
        OVL_CUDA_TRY(lat, cudaMemcpyAsync(s, b, cb, cudaMemcpyHostToDevice, lat->stream));
        src = (const double*)s;
    }
    if (int rc = ovl_pack_impl(lat, src, sv.u, 1, OVL_VEC_F64, lat->stream)) return rc;
    sv.start_given = true;
    if (int rc = sv.run(1e-12, 0, 0)) return rc;
    Mat T, Z;
    if (!sla::schur(sv.Hsingle, T, Z)) return ovl_fail(lat, OVL_ENOCONV, "ovl_ritz_values: small Schur failed");
    int n = T.r;
    for (int i = 0; i < k; i++) {
        cd v = i < n ? T(i, i) : cd(0.0);
        out[2 * i] = v.real();
        out[2 * i + 1] = v.imag();
    }
    return OVL_OK;
}
