// The Sylvester route of the Schur deflation (Sec. 3, Eqs. 18-19).
//
// With the block matrix H = [[T, X], [0, H_k]] of Eq. 15 (T = T_m upper
// triangular, X = S^dag A V_k, H_k upper Hessenberg), f(H) = [[f(T), Y],
// [0, f(H_k)]] where the coupling block Y solves the Sylvester equation
//     T Y - Y H_k = f(T) X - X f(H_k)                              (Eq. 18)
// and the approximation is y = S (f(T) S^dag b + beta Y e_1) + beta V_k f(H_k) e_1
// (Eq. 19). The sign of the two diagonal blocks comes from the library's
// Newton kernels (on the m x m and k x k blocks instead of the whole
// (m + k) x (m + k) matrix); this file forms the right-hand side and solves
// for Y, all in FP64:
//   k_syl_rhs   R = f(T) X - X f(H_k)                    one CTA per row of R
//   k_syl_rows  T upper triangular, so row i of Eq. 18 reads
//               Y_i (t_ii I - H_k) = R_i - sum_{l > i} t_il Y_l,
//               solved for i = m-1, ..., 0 (one CTA per solve): the
//               transposed matrix t_ii I - H_k^T is lower Hessenberg; the
//               superdiagonal is eliminated from the last column backwards
//               with row pivoting (one two-row update per column), and the
//               lower triangular system by column-oriented forward
//               substitution
//   k_syl_coef  g_S = f(T) S^dag b (from the Newton run on T) + beta Y e_1
#include "krylov.cuh"
#include "sylvester.cuh"

namespace {

__device__ __forceinline__ double2 ld_f(const SylDev& d, const void* F, int ldf, int i, int j) {
    // F row-major with leading dimension ldf: double-float (float4) or complex128
    if (d.df) {
        const float4 v = ((const float4*)F)[(size_t)i * ldf + j];
        return make_double2((double)v.x + (double)v.z, (double)v.y + (double)v.w);
    }
    return ((const double2*)F)[(size_t)i * ldf + j];
}

__global__ void __launch_bounds__(256) k_syl_rhs(const SylDev* sds) {
    const SylDev& d = sds[blockIdx.y];
    if (!d.on) return;
    const int i = blockIdx.x, m = d.m, k = d.k;
    if (i >= m) return;
    const int ld = d.ldH;
    const double2* H = d.H;
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        double2 acc = make_double2(0.0, 0.0);
        for (int l = 0; l < m; l++)  // f(T) X
            acc = cadd(acc, cmul(ld_f(d, d.FT, m, i, l), H[l + (size_t)(m + j) * ld]));
        for (int l = 0; l < k; l++)  // - X f(H_k)
            acc = csub(acc, cmul(H[i + (size_t)(m + l) * ld], ld_f(d, d.FH, k, l, j)));
        d.R[(size_t)i * k + j] = acc;
    }
}

constexpr int SYL_THREADS = 1024;

__device__ __forceinline__ double cabs1(double2 a) { return fabs(a.x) + fabs(a.y); }
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) { return cmul(a, cinv(b)); }

__global__ void __launch_bounds__(SYL_THREADS) k_syl_rows(const SylDev* sds) {
    const SylDev& d = sds[blockIdx.x];
    if (!d.on) return;
    const int m = d.m, k = d.k, ld = d.ldH;
    const double2* H = d.H;
    double2* A = d.W;  // k x k row-major work: (t I - H_k)^T
    double2* r = d.r;  // right-hand side, then the solution
    __shared__ double2 s_f;
    __shared__ int s_swap;
    for (int i = m - 1; i >= 0; i--) {
        const double2 t = H[i + (size_t)i * ld];
        // A[a][b] = t delta_ab - H_k[b][a]; r = R_i - sum_{l > i} t_il Y_l
        for (size_t e = threadIdx.x; e < (size_t)k * k; e += blockDim.x) {
            const int a = (int)(e / k), b = (int)(e % k);
            double2 v = b <= a + 1 ? H[(m + b) + (size_t)(m + a) * ld] : make_double2(0.0, 0.0);
            v = make_double2(-v.x, -v.y);
            if (a == b) v = cadd(v, t);
            A[e] = v;
        }
        for (int j = threadIdx.x; j < k; j += blockDim.x) {
            double2 v = d.R[(size_t)i * k + j];
            for (int l = i + 1; l < m; l++) v = csub(v, cmul(H[i + (size_t)l * ld], d.Y[(size_t)l * k + j]));
            r[j] = v;
        }
        __syncthreads();
        // eliminate the superdiagonal A[c-1][c], c = k-1 .. 1 (rows c-1 and c hold columns <= c)
        for (int c = k - 1; c >= 1; c--) {
            if (threadIdx.x == 0) {
                const double2 up = A[(size_t)(c - 1) * k + c], dg = A[(size_t)c * k + c];
                const int sw = cabs1(up) > cabs1(dg);
                s_swap = sw;
                const double2 piv = sw ? up : dg, oth = sw ? dg : up;
                s_f = cabs1(piv) > 0.0 ? cdiv(oth, piv) : make_double2(0.0, 0.0);
            }
            __syncthreads();
            const int sw = s_swap;
            const double2 f = s_f;
            double2* rc = A + (size_t)c * k;
            double2* rp = A + (size_t)(c - 1) * k;
            for (int b = threadIdx.x; b <= c; b += blockDim.x) {
                const double2 vc = rc[b], vp = rp[b];
                // pivot row (the larger entry in column c) stays at index c, the other
                // row minus f times it goes to index c - 1
                const double2 piv = sw ? vp : vc, oth = sw ? vc : vp;
                rc[b] = piv;
                rp[b] = csub(oth, cmul(f, piv));
            }
            if (threadIdx.x == 0) {
                const double2 pv = sw ? r[c - 1] : r[c], ot = sw ? r[c] : r[c - 1];
                r[c] = pv;
                r[c - 1] = csub(ot, cmul(f, pv));
            }
            __syncthreads();
        }
        // lower triangular solve, column-oriented: y_j = r_j / A_jj; r_l -= A_lj y_j (l > j)
        for (int j = 0; j < k; j++) {
            const double2 y = cdiv(r[j], A[(size_t)j * k + j]);
            for (int l = j + 1 + threadIdx.x; l < k; l += blockDim.x) r[l] = csub(r[l], cmul(A[(size_t)l * k + j], y));
            __syncthreads();
            if (threadIdx.x == 0) d.Y[(size_t)i * k + j] = y;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256) k_syl_coef(const SylDev* sds) {
    const SylDev& d = sds[blockIdx.x];
    if (!d.on) return;
    for (int i = threadIdx.x; i < d.m; i += blockDim.x)
        d.gS[i] = cadd(d.gT[i], cscale(d.Y[(size_t)i * d.k], d.beta));
}

}  // namespace

int ovl_sylvester_launch(ovl_lattice lat, const SylDev* d_sd, int nsolve, int mmax, cudaStream_t st) {
    k_syl_rhs<<<dim3(mmax, nsolve), 256, 0, st>>>(d_sd);
    OVL_LAUNCH_CHECK(lat);
    k_syl_rows<<<nsolve, SYL_THREADS, 0, st>>>(d_sd);
    OVL_LAUNCH_CHECK(lat);
    k_syl_coef<<<nsolve, 256, 0, st>>>(d_sd);
    OVL_LAUNCH_CHECK(lat);
    return OVL_OK;
}
