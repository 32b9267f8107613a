// Batched Arnoldi machinery (Sec. 2, Eq. 7; Sec. 3, Eq. 14): device-side
// descriptors shared by krylov.cu, newton.cu and sign.cu.
#pragma once
#include "ovl_common.cuh"

#define OVL_MAXCOL 960  // m + k + 1 (columns of the augmented basis) per solve
#define OVL_MAXPTR 200  // columns addressed through pointers (the Schur vectors)

// One solve of a batch. All pointers are device memory.
//
// Q = (S_m  v_1 ... v_k) is the augmented basis of Eq. 14 (m = m_q; m_q = 0
// for LR deflation and for no deflation). Column c lives at qhi[c] (FP32
// high part, packed order) and, in the FP64 mode, qlo[c] (FP32 low part);
// the two sum to a 48-bit value. H is the (m+k+1) x (m+k+1) matrix of
// Eq. 15 (column-major, leading dimension ldH): H[0:m,0:m] = T_m,
// H[0:m, m:] = S^dag A V (the X of Eq. 18), H[m:, m:] = H_k, plus the
// sub-diagonal Arnoldi residual norms. H32 is an FP32 shadow of H.
struct SolveDev {
    const float2* const* qhi;
    const float2* const* qlo;  // null in the mixed modes
    // columns c >= nptr are contiguous: vhi + (c - nptr) * N (same for vlo);
    // columns c < nptr (the Schur vectors) come from qhi/qlo
    const float2* vhi;
    const float2* vlo;
    int nptr;
    double2* u;      // Arnoldi candidate (once orthogonalised, unnormalised)
    double2* w;      // A u
    double2* H;
    float2* H32;
    double2* dots;   // pass-A results: a[0..p), b[p..2p), g_uu, g_uw, g_ww
    double2* dvec;   // d = H a  (p+1)
    float2* ap;      // pass-B coefficients a/nu            (FP32)
    float2* gh;      // pass-B coefficients g, high part    (FP32)
    float2* gl;      // pass-B coefficients g, low part     (FP32)
    double* scal;    // [0] 1/nu, [1..2] -e_p/nu (complex), [3] nu, [4] beta_k
    // plain FP64 form only (null otherwise): the pass-B coefficients in FP64,
    // a/nu in ap64[0..p) and g in g64[0..p); the basis columns then hold
    // double2 values (qhi[c] and vhi point to complex128 data, qlo/vlo unused)
    double2* ap64;
    double2* g64;
    int m_q;         // leading fixed columns (Schur vectors)
    int k;           // requested Krylov depth
    int ldH;
    int active;      // cleared on breakdown or error
    int k_used;
    int status;      // OVL_* per solve
    int fin;         // final (accurate) projection of u still pending
};

struct BatchDev {
    SolveDev* sd;    // device array of nsolve descriptors
    int nsolve;
    size_t N;
    double2* part;   // partial sums: nsolve x G x pstride
    int G;           // CTAs per solve of the streaming passes
    int pstride;     // >= 2*OVL_MAXCOL + 3
    int pmax;        // max over solves of the basis columns used at this step
    int df;          // FP64 mode: basis has low planes
    int f64;         // plain FP64 form: complex128 basis, FP64 products everywhere
    int lo16;        // 40-bit basis: the Krylov columns' low planes are BF16 (vlo holds
                     // __nv_bfloat162 entries); the Schur columns keep FP32 low planes
    int bulk16;      // set by the caller when every basis column (vhi, vlo and the pointer
                     // tables) starts on a 16-byte boundary and N % 4 == 0: pass B may then
                     // stream the columns with bulk copies (ovl_set_pass_b)
};

// launchers (krylov.cu)
int ovl_gs_dot(ovl_lattice lat, const BatchDev& b, int j, cudaStream_t st);
int ovl_gs_reduce(ovl_lattice lat, const BatchDev& b, int j, cudaStream_t st);
int ovl_gs_small(ovl_lattice lat, const BatchDev& b, int j, cudaStream_t st);
int ovl_gs_update(ovl_lattice lat, const BatchDev& b, int j, cudaStream_t st);
int ovl_gs_grid(ovl_lattice lat);

// Accurate (FP64) projections used once per solve for the deflation step and
// for the start vector: P[s][c] = sum_r conj(Q_s[r,c]) x_s[r] for c < ncol_s,
// plus P[s][ncol_s] = |x_s|^2.
struct ProjDev {
    const float2* const* qhi;  // column pointers (ncol entries)
    const float2* const* qlo;  // null: columns have no low plane
    double2* x;                // packed FP64 vector
    double2* out;              // ncol + 1 results
    const double2* coef;       // for the update: x -= sum_c Q[:,c] coef[c]
    int ncol;
    int f64;                   // columns are complex128 (qhi entries point to double2 data)
    int lo16_from, lo16_to;    // columns in [from, to) have BF16 low planes (empty: from = to = 0)
};
// f64: the columns are complex128 (plain FP64 form); else hi (+ lo) FP32 planes
int ovl_proj_dot(ovl_lattice lat, ProjDev* pd_dev, int nsolve, int maxcol, double2* part, int G, cudaStream_t st,
                 int f64 = 0);
int ovl_proj_update(ovl_lattice lat, ProjDev* pd_dev, int nsolve, int maxcol, cudaStream_t st, int f64 = 0);
int ovl_gs_final(ovl_lattice lat, const BatchDev& b, ProjDev* pd_dev, int maxcol, cudaStream_t st);

// y_s = sum_c Q_s[:,c] g_s[c] (df accumulation), FP64 packed output.
struct GemvDev {
    const float2* const* qhi;
    const float2* const* qlo;
    const double2* g;
    double2* y;
    int ncol;
    int f64;                   // columns are complex128 (qhi entries point to double2 data)
    int lo16_from, lo16_to;    // columns in [from, to) have BF16 low planes (empty: from = to = 0)
};
int ovl_gemv_df(ovl_lattice lat, GemvDev* gd_dev, int nsolve, int maxcol, cudaStream_t st, int f64 = 0);

// v_1 = x / beta into column m_q of Q (split hi/lo) and into u.
int ovl_start_vector(ovl_lattice lat, const BatchDev& b, const double* beta2_dev, int beta_stride,
                     cudaStream_t st);
