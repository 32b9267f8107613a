// Scaled Newton iteration for the sign of the small projected matrix.
#pragma once
#include "ovl_common.cuh"

#define OVL_NEWTON_MAXN 960

struct NewtonDev {
    const double2* H;  // input, column-major, leading dimension ldH
    int ldH;
    int n;             // matrix order (0 < n <= OVL_NEWTON_MAXN)
    int run;           // 0: skip this solve
    int max_iter;
    double tol;
    double2* X;        // n x n row-major: iterate, and sgn(H) on exit
    double2* W;        // n x n row-major work (inverse in place)
    double* cand_val;  // 2 x CTAs of the group (step parity)
    int* cand_row;
    double* red;       // 2 per CTA of the group
    unsigned* bar;     // group barrier counter (zero before launch)
    int* status;       // OVL_* (zero before launch)
    int* iters;
    const double2* cvec;  // coefficient vector (n) for F c
    double2* gout;        // F c (n)
    int df;               // 1: X holds double-float values (float4 hi.re, hi.im, lo.re, lo.im)
    float4* crow;         // df kernel: published candidate rows, 2 x CTAs x n
    float4* Wg;           // df kernel: work rows in global memory when they do not fit in shared memory
    // hand-off to Newton-Schulz (double-float kernels): with ns_switch > 0 the
    // Gauss-Jordan iteration stops once its relative step is below ns_switch
    // and sets *handoff; resume = 1 restarts it from the iterate already in X
    // (unscaled), as after a failed Newton-Schulz attempt
    double ns_switch;
    int resume;
    int* handoff;
};

// Newton-Schulz finish of the sign iteration (double-float): once the scaled
// Newton iterate X is close to an involution, X <- X (3 I - X^2) / 2 converges
// quadratically with matrix products only (Higham, Functions of Matrices,
// 2008, Sec. 5.3); it is used while |I - X^2|_F < 1/2, which guarantees
// convergence. One batched complex double-float GEMM kernel computes X^2,
// another X Y with the update in its epilogue.
struct NsDev {
    float4* X;     // iterate buffer 0 (the Newton X); sgn(H) here on exit
    float4* W;     // iterate buffer 1
    float4* Y;     // X^2
    double* acc;   // per 64 x 64 tile (tiles^2 each): |I - X^2|_F^2, |X_new - X|_F^2, |X_new|_F^2
    int n;
    int on;        // iterating
    int cur;       // the iterate is in X (0) or W (1)
    int done;      // converged
    int fallback;  // left the convergence region: back to Gauss-Jordan
    int iters;
    double tol;
    double prev;   // previous relative step
    double region; // |I - X^2|_F^2 bound for a step (1/4; 0 declines every step)
};
#define OVL_NS_ACC (3 * ((OVL_NEWTON_MAXN + 63) / 64) * ((OVL_NEWTON_MAXN + 63) / 64))  // doubles in NsDev::acc
int ovl_newton_schulz(ovl_lattice lat, NsDev* d_ns, NsDev* h_ns, int nsolve, int nmax, int max_iter,
                      cudaStream_t st);

int ovl_newton_cpm(ovl_lattice lat, int nsolve, int nmax);
int ovl_newton_launch(ovl_lattice lat, NewtonDev* nd_dev, int nsolve, int cpm, cudaStream_t st);
// double-float Gauss-Jordan Newton (rows in shared memory when they fit)
int ovl_newton_df_plan(ovl_lattice lat, int nsolve, int nmax, int* cpm, int* smem_rows);
int ovl_newton_df_launch(ovl_lattice lat, NewtonDev* nd_dev, int nsolve, int nmax, int cpm, int smem_rows,
                         cudaStream_t st);
// double-float Gauss-Jordan Newton, one thread-block cluster per matrix (rows in
// the CTAs' shared memory, the rest of a CTA's rows in its part of Wg);
// cl_size 0 when no cluster shape fits n
int ovl_newton_cl_plan(ovl_lattice lat, int nsolve, int nmax, int* cl_size, size_t* smem, int* nrs, int* l2rows);
int ovl_newton_cl_launch(ovl_lattice lat, NewtonDev* nd_dev, int nsolve, int cl_size, size_t smem, int nrs,
                         int l2rows, cudaStream_t st);
int ovl_fmatvec_launch(ovl_lattice lat, NewtonDev* nd_dev, int nsolve, int nmax, cudaStream_t st);
