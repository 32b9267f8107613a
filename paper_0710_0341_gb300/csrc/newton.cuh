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
};

int ovl_newton_cpm(ovl_lattice lat, int nsolve, int nmax);
int ovl_newton_launch(ovl_lattice lat, NewtonDev* nd_dev, int nsolve, int cpm, cudaStream_t st);
// double-float Gauss-Jordan Newton (rows in shared memory when they fit)
int ovl_newton_df_plan(ovl_lattice lat, int nsolve, int nmax, int* cpm, int* smem_rows);
int ovl_newton_df_launch(ovl_lattice lat, NewtonDev* nd_dev, int nsolve, int nmax, int cpm, int smem_rows,
                         cudaStream_t st);
// double-float Gauss-Jordan Newton, one thread-block cluster per matrix (rows in
// the cluster's shared memory); cl_size 0 when no cluster shape fits n
int ovl_newton_cl_plan(ovl_lattice lat, int nmax, int* cl_size, size_t* smem);
int ovl_newton_cl_launch(ovl_lattice lat, NewtonDev* nd_dev, int nsolve, int cl_size, size_t smem, cudaStream_t st);
int ovl_fmatvec_launch(ovl_lattice lat, NewtonDev* nd_dev, int nsolve, int nmax, cudaStream_t st);
