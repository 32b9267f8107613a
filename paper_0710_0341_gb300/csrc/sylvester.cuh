// The Sylvester route of the Schur deflation (Sec. 3, Eqs. 18-19): device
// descriptor and launcher (sylvester.cu).
#pragma once
#include "ovl_common.cuh"

struct SylDev {
    const double2* H;  // block matrix of Eq. 15, column-major, leading dimension ldH
    int ldH;
    int m, k;          // orders of T and H_k
    int on;            // 0: skip this solve
    int df;            // FT, FH hold double-float values (float4) instead of complex128
    const void* FT;    // sgn(T), m x m row-major (from the Newton kernels)
    const void* FH;    // sgn(H_k), k x k row-major
    double2* R;        // m x k row-major: right-hand side of Eq. 18
    double2* Y;        // m x k row-major: the coupling block
    double2* W;        // k x k work
    double2* r;        // k work
    const double2* gT; // sgn(T) S^dag b
    double2* gS;       // out: sgn(T) S^dag b + beta Y e_1 (the S part of Eq. 19's coefficients)
    double beta;       // |x_perp|
};

// R, Y and gS for nsolve solves (mmax = the largest m among the solves switched on)
int ovl_sylvester_launch(ovl_lattice lat, const SylDev* d_sd, int nsolve, int mmax, cudaStream_t st);
