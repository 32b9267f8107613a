// Streaming Gram-Schmidt kernels of the Arnoldi step (Sec. 2, Eq. 7) and of
// the augmented Arnoldi step of the Schur deflation (Sec. 3, Eq. 14).
//
// Classical Gram-Schmidt with one reorthogonalisation is organised as the
// "delayed" variant: step j makes two passes over the basis Q_p (p = m + j - 1
// final columns) instead of four:
//   pass A (k_gs_dot):    a = Q_p^dag u_j,  b = Q_p^dag w    (w = A u_j)
//   small  (k_gs_small_rows; k_gs_small for the first step and the final pass):
//                         nu = sqrt(|u_j|^2 - |a|^2); q_{p+1} = (u_j - Q_p a)/nu
//                         is the reorthogonalised, normalised column; the
//                         coefficients c of A q_{p+1} on Q_{p+1} follow from
//                         a, b and d = H a without touching Q again
//   pass B (k_gs_update): q_{p+1} = u_j/nu - Q_p (a/nu)        -> column p of Q
//                         u_{j+1} = w/nu - (e_p/nu) u_j - Q_p g -> next candidate
// By construction A q_{p+1} = Q_{p+1} c + u_{j+1} holds to the accuracy of the
// pass-B arithmetic for whatever coefficients are used, so the inner products
// of pass A only need FP32 products (they steer orthogonality), while pass B
// accumulates in double-float (48 bits) against the stored hi+lo basis.
#include <algorithm>
#include <cmath>

#include <cuda_bf16.h>

#include "bulk.cuh"
#include "df.cuh"
#include "krylov.cuh"

namespace {

constexpr int DOT_THREADS = 256;
constexpr int UPD_RPL = 4;
constexpr int UPD_RB = 32 * UPD_RPL;

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_sumd(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Low planes in BF16 (the 40-bit basis): one __nv_bfloat162 (4 bytes) per
// complex entry; two consecutive rows are one 8-byte load.
__device__ __forceinline__ float4 lo16_pair(const void* base, size_t r2) {  // rows 2 r2, 2 r2 + 1
    const uint2 v = __ldg((const uint2*)base + r2);
    const float2 a = __bfloat1622float2(*(const __nv_bfloat162*)&v.x);
    const float2 b = __bfloat1622float2(*(const __nv_bfloat162*)&v.y);
    return make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ float2 lo16_one(const void* base, size_t r) {
    return __bfloat1622float2(__ldg((const __nv_bfloat162*)base + r));
}

__device__ __forceinline__ int solve_p(const SolveDev& d, int j) { return j < 0 ? d.m_q + d.k_used : d.m_q + j - 1; }
__device__ __forceinline__ bool solve_in_step(const SolveDev& d, int j) {
    if (j < 0) return d.fin != 0;
    return d.active && j <= d.k;
}

// ---------------------------------------------------------------------------
// pass A: a = Q_p^dag u, b = Q_p^dag w and the scalars |u|^2, u^dag w, |w|^2
//
// A CTA takes a block of DOTB_RB rows (u and w staged in shared memory as
// FP32) and a group of columns (c = cg + CG * (warp + 8 i)); a warp streams one
// column at a time, each lane reading 16 float4 (32 rows) of it, and reduces
// across lanes once per column and row block. Row blocks are visited in a
// grid-stride loop; each CTA keeps FP64 sums in shared memory and writes one
// partial per column. grid = (row-block slots G, solves, column groups CG).
// ---------------------------------------------------------------------------
constexpr int DOTB_RB = 1024;               // rows per block
constexpr int DOTB_FL = DOTB_RB / 64;       // float4 loads per lane per column (16)
constexpr int DOT_BATCH = 8;                // loads in flight per lane

__global__ void __launch_bounds__(DOT_THREADS) k_gs_dot(BatchDev B, int j) {
    const int s = blockIdx.y;
    const SolveDev& d = B.sd[s];
    if (!solve_in_step(d, j)) return;
    const int p = solve_p(d, j);
    const size_t N = B.N;
    const int CG = gridDim.z, cg = blockIdx.z;
    __shared__ double2 acc[2 * OVL_MAXCOL + 3];
    __shared__ const float2* s_col[OVL_MAXPTR];
    __shared__ float4 s_uw[DOTB_RB];  // (u.re, u.im, w.re, w.im) per row
    __shared__ double s_sc[DOT_THREADS / 32][4];  // per-warp |u|^2, u^dag w, |w|^2 (summed in warp order)
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nptr = d.nptr;
    for (int o = tid; o < 2 * p + 3; o += DOT_THREADS) acc[o] = make_double2(0.0, 0.0);
    if (lane == 0)
        for (int q = 0; q < 4; q++) s_sc[warp][q] = 0.0;
    for (int c = tid; c < nptr && c < p; c += DOT_THREADS) s_col[c] = d.qhi[c];
    const double2* __restrict__ u = d.u;
    const double2* __restrict__ w = d.w;
    for (size_t base = (size_t)blockIdx.x * DOTB_RB; base < N; base += (size_t)gridDim.x * DOTB_RB) {
        __syncthreads();  // s_uw reuse
        float guu = 0.f, guwr = 0.f, guwi = 0.f, gww = 0.f;
        for (int rr = tid; rr < DOTB_RB; rr += DOT_THREADS) {
            size_t r = base + rr;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (r < N) {
                double2 a = u[r], b = w[r];
                v = make_float4((float)a.x, (float)a.y, (float)b.x, (float)b.y);
            }
            s_uw[rr] = v;
            guu = fmaf(v.x, v.x, fmaf(v.y, v.y, guu));
            gww = fmaf(v.z, v.z, fmaf(v.w, v.w, gww));
            guwr = fmaf(v.x, v.z, fmaf(v.y, v.w, guwr));
            guwi = fmaf(v.x, v.w, fmaf(-v.y, v.z, guwi));
        }
        if (cg == 0) {
            guu = warp_sum(guu);
            gww = warp_sum(gww);
            guwr = warp_sum(guwr);
            guwi = warp_sum(guwi);
            if (lane == 0) {
                s_sc[warp][0] += (double)guu;
                s_sc[warp][1] += (double)guwr;
                s_sc[warp][2] += (double)guwi;
                s_sc[warp][3] += (double)gww;
            }
        }
        __syncthreads();
        const bool full = base + DOTB_RB <= N;
        for (int c = cg + CG * warp; c < p; c += CG * (DOT_THREADS / 32)) {
            const float4* __restrict__ q =
                (const float4*)(c < nptr ? s_col[c] : d.vhi + (size_t)(c - nptr) * N) + (base >> 1);
            float ar = 0.f, ai = 0.f, br = 0.f, bi = 0.f;
#pragma unroll
            for (int h = 0; h < DOTB_FL / DOT_BATCH; h++) {  // batches of loads in flight
                float4 qq[DOT_BATCH];
#pragma unroll
                for (int i = 0; i < DOT_BATCH; i++) {
                    const int rl = 64 * (h * DOT_BATCH + i) + 2 * lane;  // local row (even)
                    qq[i] = (full || base + rl < N) ? __ldg(q + (rl >> 1)) : make_float4(0.f, 0.f, 0.f, 0.f);
                }
#pragma unroll
                for (int i = 0; i < DOT_BATCH; i++) {
                    const int rl = 64 * (h * DOT_BATCH + i) + 2 * lane;
                    const float4 x0 = s_uw[rl], x1 = s_uw[rl + 1];
                    const float4 qv = qq[i];
                    // conj(q) * u and conj(q) * w for rows rl, rl+1
                    ar = fmaf(qv.x, x0.x, fmaf(qv.y, x0.y, ar));
                    ai = fmaf(qv.x, x0.y, fmaf(-qv.y, x0.x, ai));
                    br = fmaf(qv.x, x0.z, fmaf(qv.y, x0.w, br));
                    bi = fmaf(qv.x, x0.w, fmaf(-qv.y, x0.z, bi));
                    ar = fmaf(qv.z, x1.x, fmaf(qv.w, x1.y, ar));
                    ai = fmaf(qv.z, x1.y, fmaf(-qv.w, x1.x, ai));
                    br = fmaf(qv.z, x1.z, fmaf(qv.w, x1.w, br));
                    bi = fmaf(qv.z, x1.w, fmaf(-qv.w, x1.z, bi));
                }
            }
            ar = warp_sum(ar);
            ai = warp_sum(ai);
            br = warp_sum(br);
            bi = warp_sum(bi);
            if (lane == 0) {
                acc[c].x += ar;
                acc[c].y += ai;
                acc[p + c].x += br;
                acc[p + c].y += bi;
            }
        }
    }
    __syncthreads();
    if (cg == 0 && tid == 0) {
        double t[4] = {0.0, 0.0, 0.0, 0.0};
        for (int w = 0; w < DOT_THREADS / 32; w++)
            for (int q = 0; q < 4; q++) t[q] += s_sc[w][q];
        acc[2 * p] = make_double2(t[0], 0.0);
        acc[2 * p + 1] = make_double2(t[1], t[2]);
        acc[2 * p + 2] = make_double2(t[3], 0.0);
    }
    __syncthreads();
    double2* out = B.part + ((size_t)s * B.G + blockIdx.x) * B.pstride;
    // columns of this group (and the scalars from group 0); other groups write theirs
    for (int c = cg + CG * tid; c < p; c += CG * DOT_THREADS) {
        out[c] = acc[c];
        out[p + c] = acc[p + c];
    }
    if (cg == 0 && tid < 3) out[2 * p + tid] = acc[2 * p + tid];
}

// sum the per-block partials: dots[s][o] = sum_g part[s][g][o]
__global__ void __launch_bounds__(256) k_gs_reduce(BatchDev B, int j, int G_used) {
    const int s = blockIdx.y;
    const SolveDev& d = B.sd[s];
    if (!solve_in_step(d, j)) return;
    const int p = solve_p(d, j);
    const int nout = 2 * p + 3;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int o = blockIdx.x * 32 + lane;
    __shared__ double2 red[8][32];
    double2 v = make_double2(0.0, 0.0);
    if (o < nout)
        for (int g = warp; g < G_used; g += 8) {
            double2 t = B.part[((size_t)s * B.G + g) * B.pstride + o];
            v.x += t.x;
            v.y += t.y;
        }
    red[warp][lane] = v;
    __syncthreads();
    if (warp == 0 && o < nout) {
        double2 t = red[0][lane];
        for (int k = 1; k < 8; k++) {
            t.x += red[k][lane].x;
            t.y += red[k][lane].y;
        }
        d.dots[o] = t;
    }
}

// ---------------------------------------------------------------------------
// small step: d = H a (FP32 is enough: |a| is at the rounding level of one
// Gram-Schmidt pass), then nu, c, e and the pass-B coefficients; H update.
// k_gs_small: one CTA per solve, for the first step (no d) and for the final
// pass (j < 0: only the H update of column p-1). k_gs_small_rows: every other
// step, a CTA per 32 rows of d.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_gs_small(BatchDev B, int j) {
    const int s = blockIdx.y;
    SolveDev& d = B.sd[s];
    if (!solve_in_step(d, j)) return;
    const int p = solve_p(d, j);
    const int ld = d.ldH;
    const bool first = (j == 1);
    const bool final_pass = (j < 0);
    const int tid = threadIdx.x;
    const double2* dots = d.dots;
    // phase 2: one block per solve
    __shared__ double sh_r[8];
    __shared__ double2 sh_c[8];
    __shared__ double sh_nu, sh_ep_r, sh_ep_i;
    __shared__ int sh_stop;
    const int lane = tid & 31, warp = tid >> 5;
    // |a|^2 and a^dag b
    double aa = 0.0;
    double2 ab = make_double2(0.0, 0.0);
    if (!first)
        for (int c = tid; c < p; c += 256) {
            double2 av = dots[c], bv = dots[p + c];
            aa += av.x * av.x + av.y * av.y;
            ab.x += av.x * bv.x + av.y * bv.y;
            ab.y += av.x * bv.y - av.y * bv.x;
        }
    aa = warp_sumd(aa);
    ab.x = warp_sumd(ab.x);
    ab.y = warp_sumd(ab.y);
    if (lane == 0) {
        sh_r[warp] = aa;
        sh_c[warp] = ab;
    }
    __syncthreads();
    if (tid == 0) {
        double A2 = 0.0;
        double2 AB = make_double2(0.0, 0.0);
        for (int k = 0; k < 8; k++) {
            A2 += sh_r[k];
            AB.x += sh_c[k].x;
            AB.y += sh_c[k].y;
        }
        double guu = final_pass ? dots[p].x : dots[2 * p].x;
        double nu2 = first ? 1.0 : guu - A2;
        int stop = 0;
        if (!(nu2 == nu2) || !(guu == guu)) {
            stop = 2;  // NaN
        } else if (!first && !final_pass && nu2 <= 1e-24 * guu) {
            stop = 1;  // invariant subspace reached (happy breakdown)
            nu2 = 0.0;
        }
        double nu = sqrt(nu2 > 0.0 ? nu2 : 0.0);
        sh_nu = nu;
        sh_stop = stop;
        if (!final_pass && !stop) {
            // q^dag w = (u^dag w - a^dag b)/nu, and d_p = nu a_{p-1}
            double2 guw = dots[2 * p + 1];
            double2 qw = make_double2((guw.x - AB.x) / nu, (guw.y - AB.y) / nu);
            double2 dp = make_double2(0.0, 0.0);
            if (!first) {
                double2 al = dots[p - 1];
                dp = make_double2(nu * al.x, nu * al.y);
            }
            d.dvec[p] = dp;
            double2 cp = make_double2((qw.x - dp.x) / nu, (qw.y - dp.y) / nu);
            double2 ep = make_double2(dp.x / nu + cp.x, dp.y / nu + cp.y);
            d.H[p + (size_t)p * ld] = cp;
            d.H32[p + (size_t)p * ld] = make_float2((float)cp.x, (float)cp.y);
            sh_ep_r = ep.x;
            sh_ep_i = ep.y;
            d.scal[0] = 1.0 / nu;
            d.scal[1] = -ep.x / nu;
            d.scal[2] = -ep.y / nu;
            d.scal[3] = nu;
        }
    }
    __syncthreads();
    const double nu = sh_nu;
    const int stop = sh_stop;
    // update column p-1 with the reorthogonalisation coefficients and nu
    // (on breakdown the accurate final pass does it with k_used = j - 1)
    if (!first && stop != 1) {
        for (int c = tid; c < p; c += 256) {
            double2 av = dots[c];
            double2 h = d.H[c + (size_t)(p - 1) * ld];
            h.x += av.x;
            h.y += av.y;
            d.H[c + (size_t)(p - 1) * ld] = h;
            d.H32[c + (size_t)(p - 1) * ld] = make_float2((float)h.x, (float)h.y);
        }
        if (tid == 0) {
            d.H[p + (size_t)(p - 1) * ld] = make_double2(nu, 0.0);
            d.H32[p + (size_t)(p - 1) * ld] = make_float2((float)nu, 0.f);
        }
    }
    if (final_pass || stop) {
        if (tid == 0) {
            d.scal[4] = nu;
            if (stop == 2) {
                d.status = OVL_ENOCONV;
                d.active = 0;
            } else if (stop == 1 && !final_pass) {
                d.k_used = j - 1;  // the space spanned so far is invariant
                d.active = 0;
                d.fin = 1;         // u_j is in span(Q): the final pass projects it
            }
            if (final_pass) {
                d.active = 0;
                d.fin = 0;
            }
        }
        return;
    }
    // coefficients of column p (rows 0..p-1) and of pass B
    const double inv_nu = 1.0 / nu;
    const double epr = sh_ep_r, epi = sh_ep_i;
    for (int c = tid; c < p; c += 256) {
        double2 av = first ? make_double2(0.0, 0.0) : dots[c];
        double2 bv = dots[p + c];
        double2 dv = first ? make_double2(0.0, 0.0) : d.dvec[c];
        double2 cc = make_double2((bv.x - dv.x) * inv_nu, (bv.y - dv.y) * inv_nu);
        d.H[c + (size_t)p * ld] = cc;
        d.H32[c + (size_t)p * ld] = make_float2((float)cc.x, (float)cc.y);
        double2 e = make_double2(dv.x * inv_nu + cc.x, dv.y * inv_nu + cc.y);
        // g = e - (e_p/nu) a
        double2 g = make_double2(e.x - (epr * av.x - epi * av.y) * inv_nu, e.y - (epr * av.y + epi * av.x) * inv_nu);
        d.ap[c] = make_float2((float)(av.x * inv_nu), (float)(av.y * inv_nu));
        float2 sx = split_d(g.x), sy = split_d(g.y);
        d.gh[c] = make_float2(sx.x, sy.x);
        d.gl[c] = make_float2(sx.y, sy.y);
        if (d.ap64) {
            d.ap64[c] = cscale(av, inv_nu);
            d.g64[c] = g;
        }
    }
}

// Small step for j >= 2, one CTA per 32 rows r of the tile [r0, r0 + 32):
//  d_r = sum_c H32[r][c] a_c, the 16 warps splitting the columns (a lane per
//  row: coalesced column reads), then the step scalars (nu, c_p, e_p), which
//  every CTA of the solve computes from the same data in the same order (the
//  same bits), then column p of H, the correction of column p-1 and the
//  pass-B coefficients of its own rows. CTA 0 writes the entries of row p and
//  the scalars of the solve. A CTA writes H only in its own rows and reads
//  only its own rows of H32, so the CTAs need no ordering among themselves.
constexpr int SR_ROWS = 32;
constexpr int SR_THREADS = 512;

__global__ void __launch_bounds__(SR_THREADS) k_gs_small_rows(BatchDev B, int j) {
    const int s = blockIdx.y;
    SolveDev& d = B.sd[s];
    if (!solve_in_step(d, j)) return;
    const int p = solve_p(d, j);  // >= 1
    const int r0 = blockIdx.x * SR_ROWS;
    if (r0 >= p) return;
    const int ld = d.ldH;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const double2* dots = d.dots;
    __shared__ float2 red[SR_THREADS / 32][SR_ROWS];
    __shared__ double2 red64[SR_THREADS / 32][SR_ROWS];
    __shared__ double sh_r[SR_THREADS / 32];
    __shared__ double2 sh_c[SR_THREADS / 32];
    __shared__ double sh_nu, sh_inv, sh_ep_r, sh_ep_i;
    __shared__ int sh_stop;
    {
        const int row = r0 + lane;
        // H is upper Hessenberg below the Schur block: row i has no entries left of column i-1
        const int cmin = row >= d.m_q + 1 ? row - 1 : 0;
        float2 acc = make_float2(0.f, 0.f);
        if (row < p) {
#pragma unroll 8
            for (int c = warp; c < p; c += SR_THREADS / 32) {
                if (c < cmin) continue;
                const float2 h = d.H32[row + (size_t)c * ld];
                const double2 a = dots[c];
                const float2 av = make_float2((float)a.x, (float)a.y);
                acc.x = fmaf(h.x, av.x, fmaf(-h.y, av.y, acc.x));
                acc.y = fmaf(h.x, av.y, fmaf(h.y, av.x, acc.y));
            }
        }
        red[warp][lane] = acc;
        if (B.f64) {  // plain FP64 form: d = H a in FP64 from the FP64 H
            double2 a64 = make_double2(0.0, 0.0);
            if (row < p)
                for (int c = warp; c < p; c += SR_THREADS / 32) {
                    if (c < cmin) continue;
                    a64 = cadd(a64, cmul(d.H[row + (size_t)c * ld], dots[c]));
                }
            red64[warp][lane] = a64;
        }
    }
    // |a|^2 and a^dag b (same order in every CTA)
    double aa = 0.0;
    double2 ab = make_double2(0.0, 0.0);
    for (int c = tid; c < p; c += SR_THREADS) {
        const double2 av = dots[c], bv = dots[p + c];
        aa += av.x * av.x + av.y * av.y;
        ab.x += av.x * bv.x + av.y * bv.y;
        ab.y += av.x * bv.y - av.y * bv.x;
    }
    aa = warp_sumd(aa);
    ab.x = warp_sumd(ab.x);
    ab.y = warp_sumd(ab.y);
    if (lane == 0) {
        sh_r[warp] = aa;
        sh_c[warp] = ab;
    }
    __syncthreads();
    if (tid == 0) {
        double A2 = 0.0;
        double2 AB = make_double2(0.0, 0.0);
        for (int k = 0; k < SR_THREADS / 32; k++) {
            A2 += sh_r[k];
            AB.x += sh_c[k].x;
            AB.y += sh_c[k].y;
        }
        const double guu = dots[2 * p].x;
        double nu2 = guu - A2;
        int stop = 0;
        if (!(nu2 == nu2) || !(guu == guu)) {
            stop = 2;  // NaN
        } else if (nu2 <= 1e-24 * guu) {
            stop = 1;  // invariant subspace reached (happy breakdown)
            nu2 = 0.0;
        }
        const double nu = sqrt(nu2 > 0.0 ? nu2 : 0.0);
        sh_nu = nu;
        sh_stop = stop;
        if (!stop) {
            // q^dag w = (u^dag w - a^dag b)/nu, d_p = nu a_{p-1}, c_p = (q^dag w - d_p)/nu
            const double inv = 1.0 / nu;
            const double2 guw = dots[2 * p + 1];
            const double2 qw = make_double2((guw.x - AB.x) * inv, (guw.y - AB.y) * inv);
            const double2 al = dots[p - 1];
            const double2 dp = make_double2(nu * al.x, nu * al.y);
            const double2 cp = make_double2((qw.x - dp.x) * inv, (qw.y - dp.y) * inv);
            sh_inv = inv;
            sh_ep_r = dp.x * inv + cp.x;
            sh_ep_i = dp.y * inv + cp.y;
            if (blockIdx.x == 0) {
                d.dvec[p] = dp;
                d.H[p + (size_t)p * ld] = cp;
                d.H32[p + (size_t)p * ld] = make_float2((float)cp.x, (float)cp.y);
                d.scal[0] = inv;
                d.scal[1] = -sh_ep_r * inv;
                d.scal[2] = -sh_ep_i * inv;
                d.scal[3] = nu;
            }
        }
    }
    __syncthreads();
    const double nu = sh_nu;
    const int stop = sh_stop;
    if (warp == 0) {
        const int c = r0 + lane;
        float2 dr = red[0][lane];
        for (int w = 1; w < SR_THREADS / 32; w++) {
            dr.x += red[w][lane].x;
            dr.y += red[w][lane].y;
        }
        double2 dr64 = red64[0][lane];
        if (B.f64)
            for (int w = 1; w < SR_THREADS / 32; w++) dr64 = cadd(dr64, red64[w][lane]);
        if (c < p) {
            const double2 av = dots[c];
            // column p-1 += reorthogonalisation coefficients (on breakdown the
            // accurate final pass does it with k_used = j - 1)
            if (stop != 1) {
                double2 h = d.H[c + (size_t)(p - 1) * ld];
                h.x += av.x;
                h.y += av.y;
                d.H[c + (size_t)(p - 1) * ld] = h;
                d.H32[c + (size_t)(p - 1) * ld] = make_float2((float)h.x, (float)h.y);
            }
            if (!stop) {
                const double inv_nu = sh_inv, epr = sh_ep_r, epi = sh_ep_i;
                const double2 bv = dots[p + c];
                const double2 dv = B.f64 ? dr64 : make_double2(dr.x, dr.y);
                d.dvec[c] = dv;
                const double2 cc = make_double2((bv.x - dv.x) * inv_nu, (bv.y - dv.y) * inv_nu);
                d.H[c + (size_t)p * ld] = cc;
                d.H32[c + (size_t)p * ld] = make_float2((float)cc.x, (float)cc.y);
                const double2 e = make_double2(dv.x * inv_nu + cc.x, dv.y * inv_nu + cc.y);
                // g = e - (e_p/nu) a
                const double2 g = make_double2(e.x - (epr * av.x - epi * av.y) * inv_nu,
                                               e.y - (epr * av.y + epi * av.x) * inv_nu);
                d.ap[c] = make_float2((float)(av.x * inv_nu), (float)(av.y * inv_nu));
                const float2 sx = split_d(g.x), sy = split_d(g.y);
                d.gh[c] = make_float2(sx.x, sy.x);
                d.gl[c] = make_float2(sx.y, sy.y);
                if (d.ap64) {
                    d.ap64[c] = cscale(av, inv_nu);
                    d.g64[c] = g;
                }
            }
        }
    }
    if (blockIdx.x == 0 && tid == 0) {
        if (stop != 1) {
            d.H[p + (size_t)(p - 1) * ld] = make_double2(nu, 0.0);
            d.H32[p + (size_t)(p - 1) * ld] = make_float2((float)nu, 0.f);
        }
        if (stop) {
            d.scal[4] = nu;
            if (stop == 2) {
                d.status = OVL_ENOCONV;
                d.active = 0;
            } else {
                d.k_used = j - 1;  // the space spanned so far is invariant
                d.active = 0;
                d.fin = 1;         // u_j is in span(Q): the final pass projects it
            }
        }
    }
}

// ---------------------------------------------------------------------------
// pass B: q_{p+1} and u_{j+1} (see the file header)
// ---------------------------------------------------------------------------
template <int LO, int MINB = 3>  // LO 0: no low plane; 1: FP32 low planes; 2: BF16 low planes of the Krylov columns
__global__ void __launch_bounds__(256, MINB) k_gs_update(BatchDev B, int j) {
    constexpr bool DF = LO > 0;
    const int s = blockIdx.y;
    const SolveDev& d = B.sd[s];
    if (!solve_in_step(d, j)) return;
    const int p = solve_p(d, j);
    const size_t N = B.N;
    extern __shared__ float2 upd_dyn[];  // ap, gh, gl (pmax each), then column pointers
    float2* s_ap = upd_dyn;
    float2* s_gh = s_ap + B.pmax;
    float2* s_gl = s_gh + B.pmax;
    const float2** s_qh = (const float2**)(s_gl + B.pmax);
    const float2** s_ql = s_qh + OVL_MAXPTR;
    __shared__ float4 red_q[8][UPD_RB / 2];   // sq for row pairs
    __shared__ float4 red_g[8][UPD_RB];       // (s.x, s.y, t.x, t.y) per row
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nptr = d.nptr;
    for (int c = tid; c < p; c += 256) {
        s_ap[c] = d.ap[c];
        s_gh[c] = d.gh[c];
        if (DF) s_gl[c] = d.gl[c];
    }
    for (int c = tid; c < nptr && c < p; c += 256) {
        s_qh[c] = d.qhi[c];
        if (DF) s_ql[c] = d.qlo[c];
    }
    const double inv_nu = d.scal[0];
    const double2 cu = make_double2(d.scal[1], d.scal[2]);
    float2* qh_out = (float2*)(p < nptr ? d.qhi[p] : d.vhi + (size_t)(p - nptr) * N);
    float2* ql_out = LO == 1 ? (float2*)(p < nptr ? d.qlo[p] : d.vlo + (size_t)(p - nptr) * N) : nullptr;
    __nv_bfloat162* ql16_out = LO == 2 ? (__nv_bfloat162*)d.vlo + (size_t)(p - nptr) * N : nullptr;
    __syncthreads();
    for (size_t base = (size_t)blockIdx.x * UPD_RB; base < N; base += (size_t)gridDim.x * UPD_RB) {
        const bool full = base + UPD_RB <= N;
        float2 sq[UPD_RPL];
        dfacc sg[UPD_RPL];
#pragma unroll
        for (int i = 0; i < UPD_RPL; i++) {
            sq[i] = make_float2(0.f, 0.f);
            dfacc_zero(sg[i]);
        }
        // columns in descending order (pass A read them ascending: the most
        // recently read ones may still be in L2); two columns per iteration
        int c0 = p - 1 - warp;
        if constexpr (LO == 2) {
            // Krylov columns (c >= nptr): FP32 high plane + BF16 low plane, no
            // per-column branches so that all four loads of a lane are in flight
            const __nv_bfloat162* __restrict__ vlo16 = (const __nv_bfloat162*)d.vlo;
            for (; c0 - 8 >= nptr; c0 -= 16) {
                float4 h4[2][UPD_RPL / 2], l4[2][UPD_RPL / 2];
#pragma unroll
                for (int bb = 0; bb < 2; bb++) {
                    const size_t off = (size_t)(c0 - 8 * bb - nptr) * N;
                    const float4* __restrict__ qh = (const float4*)(d.vhi + off);
                    const void* ql16 = (const void*)(vlo16 + off);
#pragma unroll
                    for (int i = 0; i < UPD_RPL / 2; i++) {
                        const size_t r = base + 64 * i + 2 * lane;
                        const bool ok = full || r < N;
                        h4[bb][i] = ok ? __ldg(qh + (r >> 1)) : make_float4(0.f, 0.f, 0.f, 0.f);
                        l4[bb][i] = ok ? lo16_pair(ql16, r >> 1) : make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                }
#pragma unroll
                for (int bb = 0; bb < 2; bb++) {
                    const int c = c0 - 8 * bb;
                    const float2 apc = s_ap[c], ghc = s_gh[c], glc = s_gl[c];
#pragma unroll
                    for (int i = 0; i < UPD_RPL / 2; i++) {
                        const float4 hv = h4[bb][i], lv = l4[bb][i];
                        const float2 h0 = make_float2(hv.x, hv.y), h1 = make_float2(hv.z, hv.w);
                        sq[2 * i].x = fmaf(h0.x, apc.x, fmaf(-h0.y, apc.y, sq[2 * i].x));
                        sq[2 * i].y = fmaf(h0.x, apc.y, fmaf(h0.y, apc.x, sq[2 * i].y));
                        sq[2 * i + 1].x = fmaf(h1.x, apc.x, fmaf(-h1.y, apc.y, sq[2 * i + 1].x));
                        sq[2 * i + 1].y = fmaf(h1.x, apc.y, fmaf(h1.y, apc.x, sq[2 * i + 1].y));
                        dfacc_mac(sg[2 * i], h0, make_float2(lv.x, lv.y), ghc, glc);
                        dfacc_mac(sg[2 * i + 1], h1, make_float2(lv.z, lv.w), ghc, glc);
                    }
                }
            }
            // the rest (the Schur columns, FP32 low planes, and a last Krylov
            // column): one column per step, to keep the register peak at the loop above
            for (int c = c0; c >= 0; c -= 8) {
                const float4* __restrict__ qh =
                    (const float4*)(c < nptr ? s_qh[c] : d.vhi + (size_t)(c - nptr) * N);
                const float4* __restrict__ ql = c < nptr ? (const float4*)s_ql[c] : nullptr;
                const void* ql16 = c < nptr ? nullptr : (const void*)(vlo16 + (size_t)(c - nptr) * N);
                const float2 apc = s_ap[c], ghc = s_gh[c], glc = s_gl[c];
#pragma unroll
                for (int i = 0; i < UPD_RPL / 2; i++) {
                    const size_t r = base + 64 * i + 2 * lane;
                    if (!(full || r < N)) continue;
                    const float4 hv = __ldg(qh + (r >> 1));
                    const float4 lv = ql ? __ldg(ql + (r >> 1)) : lo16_pair(ql16, r >> 1);
                    const float2 h0 = make_float2(hv.x, hv.y), h1 = make_float2(hv.z, hv.w);
                    sq[2 * i].x = fmaf(h0.x, apc.x, fmaf(-h0.y, apc.y, sq[2 * i].x));
                    sq[2 * i].y = fmaf(h0.x, apc.y, fmaf(h0.y, apc.x, sq[2 * i].y));
                    sq[2 * i + 1].x = fmaf(h1.x, apc.x, fmaf(-h1.y, apc.y, sq[2 * i + 1].x));
                    sq[2 * i + 1].y = fmaf(h1.x, apc.y, fmaf(h1.y, apc.x, sq[2 * i + 1].y));
                    dfacc_mac(sg[2 * i], h0, make_float2(lv.x, lv.y), ghc, glc);
                    dfacc_mac(sg[2 * i + 1], h1, make_float2(lv.z, lv.w), ghc, glc);
                }
            }
            c0 = -1;
        }
        for (; c0 >= 0; c0 -= 16) {
            float4 h4[2][UPD_RPL / 2], l4[2][UPD_RPL / 2];
#pragma unroll
            for (int bb = 0; bb < 2; bb++) {
                const int c = c0 - 8 * bb;
                const float4* __restrict__ qh =
                    c >= 0 ? (const float4*)(c < nptr ? s_qh[c] : d.vhi + (size_t)(c - nptr) * N) : nullptr;
                const float4* __restrict__ ql =
                    (LO == 1 && c >= 0) ? (const float4*)(c < nptr ? s_ql[c] : d.vlo + (size_t)(c - nptr) * N)
                    : (LO == 2 && c >= 0 && c < nptr) ? (const float4*)s_ql[c] : nullptr;
                const void* ql16 = (LO == 2 && c >= nptr) ? (const void*)((const __nv_bfloat162*)d.vlo +
                                                                          (size_t)(c - nptr) * N)
                                                          : nullptr;
#pragma unroll
                for (int i = 0; i < UPD_RPL / 2; i++) {
                    size_t r = base + 64 * i + 2 * lane;
                    bool ok = qh && (full || r < N);
                    h4[bb][i] = ok ? __ldg(qh + (r >> 1)) : make_float4(0.f, 0.f, 0.f, 0.f);
                    if (LO == 2)
                        l4[bb][i] = !ok ? make_float4(0.f, 0.f, 0.f, 0.f)
                                        : ql16 ? lo16_pair(ql16, r >> 1) : __ldg(ql + (r >> 1));
                    else
                        l4[bb][i] = (DF && ok) ? __ldg(ql + (r >> 1)) : make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
#pragma unroll
            for (int bb = 0; bb < 2; bb++) {
                const int c = c0 - 8 * bb;
                if (c < 0) continue;
                const float2 apc = s_ap[c], ghc = s_gh[c];
                const float2 glc = DF ? s_gl[c] : make_float2(0.f, 0.f);
#pragma unroll
                for (int i = 0; i < UPD_RPL / 2; i++) {
                    const float4 hv = h4[bb][i], lv = l4[bb][i];
                    float2 h0 = make_float2(hv.x, hv.y), h1 = make_float2(hv.z, hv.w);
                    float2 l0 = make_float2(lv.x, lv.y), l1 = make_float2(lv.z, lv.w);
                    // sq += q * ap   (FP32; |ap| is tiny)
                    sq[2 * i].x = fmaf(h0.x, apc.x, fmaf(-h0.y, apc.y, sq[2 * i].x));
                    sq[2 * i].y = fmaf(h0.x, apc.y, fmaf(h0.y, apc.x, sq[2 * i].y));
                    sq[2 * i + 1].x = fmaf(h1.x, apc.x, fmaf(-h1.y, apc.y, sq[2 * i + 1].x));
                    sq[2 * i + 1].y = fmaf(h1.x, apc.y, fmaf(h1.y, apc.x, sq[2 * i + 1].y));
                    if (DF) {
                        dfacc_mac(sg[2 * i], h0, l0, ghc, glc);
                        dfacc_mac(sg[2 * i + 1], h1, l1, ghc, glc);
                    } else {
                        sg[2 * i].s.x = fmaf(h0.x, ghc.x, fmaf(-h0.y, ghc.y, sg[2 * i].s.x));
                        sg[2 * i].s.y = fmaf(h0.x, ghc.y, fmaf(h0.y, ghc.x, sg[2 * i].s.y));
                        sg[2 * i + 1].s.x = fmaf(h1.x, ghc.x, fmaf(-h1.y, ghc.y, sg[2 * i + 1].s.x));
                        sg[2 * i + 1].s.y = fmaf(h1.x, ghc.y, fmaf(h1.y, ghc.x, sg[2 * i + 1].s.y));
                    }
                }
            }
        }
        // cross-warp reduction
#pragma unroll
        for (int i = 0; i < UPD_RPL / 2; i++) {
            int rr = 64 * i + 2 * lane;  // local row (even)
            red_q[warp][rr >> 1] = make_float4(sq[2 * i].x, sq[2 * i].y, sq[2 * i + 1].x, sq[2 * i + 1].y);
            red_g[warp][rr] = make_float4(sg[2 * i].s.x, sg[2 * i].s.y, sg[2 * i].t.x, sg[2 * i].t.y);
            red_g[warp][rr + 1] =
                make_float4(sg[2 * i + 1].s.x, sg[2 * i + 1].s.y, sg[2 * i + 1].t.x, sg[2 * i + 1].t.y);
        }
        __syncthreads();
        if (tid < UPD_RB) {
            const int rr = tid;
            const size_t r = base + rr;
            if (r < N) {
                float2 tq = make_float2(0.f, 0.f);
                dfacc tg;
                dfacc_zero(tg);
                for (int k = 0; k < 8; k++) {
                    float4 q4 = red_q[k][rr >> 1];
                    tq.x += (rr & 1) ? q4.z : q4.x;
                    tq.y += (rr & 1) ? q4.w : q4.y;
                    float4 g4 = red_g[k][rr];
                    dfacc t;
                    t.s = make_float2(g4.x, g4.y);
                    t.t = make_float2(g4.z, g4.w);
                    dfacc_add(tg, t);
                }
                double2 ur = d.u[r], wr = d.w[r];
                double2 sgv = dfacc_value(tg);
                double2 q = make_double2(ur.x * inv_nu - (double)tq.x, ur.y * inv_nu - (double)tq.y);
                double2 un = make_double2(wr.x * inv_nu + (cu.x * ur.x - cu.y * ur.y) - sgv.x,
                                          wr.y * inv_nu + (cu.x * ur.y + cu.y * ur.x) - sgv.y);
                float2 qx = split_d(q.x), qy = split_d(q.y);
                qh_out[r] = make_float2(qx.x, qy.x);
                if (LO == 1) ql_out[r] = make_float2(qx.y, qy.y);
                if (LO == 2) ql16_out[r] = __floats2bfloat162_rn(qx.y, qy.y);
                d.u[r] = un;
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// pass B with the basis streamed by bulk copies (k_gs_update_bulk). The
// arithmetic is that of k_gs_update: the same columns per warp (c = p-1-w,
// p-9-w, ...), the same rows per lane and the same order of operations per
// accumulator, so the results are bit for bit those of k_gs_update. What
// differs is how a column reaches the registers: each warp owns a ring of
// PB_STAGES shared-memory stages; lane 0 fills a stage with one column over
// the CTA's current row block (cp.async.bulk of the high plane and of the low
// plane, completed on the stage's mbarrier) PB_STAGES columns ahead of use,
// continuing into the next row block, so the warp's loads stay in flight while
// it computes instead of being issued just before the arithmetic.
// On GB300 it removes the global-load stalls but is the slower path (16^3x32
// batch: 11.8 against 9.9 s of pass B per step in the 48-bit form, 12.8
// against 10.0 s in the 40-bit form): the per-column wait, vote and lane-0
// issue raise the executed instructions by 63 % and the kernel becomes
// issue-bound, so the register path (k_gs_update) is the default.
// ---------------------------------------------------------------------------
constexpr int PB_STAGES = 4;
constexpr int PB_HI = UPD_RB * (int)sizeof(float2);  // one column's high plane over a row block (1 KB)
constexpr int PB_STAGE = 2 * PB_HI;                  // + its low plane (FP32; a BF16 plane uses half)
constexpr int PB_RING = 8 * PB_STAGES * PB_STAGE;    // 8 warps
constexpr long long PB_MAX_POLLS = 1ll << 22;        // bounded stage waits (seconds)

size_t pb_dyn_bytes(int pmax) {
    return (size_t)PB_RING + 8 * PB_STAGES * sizeof(uint64_t) + (size_t)pmax * 3 * sizeof(float2) +
           2 * OVL_MAXPTR * sizeof(void*);
}

__device__ __forceinline__ float4 lo16_unpack(uint2 v) {  // two rows of BF16 low parts
    const float2 a = __bfloat1622float2(*(const __nv_bfloat162*)&v.x);
    const float2 b = __bfloat1622float2(*(const __nv_bfloat162*)&v.y);
    return make_float4(a.x, a.y, b.x, b.y);
}

template <int LO>  // 1: FP32 low planes; 2: BF16 low planes of the Krylov columns
__global__ void __launch_bounds__(256, 2) k_gs_update_bulk(BatchDev B, int j) {
    const int s = blockIdx.y;
    SolveDev& d = B.sd[s];
    if (!solve_in_step(d, j)) return;
    const int p = solve_p(d, j);
    const size_t N = B.N;
    extern __shared__ __align__(128) unsigned char pb_dyn[];
    unsigned char* ring = pb_dyn;
    uint64_t* bars = (uint64_t*)(pb_dyn + PB_RING);
    float2* s_ap = (float2*)(bars + 8 * PB_STAGES);
    float2* s_gh = s_ap + B.pmax;
    float2* s_gl = s_gh + B.pmax;
    const float2** s_qh = (const float2**)(s_gl + B.pmax);
    const float2** s_ql = s_qh + OVL_MAXPTR;
    __shared__ float4 red_q[8][UPD_RB / 2];
    __shared__ float4 red_g[8][UPD_RB];
    __shared__ int abort_flag;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nptr = d.nptr;
    for (int c = tid; c < p; c += 256) {
        s_ap[c] = d.ap[c];
        s_gh[c] = d.gh[c];
        s_gl[c] = d.gl[c];
    }
    for (int c = tid; c < nptr && c < p; c += 256) {
        s_qh[c] = d.qhi[c];
        s_ql[c] = d.qlo[c];
    }
    uint64_t* wbar = bars + warp * PB_STAGES;
    unsigned char* wring = ring + (size_t)warp * PB_STAGES * PB_STAGE;
    if (lane == 0)
        for (int st = 0; st < PB_STAGES; st++) mbar_init(wbar + st, 1);
    if (tid == 0) abort_flag = 0;
    mbar_init_fence();
    const double inv_nu = d.scal[0];
    const double2 cu = make_double2(d.scal[1], d.scal[2]);
    float2* qh_out = (float2*)(p < nptr ? d.qhi[p] : d.vhi + (size_t)(p - nptr) * N);
    float2* ql_out = LO == 1 ? (float2*)(p < nptr ? d.qlo[p] : d.vlo + (size_t)(p - nptr) * N) : nullptr;
    __nv_bfloat162* ql16_out = LO == 2 ? (__nv_bfloat162*)d.vlo + (size_t)(p - nptr) * N : nullptr;
    __syncthreads();
    // this warp's work: row blocks bi of the CTA (grid-stride) x its columns t
    const int ncw = p - 1 - warp >= 0 ? (p - 1 - warp) / 8 + 1 : 0;
    const size_t nblk = (N + UPD_RB - 1) / UPD_RB;
    const int nb = (size_t)blockIdx.x < nblk ? (int)((nblk - 1 - blockIdx.x) / gridDim.x + 1) : 0;
    const long long nitems = (long long)nb * ncw;
    auto issue = [&](long long it) {  // lane 0: item it -> stage it % PB_STAGES
        const int bi = (int)(it / ncw), t = (int)(it - (long long)bi * ncw);
        const size_t base = ((size_t)blockIdx.x + (size_t)bi * gridDim.x) * UPD_RB;
        const unsigned rows = (unsigned)((N - base) < (size_t)UPD_RB ? (N - base) : (size_t)UPD_RB);
        const int c = p - 1 - warp - 8 * t;
        const void* hs;
        const void* ls;
        unsigned lb;
        if (c < nptr) {
            hs = s_qh[c] + base;
            ls = s_ql[c] + base;
            lb = rows * 8u;
        } else {
            const size_t off = (size_t)(c - nptr) * N + base;
            hs = d.vhi + off;
            if (LO == 2) {
                ls = (const __nv_bfloat162*)d.vlo + off;
                lb = rows * 4u;
            } else {
                ls = d.vlo + off;
                lb = rows * 8u;
            }
        }
        const int st = (int)(it % PB_STAGES);
        unsigned char* dst = wring + st * PB_STAGE;
        mbar_arrive_expect_tx(wbar + st, rows * 8u + lb);
        bulk_copy_g2s(dst, hs, rows * 8u, wbar + st);
        bulk_copy_g2s(dst + PB_HI, ls, lb, wbar + st);
    };
    long long issued = 0;  // lane 0's count
    if (lane == 0)
        for (; issued < nitems && issued < PB_STAGES; issued++) issue(issued);
    long long it = 0;
    long long landed = 0;  // items whose stage wait completed (all of them unless a wait timed out)
    bool aborted = false;
    for (int bi = 0; bi < nb; bi++) {
        const size_t base = ((size_t)blockIdx.x + (size_t)bi * gridDim.x) * UPD_RB;
        const bool full = base + UPD_RB <= N;
        float2 sq[UPD_RPL];
        dfacc sg[UPD_RPL];
#pragma unroll
        for (int i = 0; i < UPD_RPL; i++) {
            sq[i] = make_float2(0.f, 0.f);
            dfacc_zero(sg[i]);
        }
        for (int t = 0; t < ncw; t++, it++) {
            if (aborted) continue;
            const int st = (int)(it % PB_STAGES);
            const bool ok_wait = *(volatile int*)&abort_flag == 0 &&
                                 mbar_wait(wbar + st, (unsigned)((it / PB_STAGES) & 1), PB_MAX_POLLS);
            if (__any_sync(0xffffffffu, !ok_wait)) {  // warp-uniform
                aborted = true;
                if (lane == 0) atomicExch(&abort_flag, 1);
                continue;
            }
            landed = it + 1;
            const int c = p - 1 - warp - 8 * t;
            const float2 apc = s_ap[c], ghc = s_gh[c], glc = s_gl[c];
            const unsigned char* sp = wring + st * PB_STAGE;
            const bool lo32 = LO == 1 || c < nptr;
#pragma unroll
            for (int i = 0; i < UPD_RPL / 2; i++) {
                const bool ok = full || base + 64 * i + 2 * lane < N;
                const float4 hv = ok ? ((const float4*)sp)[32 * i + lane] : make_float4(0.f, 0.f, 0.f, 0.f);
                const float4 lv = !ok   ? make_float4(0.f, 0.f, 0.f, 0.f)
                                  : lo32 ? ((const float4*)(sp + PB_HI))[32 * i + lane]
                                         : lo16_unpack(((const uint2*)(sp + PB_HI))[32 * i + lane]);
                const float2 h0 = make_float2(hv.x, hv.y), h1 = make_float2(hv.z, hv.w);
                // sq += q * ap   (FP32; |ap| is tiny)
                sq[2 * i].x = fmaf(h0.x, apc.x, fmaf(-h0.y, apc.y, sq[2 * i].x));
                sq[2 * i].y = fmaf(h0.x, apc.y, fmaf(h0.y, apc.x, sq[2 * i].y));
                sq[2 * i + 1].x = fmaf(h1.x, apc.x, fmaf(-h1.y, apc.y, sq[2 * i + 1].x));
                sq[2 * i + 1].y = fmaf(h1.x, apc.y, fmaf(h1.y, apc.x, sq[2 * i + 1].y));
                dfacc_mac(sg[2 * i], h0, make_float2(lv.x, lv.y), ghc, glc);
                dfacc_mac(sg[2 * i + 1], h1, make_float2(lv.z, lv.w), ghc, glc);
            }
            __syncwarp();
            if (lane == 0 && issued < nitems) {  // refill this stage PB_STAGES items ahead
                fence_proxy_async_smem();
                issue(issued);
                issued++;
            }
        }
        // cross-warp reduction (as k_gs_update)
#pragma unroll
        for (int i = 0; i < UPD_RPL / 2; i++) {
            int rr = 64 * i + 2 * lane;
            red_q[warp][rr >> 1] = make_float4(sq[2 * i].x, sq[2 * i].y, sq[2 * i + 1].x, sq[2 * i + 1].y);
            red_g[warp][rr] = make_float4(sg[2 * i].s.x, sg[2 * i].s.y, sg[2 * i].t.x, sg[2 * i].t.y);
            red_g[warp][rr + 1] =
                make_float4(sg[2 * i + 1].s.x, sg[2 * i + 1].s.y, sg[2 * i + 1].t.x, sg[2 * i + 1].t.y);
        }
        __syncthreads();
        if (tid < UPD_RB && *(volatile int*)&abort_flag == 0) {
            const int rr = tid;
            const size_t r = base + rr;
            if (r < N) {
                float2 tq = make_float2(0.f, 0.f);
                dfacc tg;
                dfacc_zero(tg);
                for (int k = 0; k < 8; k++) {
                    float4 q4 = red_q[k][rr >> 1];
                    tq.x += (rr & 1) ? q4.z : q4.x;
                    tq.y += (rr & 1) ? q4.w : q4.y;
                    float4 g4 = red_g[k][rr];
                    dfacc tt;
                    tt.s = make_float2(g4.x, g4.y);
                    tt.t = make_float2(g4.z, g4.w);
                    dfacc_add(tg, tt);
                }
                double2 ur = d.u[r], wr = d.w[r];
                double2 sgv = dfacc_value(tg);
                double2 q = make_double2(ur.x * inv_nu - (double)tq.x, ur.y * inv_nu - (double)tq.y);
                double2 un = make_double2(wr.x * inv_nu + (cu.x * ur.x - cu.y * ur.y) - sgv.x,
                                          wr.y * inv_nu + (cu.x * ur.y + cu.y * ur.x) - sgv.y);
                float2 qx = split_d(q.x), qy = split_d(q.y);
                qh_out[r] = make_float2(qx.x, qy.x);
                if (LO == 1) ql_out[r] = make_float2(qx.y, qy.y);
                if (LO == 2) ql16_out[r] = __floats2bfloat162_rn(qx.y, qy.y);
                d.u[r] = un;
            }
        }
        __syncthreads();
    }
    if (lane == 0 && issued > landed) {
        // only after a timed-out or abandoned wait: let this warp's copies in
        // flight land (bounded) before the CTA's shared memory is released
        for (long long k = landed; k < issued; k++)
            mbar_wait(wbar + (int)(k % PB_STAGES), (unsigned)((k / PB_STAGES) & 1), PB_MAX_POLLS);
    }
    if (tid == 0 && *(volatile int*)&abort_flag) {
        atomicExch(&d.status, OVL_ETIMEOUT);
        d.active = 0;
    }
}

// ---------------------------------------------------------------------------
// accurate projections for deflation, start vectors and the final Galerkin
// pass: P[c] = Q[:,c]^dag x in double-float (products of the 48-bit basis
// hi + lo with x split into hi + lo, error about 2^-46 of sum |q| |x|), and
// |x|^2 in FP64. Like pass A, a CTA stages a block of PJ_RB rows of x in
// shared memory (split once) and a warp streams one column over the block,
// each lane 32 rows, with one FP64 reduction per column and block.
// ---------------------------------------------------------------------------
constexpr int PJ_RB = 1024;
constexpr int PJ_FL = PJ_RB / 64;  // float4 (two rows) per lane per column

__global__ void __launch_bounds__(256) k_proj_dot(ProjDev* pds, double2* part, int G, int pstride, size_t N) {
    const int s = blockIdx.y;
    const ProjDev d = pds[s];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    __shared__ double2 acc[OVL_MAXCOL + 1];
    __shared__ float4 s_x[PJ_RB];  // x split: (hi.re, hi.im, lo.re, lo.im)
    __shared__ double s_nn[8];      // per-warp |x|^2 (summed in warp order)
    for (int o = tid; o <= d.ncol; o += 256) acc[o] = make_double2(0.0, 0.0);
    if (lane == 0) s_nn[warp] = 0.0;
    for (size_t base = (size_t)blockIdx.x * PJ_RB; base < N; base += (size_t)gridDim.x * PJ_RB) {
        __syncthreads();  // acc zeroed / s_x reuse
        double nn = 0.0;
        for (int rr = tid; rr < PJ_RB; rr += 256) {
            const size_t r = base + rr;
            const double2 x = r < N ? d.x[r] : make_double2(0.0, 0.0);
            const float2 xr = split_d(x.x), xi = split_d(x.y);
            s_x[rr] = make_float4(xr.x, xi.x, xr.y, xi.y);
            nn += x.x * x.x + x.y * x.y;
        }
        nn = warp_sumd(nn);
        if (lane == 0) s_nn[warp] += nn;
        __syncthreads();
        const bool full = base + PJ_RB <= N;  // N is even: a float4 never straddles the end
        for (int c = warp; c < d.ncol; c += 8) {
            const float4* __restrict__ qh = (const float4*)d.qhi[c] + (base >> 1);
            // columns without a low plane (FP32 basis) have a null entry: offset only real planes
            const float2* const qlc = d.qlo ? d.qlo[c] : nullptr;
            const bool l16 = c >= d.lo16_from && c < d.lo16_to;  // BF16 low plane (40-bit basis)
            const float4* __restrict__ ql = (qlc && !l16) ? (const float4*)qlc + (base >> 1) : nullptr;
            const void* ql16 = (qlc && l16) ? (const void*)((const __nv_bfloat162*)qlc + base) : nullptr;
            dfacc a;
            dfacc_zero(a);
#pragma unroll
            for (int hb = 0; hb < 2; hb++) {  // two batches of loads in flight
                float4 hv[PJ_FL / 2], lv[PJ_FL / 2];
#pragma unroll
                for (int i = 0; i < PJ_FL / 2; i++) {
                    const int rl = 64 * (hb * (PJ_FL / 2) + i) + 2 * lane;
                    const bool on = full || base + rl < N;
                    hv[i] = on ? __ldg(qh + (rl >> 1)) : make_float4(0.f, 0.f, 0.f, 0.f);
                    lv[i] = on && ql     ? __ldg(ql + (rl >> 1))
                            : on && ql16 ? lo16_pair(ql16, rl >> 1)
                                         : make_float4(0.f, 0.f, 0.f, 0.f);
                }
#pragma unroll
                for (int i = 0; i < PJ_FL / 2; i++) {
                    const int rl = 64 * (hb * (PJ_FL / 2) + i) + 2 * lane;
                    const float4 x0 = s_x[rl], x1 = s_x[rl + 1];
                    // conj(q) x for rows rl, rl+1
                    dfacc_mac(a, make_float2(hv[i].x, -hv[i].y), make_float2(lv[i].x, -lv[i].y),
                              make_float2(x0.x, x0.y), make_float2(x0.z, x0.w));
                    dfacc_mac(a, make_float2(hv[i].z, -hv[i].w), make_float2(lv[i].z, -lv[i].w),
                              make_float2(x1.x, x1.y), make_float2(x1.z, x1.w));
                }
            }
            const double2 v = dfacc_value(a);
            const double ar = warp_sumd(v.x), ai = warp_sumd(v.y);
            if (lane == 0) {
                acc[c].x += ar;
                acc[c].y += ai;
            }
        }
    }
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; w++) t += s_nn[w];
        acc[d.ncol] = make_double2(t, 0.0);
    }
    __syncthreads();
    double2* out = part + ((size_t)s * G + blockIdx.x) * pstride;
    for (int o = tid; o <= d.ncol; o += 256) out[o] = acc[o];
}

__global__ void __launch_bounds__(256) k_proj_reduce(ProjDev* pds, const double2* part, int G, int pstride) {
    const int s = blockIdx.y;
    const ProjDev d = pds[s];
    const int nout = d.ncol + 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int o = blockIdx.x * 32 + lane;
    __shared__ double2 red[8][32];
    double2 v = make_double2(0.0, 0.0);
    if (o < nout)
        for (int g = warp; g < G; g += 8) {
            double2 t = part[((size_t)s * G + g) * pstride + o];
            v.x += t.x;
            v.y += t.y;
        }
    red[warp][lane] = v;
    __syncthreads();
    if (warp == 0 && o < nout) {
        double2 t = red[0][lane];
        for (int k = 1; k < 8; k++) {
            t.x += red[k][lane].x;
            t.y += red[k][lane].y;
        }
        d.out[o] = t;
    }
}

// x -= sum_c Q[:,c] coef[c]   (df accumulation, FP64 subtraction)
__global__ void __launch_bounds__(256) k_proj_update(ProjDev* pds, size_t N) {
    const int s = blockIdx.y;
    const ProjDev d = pds[s];
    __shared__ float2 gh[OVL_MAXCOL], gl[OVL_MAXCOL];
    for (int c = threadIdx.x; c < d.ncol; c += 256) {
        double2 g = d.coef[c];
        float2 a = split_d(g.x), b = split_d(g.y);
        gh[c] = make_float2(a.x, b.x);
        gl[c] = make_float2(a.y, b.y);
    }
    __syncthreads();
    for (size_t r = blockIdx.x * (size_t)256 + threadIdx.x; r < N; r += (size_t)gridDim.x * 256) {
        dfacc acc;
        dfacc_zero(acc);
        for (int c = 0; c < d.ncol; c++) {
            const float2* lp = d.qlo ? d.qlo[c] : nullptr;  // null: column without a low plane
            dfacc_mac(acc, d.qhi[c][r], lp ? lp[r] : make_float2(0.f, 0.f), gh[c], gl[c]);
        }
        double2 v = dfacc_value(acc);
        double2 x = d.x[r];
        d.x[r] = make_double2(x.x - v.x, x.y - v.y);
    }
}

// y = sum_c Q[:,c] g[c]   (df accumulation)
__global__ void __launch_bounds__(256) k_gemv(GemvDev* gds, size_t N) {
    const int s = blockIdx.y;
    const GemvDev d = gds[s];
    __shared__ float2 gh[OVL_MAXCOL + 64], gl[OVL_MAXCOL + 64];
    for (int c = threadIdx.x; c < d.ncol; c += 256) {
        double2 g = d.g[c];
        float2 a = split_d(g.x), b = split_d(g.y);
        gh[c] = make_float2(a.x, b.x);
        gl[c] = make_float2(a.y, b.y);
    }
    __syncthreads();
    for (size_t r = blockIdx.x * (size_t)256 + threadIdx.x; r < N; r += (size_t)gridDim.x * 256) {
        dfacc acc;
        dfacc_zero(acc);
        for (int c = 0; c < d.ncol; c++) {
            float2 h = d.qhi[c][r];
            const float2* lp = d.qlo[c];
            float2 l = !lp ? make_float2(0.f, 0.f) : (c >= d.lo16_from && c < d.lo16_to) ? lo16_one(lp, r) : lp[r];
            dfacc_mac(acc, h, l, gh[c], gl[c]);
        }
        d.y[r] = dfacc_value(acc);
    }
}

// start vector: v1 = x/beta into column m_q and u
template <int LO>  // as k_gs_update
__global__ void __launch_bounds__(256) k_start(BatchDev B, const double* beta2, int stride) {
    const int s = blockIdx.y;
    SolveDev& d = B.sd[s];
    if (!d.active) return;
    double b2 = beta2[(size_t)s * stride];
    if (!(b2 > 0.0)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            d.active = 0;
            d.k_used = 0;
            d.fin = 0;
        }
        return;
    }
    double inv = 1.0 / sqrt(b2);
    const int c0 = d.m_q;
    float2* qh = (float2*)(c0 < d.nptr ? d.qhi[c0] : d.vhi + (size_t)(c0 - d.nptr) * B.N);
    float2* ql = LO == 1 ? (float2*)(c0 < d.nptr ? d.qlo[c0] : d.vlo + (size_t)(c0 - d.nptr) * B.N) : nullptr;
    __nv_bfloat162* ql16 = LO == 2 ? (__nv_bfloat162*)d.vlo + (size_t)(c0 - d.nptr) * B.N : nullptr;
    for (size_t r = blockIdx.x * (size_t)256 + threadIdx.x; r < B.N; r += (size_t)gridDim.x * 256) {
        double2 x = d.u[r];
        double2 v = make_double2(x.x * inv, x.y * inv);
        float2 a = split_d(v.x), b = split_d(v.y);
        qh[r] = make_float2(a.x, b.x);
        if (LO == 1) ql[r] = make_float2(a.y, b.y);
        // u_1 must be the stored value: 48-bit (FP32 low plane), 40-bit (BF16 low plane) or FP32
        if (LO == 2) {
            const __nv_bfloat162 l = __floats2bfloat162_rn(a.y, b.y);
            ql16[r] = l;
            const float2 lf = __bfloat1622float2(l);
            d.u[r] = make_double2((double)a.x + (double)lf.x, (double)b.x + (double)lf.y);
        } else {
            d.u[r] = LO == 1 ? make_double2((double)a.x + (double)a.y, (double)b.x + (double)b.y)
                             : make_double2(a.x, b.x);
        }
    }
}

// ---------------------------------------------------------------------------
// Plain FP64 form: the same passes on a complex128 basis with FP64 products
// and FP64 sums throughout (no FP32 storage, no double-float arithmetic).
// Column c of a solve is (const double2*)qhi[c] for c < nptr, else
// (const double2*)vhi + (c - nptr) N. GB300 issues FP64 at about 2 FMA per
// clock and SM, so these kernels are bound by the FP64 pipe (8 FMA per
// 16-byte basis entry in each pass), not by HBM.
// ---------------------------------------------------------------------------
constexpr int D64_RB = 256;  // rows per block of the FP64 inner-product passes

__device__ __forceinline__ const double2* col64(const SolveDev& d, const double2* const* sq, int c, size_t N) {
    return c < d.nptr ? sq[c] : (const double2*)d.vhi + (size_t)(c - d.nptr) * N;
}

// pass A: a = Q^dag u, b = Q^dag w, |u|^2, u^dag w, |w|^2 (partials per CTA)
__global__ void __launch_bounds__(256) k_gs_dot64(BatchDev B, int j) {
    const int s = blockIdx.y;
    const SolveDev& d = B.sd[s];
    if (!solve_in_step(d, j)) return;
    const int p = solve_p(d, j);
    const size_t N = B.N;
    const int CG = gridDim.z, cg = blockIdx.z;
    __shared__ double2 acc[2 * OVL_MAXCOL + 3];
    __shared__ const double2* s_col[OVL_MAXPTR];
    __shared__ double2 s_u[D64_RB], s_w[D64_RB];
    __shared__ double s_sc[8][4];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int o = tid; o < 2 * p + 3; o += 256) acc[o] = make_double2(0.0, 0.0);
    if (lane == 0)
        for (int q = 0; q < 4; q++) s_sc[warp][q] = 0.0;
    for (int c = tid; c < d.nptr && c < p; c += 256) s_col[c] = (const double2*)d.qhi[c];
    for (size_t base = (size_t)blockIdx.x * D64_RB; base < N; base += (size_t)gridDim.x * D64_RB) {
        __syncthreads();
        {
            const size_t r = base + tid;
            const double2 a = r < N ? d.u[r] : make_double2(0.0, 0.0);
            const double2 b = r < N ? d.w[r] : make_double2(0.0, 0.0);
            s_u[tid] = a;
            s_w[tid] = b;
            if (cg == 0) {
                double uu = cabs2(a), ww = cabs2(b);
                double2 uw = cconjmul(a, b);
                uu = warp_sumd(uu);
                ww = warp_sumd(ww);
                uw.x = warp_sumd(uw.x);
                uw.y = warp_sumd(uw.y);
                if (lane == 0) {
                    s_sc[warp][0] += uu;
                    s_sc[warp][1] += uw.x;
                    s_sc[warp][2] += uw.y;
                    s_sc[warp][3] += ww;
                }
            }
        }
        __syncthreads();
        for (int c = cg + CG * warp; c < p; c += CG * 8) {
            const double2* __restrict__ q = col64(d, s_col, c, N) + base;
            double2 ea = make_double2(0.0, 0.0), eb = make_double2(0.0, 0.0);
#pragma unroll
            for (int i = 0; i < D64_RB / 32; i++) {
                const int rl = 32 * i + lane;
                if (base + rl < N) {
                    const double2 qv = __ldg(q + rl);
                    ea = cadd(ea, cconjmul(qv, s_u[rl]));
                    eb = cadd(eb, cconjmul(qv, s_w[rl]));
                }
            }
            ea.x = warp_sumd(ea.x);
            ea.y = warp_sumd(ea.y);
            eb.x = warp_sumd(eb.x);
            eb.y = warp_sumd(eb.y);
            if (lane == 0) {
                acc[c] = cadd(acc[c], ea);
                acc[p + c] = cadd(acc[p + c], eb);
            }
        }
    }
    __syncthreads();
    if (cg == 0 && tid == 0) {
        double t[4] = {0.0, 0.0, 0.0, 0.0};
        for (int w = 0; w < 8; w++)
            for (int q = 0; q < 4; q++) t[q] += s_sc[w][q];
        acc[2 * p] = make_double2(t[0], 0.0);
        acc[2 * p + 1] = make_double2(t[1], t[2]);
        acc[2 * p + 2] = make_double2(t[3], 0.0);
    }
    __syncthreads();
    double2* out = B.part + ((size_t)s * B.G + blockIdx.x) * B.pstride;
    for (int c = cg + CG * tid; c < p; c += CG * 256) {
        out[c] = acc[c];
        out[p + c] = acc[p + c];
    }
    if (cg == 0 && tid < 3) out[2 * p + tid] = acc[2 * p + tid];
}

// pass B: q_{p+1} = u/nu - Q (a/nu) -> column p; u <- w/nu - (e_p/nu) u - Q g
__global__ void __launch_bounds__(256) k_gs_update64(BatchDev B, int j) {
    const int s = blockIdx.y;
    const SolveDev& d = B.sd[s];
    if (!solve_in_step(d, j)) return;
    const int p = solve_p(d, j);
    const size_t N = B.N;
    extern __shared__ double2 upd64_dyn[];  // ap (pmax), g (pmax), then column pointers
    double2* s_ap = upd64_dyn;
    double2* s_g = s_ap + B.pmax;
    const double2** s_col = (const double2**)(s_g + B.pmax);
    for (int c = threadIdx.x; c < p; c += 256) {
        s_ap[c] = d.ap64[c];
        s_g[c] = d.g64[c];
    }
    for (int c = threadIdx.x; c < d.nptr && c < p; c += 256) s_col[c] = (const double2*)d.qhi[c];
    const double inv_nu = d.scal[0];
    const double2 cu = make_double2(d.scal[1], d.scal[2]);
    double2* q_out = (double2*)(p < d.nptr ? (const double2*)d.qhi[p] : (const double2*)d.vhi + (size_t)(p - d.nptr) * N);
    __syncthreads();
    for (size_t r = blockIdx.x * (size_t)256 + threadIdx.x; r < N; r += (size_t)gridDim.x * 256) {
        double2 sq = make_double2(0.0, 0.0), sg = make_double2(0.0, 0.0);
        int c = 0;
        for (; c + 4 <= p; c += 4) {  // four loads in flight
            double2 qv[4];
#pragma unroll
            for (int t = 0; t < 4; t++) qv[t] = __ldg(col64(d, s_col, c + t, N) + r);
#pragma unroll
            for (int t = 0; t < 4; t++) {
                sq = cadd(sq, cmul(qv[t], s_ap[c + t]));
                sg = cadd(sg, cmul(qv[t], s_g[c + t]));
            }
        }
        for (; c < p; c++) {
            const double2 qv = __ldg(col64(d, s_col, c, N) + r);
            sq = cadd(sq, cmul(qv, s_ap[c]));
            sg = cadd(sg, cmul(qv, s_g[c]));
        }
        const double2 ur = d.u[r], wr = d.w[r];
        q_out[r] = csub(cscale(ur, inv_nu), sq);
        d.u[r] = csub(cadd(cscale(wr, inv_nu), cmul(cu, ur)), sg);
    }
}

// P[c] = Q[:,c]^dag x (c < ncol) and |x|^2, partials per CTA
__global__ void __launch_bounds__(256) k_proj_dot64(ProjDev* pds, double2* part, int G, int pstride, size_t N) {
    const int s = blockIdx.y;
    const ProjDev d = pds[s];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    __shared__ double2 acc[OVL_MAXCOL + 1];
    __shared__ double2 s_x[D64_RB];
    __shared__ double s_nn[8];
    for (int o = tid; o <= d.ncol; o += 256) acc[o] = make_double2(0.0, 0.0);
    if (lane == 0) s_nn[warp] = 0.0;
    for (size_t base = (size_t)blockIdx.x * D64_RB; base < N; base += (size_t)gridDim.x * D64_RB) {
        __syncthreads();
        const size_t r = base + tid;
        const double2 x = r < N ? d.x[r] : make_double2(0.0, 0.0);
        s_x[tid] = x;
        const double nn = warp_sumd(cabs2(x));
        if (lane == 0) s_nn[warp] += nn;
        __syncthreads();
        for (int c = warp; c < d.ncol; c += 8) {
            const double2* __restrict__ q = (const double2*)d.qhi[c] + base;
            double2 e = make_double2(0.0, 0.0);
#pragma unroll
            for (int i = 0; i < D64_RB / 32; i++) {
                const int rl = 32 * i + lane;
                if (base + rl < N) e = cadd(e, cconjmul(__ldg(q + rl), s_x[rl]));
            }
            e.x = warp_sumd(e.x);
            e.y = warp_sumd(e.y);
            if (lane == 0) acc[c] = cadd(acc[c], e);
        }
    }
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; w++) t += s_nn[w];
        acc[d.ncol] = make_double2(t, 0.0);
    }
    __syncthreads();
    double2* out = part + ((size_t)s * G + blockIdx.x) * pstride;
    for (int o = tid; o <= d.ncol; o += 256) out[o] = acc[o];
}

// x -= sum_c Q[:,c] coef[c]
__global__ void __launch_bounds__(256) k_proj_update64(ProjDev* pds, size_t N) {
    const int s = blockIdx.y;
    const ProjDev d = pds[s];
    __shared__ double2 co[OVL_MAXCOL];
    for (int c = threadIdx.x; c < d.ncol; c += 256) co[c] = d.coef[c];
    __syncthreads();
    for (size_t r = blockIdx.x * (size_t)256 + threadIdx.x; r < N; r += (size_t)gridDim.x * 256) {
        double2 v = make_double2(0.0, 0.0);
        for (int c = 0; c < d.ncol; c++) v = cadd(v, cmul(__ldg((const double2*)d.qhi[c] + r), co[c]));
        d.x[r] = csub(d.x[r], v);
    }
}

// y = sum_c Q[:,c] g[c]
__global__ void __launch_bounds__(256) k_gemv64(GemvDev* gds, size_t N) {
    const int s = blockIdx.y;
    const GemvDev d = gds[s];
    __shared__ double2 co[OVL_MAXCOL + 64];
    for (int c = threadIdx.x; c < d.ncol; c += 256) co[c] = d.g[c];
    __syncthreads();
    for (size_t r = blockIdx.x * (size_t)256 + threadIdx.x; r < N; r += (size_t)gridDim.x * 256) {
        double2 v = make_double2(0.0, 0.0);
        for (int c = 0; c < d.ncol; c++) v = cadd(v, cmul(__ldg((const double2*)d.qhi[c] + r), co[c]));
        d.y[r] = v;
    }
}

// v_1 = x / beta into column m_q (complex128) and into u
__global__ void __launch_bounds__(256) k_start64(BatchDev B, const double* beta2, int stride) {
    const int s = blockIdx.y;
    SolveDev& d = B.sd[s];
    if (!d.active) return;
    const double b2 = beta2[(size_t)s * stride];
    if (!(b2 > 0.0)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            d.active = 0;
            d.k_used = 0;
            d.fin = 0;
        }
        return;
    }
    const double inv = 1.0 / sqrt(b2);
    const int c0 = d.m_q;
    double2* q = (double2*)(c0 < d.nptr ? (const double2*)d.qhi[c0] : (const double2*)d.vhi + (size_t)(c0 - d.nptr) * B.N);
    for (size_t r = blockIdx.x * (size_t)256 + threadIdx.x; r < B.N; r += (size_t)gridDim.x * 256) {
        const double2 v = cscale(d.u[r], inv);
        q[r] = v;
        d.u[r] = v;
    }
}

}  // namespace

int ovl_gs_grid(ovl_lattice lat) {
    size_t blocks = (lat->N + DOTB_RB - 1) / DOTB_RB;
    size_t g = (size_t)lat->num_sms * 2;
    if (blocks < g) g = blocks;
    if (g < 1) g = 1;
    return (int)g;
}

int ovl_gs_dot(ovl_lattice lat, const BatchDev& b, int j, cudaStream_t st) {
    // Column groups: the grid G x nsolve x CG should fill whole waves of
    // resident CTAs (measured at 8^4, 8 solves: CG = 3, 1.89 waves, 5.34 TB/s;
    // CG = 4, 2.53 waves, 4.89 TB/s); among CG = 1..8 take the largest
    // waves / ceil(waves), ties to fewer groups (less staging of u, w).
    if (!lat->gs_dot_occ) {
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_gs_dot, DOT_THREADS, 0);
        lat->gs_dot_occ = occ < 1 ? 1 : occ;
    }
    const double slots = (double)lat->gs_dot_occ * lat->num_sms;
    int cgs = 1;
    double best = -1.0;
    for (int cg = 1; cg <= 8; cg++) {
        if (cg > 1 && b.pmax < 8 * cg) break;  // at least 8 columns per group
        const double w = (double)b.G * b.nsolve * cg / slots;
        const double eff = w / std::ceil(w);
        if (eff > best + 0.01) {
            best = eff;
            cgs = cg;
        }
    }
    dim3 grid(b.G, b.nsolve, cgs);
    if (b.f64)
        k_gs_dot64<<<grid, 256, 0, st>>>(b, j);
    else
        k_gs_dot<<<grid, DOT_THREADS, 0, st>>>(b, j);
    OVL_LAUNCH_CHECK(lat);
    return OVL_OK;
}

int ovl_gs_reduce(ovl_lattice lat, const BatchDev& b, int j, cudaStream_t st) {
    int maxout = 2 * b.pmax + 3;
    dim3 grid((maxout + 31) / 32, b.nsolve);
    k_gs_reduce<<<grid, 256, 0, st>>>(b, j, b.G);
    OVL_LAUNCH_CHECK(lat);
    return OVL_OK;
}

int ovl_gs_small(ovl_lattice lat, const BatchDev& b, int j, cudaStream_t st) {
    if (j == 1 || j < 0) {
        k_gs_small<<<dim3(1, b.nsolve), 256, 0, st>>>(b, j);
    } else {
        // row tiles of the longest solve (p <= pmax < OVL_MAXCOL)
        k_gs_small_rows<<<dim3((b.pmax + SR_ROWS - 1) / SR_ROWS, b.nsolve), SR_THREADS, 0, st>>>(b, j);
    }
    OVL_LAUNCH_CHECK(lat);
    return OVL_OK;
}

int ovl_gs_update(ovl_lattice lat, const BatchDev& b, int j, cudaStream_t st) {
    size_t blocks = (b.N + UPD_RB - 1) / UPD_RB;
    size_t g = (size_t)lat->num_sms * 4;
    if (blocks < g) g = blocks;
    dim3 grid((unsigned)g, b.nsolve);
    // the batch is homogeneous in precision (checked by the caller)
    size_t dyn = (size_t)b.pmax * 3 * sizeof(float2) + 2 * OVL_MAXPTR * sizeof(void*);
    if (!lat->gs_update_attr) {  // a function attribute of the lattice's device
        OVL_CUDA_TRY(lat, cudaFuncSetAttribute(k_gs_update<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               64 * 1024));
        OVL_CUDA_TRY(lat, cudaFuncSetAttribute(k_gs_update<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               64 * 1024));
        OVL_CUDA_TRY(lat, cudaFuncSetAttribute(k_gs_update<2, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               64 * 1024));
        lat->gs_update_attr = true;
    }
    if (b.f64) {
        const size_t dyn64 = (size_t)b.pmax * 2 * sizeof(double2) + OVL_MAXPTR * sizeof(void*);
        if (dyn64 > 48 * 1024 && !lat->gs_update64_attr) {  // set once per lattice (not while a graph is captured)
            OVL_CUDA_TRY(lat, cudaFuncSetAttribute(k_gs_update64, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   64 * 1024));
            lat->gs_update64_attr = true;
        }
        k_gs_update64<<<grid, 256, dyn64, st>>>(b, j);
    } else if (b.df && b.bulk16 && lat->pass_b_bulk && b.pmax <= OVL_MAXCOL) {
        const size_t dynb = pb_dyn_bytes(b.pmax);
        if (!lat->gs_bulk_attr) {
            const int mx = (int)pb_dyn_bytes(OVL_MAXCOL);
            OVL_CUDA_TRY(lat, cudaFuncSetAttribute(k_gs_update_bulk<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
            OVL_CUDA_TRY(lat, cudaFuncSetAttribute(k_gs_update_bulk<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
            lat->gs_bulk_attr = true;
        }
        if (b.lo16)
            k_gs_update_bulk<2><<<grid, 256, dynb, st>>>(b, j);
        else
            k_gs_update_bulk<1><<<grid, 256, dynb, st>>>(b, j);
    } else if (b.lo16) {
        // two CTAs per SM without spills (120 registers); at three (80 registers)
        // it spills and measured 11.3 against 9.4 s of pass B per 16^3x32 step
        k_gs_update<2, 2><<<grid, 256, dyn, st>>>(b, j);
    }
    else if (b.df)
        k_gs_update<1><<<grid, 256, dyn, st>>>(b, j);
    else
        k_gs_update<0><<<grid, 256, dyn, st>>>(b, j);
    OVL_LAUNCH_CHECK(lat);
    return OVL_OK;
}

extern "C" int ovl_set_pass_b(ovl_lattice lat, int bulk) {
    if (!lat || bulk < 0 || bulk > 1) return ovl_fail(lat, OVL_EINVAL, "ovl_set_pass_b: bad argument");
    lat->pass_b_bulk = bulk;
    return OVL_OK;
}

int ovl_gs_final(ovl_lattice lat, const BatchDev& b, ProjDev* pd_dev, int maxcol, cudaStream_t st) {
    // Galerkin correction of the last column: s = Q^dag u_{k+1} in FP64
    // against the full hi+lo basis (the per-step FP32 inner products leave
    // the basis orthonormal to ~1e-7 only; the Arnoldi relation itself is
    // exact, and with an accurate s the projected matrix equals
    // Q^+ A Q, i.e. the result is the Galerkin approximation on span(Q)).
    if (int rc = ovl_proj_dot(lat, pd_dev, b.nsolve, maxcol, b.part, b.G, st, b.f64)) return rc;
    return ovl_gs_small(lat, b, -1, st);
}

int ovl_proj_dot(ovl_lattice lat, ProjDev* pd_dev, int nsolve, int maxcol, double2* part, int G, cudaStream_t st,
                 int f64) {
    int pstride = maxcol + 1;
    dim3 grid(G, nsolve);
    if (f64)
        k_proj_dot64<<<grid, 256, 0, st>>>(pd_dev, part, G, pstride, lat->N);
    else
        k_proj_dot<<<grid, 256, 0, st>>>(pd_dev, part, G, pstride, lat->N);
    OVL_LAUNCH_CHECK(lat);
    dim3 g2((maxcol + 1 + 31) / 32, nsolve);
    k_proj_reduce<<<g2, 256, 0, st>>>(pd_dev, part, G, pstride);
    OVL_LAUNCH_CHECK(lat);
    return OVL_OK;
}

int ovl_proj_update(ovl_lattice lat, ProjDev* pd_dev, int nsolve, int maxcol, cudaStream_t st, int f64) {
    (void)maxcol;
    size_t blocks = (lat->N + 255) / 256;
    size_t g = (size_t)lat->num_sms * 4;
    if (blocks < g) g = blocks;
    dim3 grid((unsigned)g, nsolve);
    if (f64)
        k_proj_update64<<<grid, 256, 0, st>>>(pd_dev, lat->N);
    else
        k_proj_update<<<grid, 256, 0, st>>>(pd_dev, lat->N);
    OVL_LAUNCH_CHECK(lat);
    return OVL_OK;
}

int ovl_gemv_df(ovl_lattice lat, GemvDev* gd_dev, int nsolve, int maxcol, cudaStream_t st, int f64) {
    (void)maxcol;
    size_t blocks = (lat->N + 255) / 256;
    size_t g = (size_t)lat->num_sms * 4;
    if (blocks < g) g = blocks;
    dim3 grid((unsigned)g, nsolve);
    if (f64)
        k_gemv64<<<grid, 256, 0, st>>>(gd_dev, lat->N);
    else
        k_gemv<<<grid, 256, 0, st>>>(gd_dev, lat->N);
    OVL_LAUNCH_CHECK(lat);
    return OVL_OK;
}

int ovl_start_vector(ovl_lattice lat, const BatchDev& b, const double* beta2_dev, int beta_stride, cudaStream_t st) {
    size_t blocks = (b.N + 255) / 256;
    size_t g = (size_t)lat->num_sms * 4;
    if (blocks < g) g = blocks;
    dim3 grid((unsigned)g, b.nsolve);
    if (b.f64)
        k_start64<<<grid, 256, 0, st>>>(b, beta2_dev, beta_stride);
    else if (b.lo16)
        k_start<2><<<grid, 256, 0, st>>>(b, beta2_dev, beta_stride);
    else if (b.df)
        k_start<1><<<grid, 256, 0, st>>>(b, beta2_dev, beta_stride);
    else
        k_start<0><<<grid, 256, 0, st>>>(b, beta2_dev, beta_stride);
    OVL_LAUNCH_CHECK(lat);
    return OVL_OK;
}
