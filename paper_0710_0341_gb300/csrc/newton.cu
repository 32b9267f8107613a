// Sign of the small projected matrix by the scaled Newton (Roberts)
// iteration (the matrix iterations Sec. 2 refers to; used for f(H_k) in
// Eqs. 11 and 22 and for f(H) on the whole block matrix of Eqs. 15-17):
//   X_0 = H,  X_{i+1} = (c_i X_i + X_i^{-1} / c_i) / 2,  c_i = |det X_i|^{-1/n},
// scaling dropped once the relative step |X_{i+1} - X_i|_F / |X_{i+1}|_F is
// below 1e-2; stopped when the relative step is below tol, one step after it
// fell below 1e-10 (quadratic convergence puts the next one near rounding),
// or when rounding stalls it (the step below 1e-8 no longer halves).
//
// Three implementations of the iteration live here: the FP64 kernel (below,
// newton_fp64 = 1), the double-float cooperative kernel (the fallback when no
// cluster shape fits), and the double-float kernel on thread-block clusters
// (the default; its comment block further down describes it). By default the
// iteration hands over to the Newton-Schulz finish of newton_schulz.cu once
// a step is below a threshold.
//
// FP64 kernel: one cooperative launch runs every iteration of every solve of
// a batch. The CTAs of one solve form a group that owns the matrix rows round-robin and
// inverts X_i by Gauss-Jordan elimination with partial pivoting (pivot rows
// chosen implicitly, no row swaps); the group meets at one barrier per pivot.
// Barriers are counters in global memory with a bounded wait: a wait that
// runs out sets OVL_ETIMEOUT for the solve and every CTA of the group leaves.
#include <algorithm>

#include "newton.cuh"
#include "wait.cuh"

namespace {

constexpr int NT = 256;
constexpr long long SPIN_LIMIT = 1ll << 24;  // polls of ~100 ns: about 2 s

// Barrier for the CTAs of one solve (group_wait in wait.cuh, bounded).
__device__ __forceinline__ bool group_sync(NewtonDev& d, unsigned& gen, int cpm) {
    return group_wait(d.bar, d.status, gen, cpm, SPIN_LIMIT);
}

__device__ __forceinline__ double warp_maxloc(double v, int& idx) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        double ov = __shfl_xor_sync(0xffffffffu, v, o);
        int oi = __shfl_xor_sync(0xffffffffu, idx, o);
        if (ov > v || (ov == v && oi < idx)) {
            v = ov;
            idx = oi;
        }
    }
    return v;
}

__global__ void __launch_bounds__(NT) k_newton(NewtonDev* nds, int nsolve, int cpm) {
    const int s = blockIdx.x / cpm;
    const int g = blockIdx.x % cpm;
    if (s >= nsolve) return;
    NewtonDev& d = nds[s];
    if (!d.run) return;
    const int n = d.n;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double2* __restrict__ X = d.X;
    double2* __restrict__ W = d.W;
    __shared__ double2 prow[2][OVL_NEWTON_MAXN];
    __shared__ unsigned char used[OVL_NEWTON_MAXN];
    __shared__ int piv[OVL_NEWTON_MAXN];
    __shared__ double s_red[NT / 32][2];
    __shared__ int s_idx[NT / 32];
    __shared__ double2 s_inv;
    __shared__ double s_c;
    unsigned gen = 0;
    // X_0 = H (column-major input, row-major iterate)
    for (int i = g; i < n; i += cpm)
        for (int l = tid; l < n; l += NT) X[(size_t)i * n + l] = d.H[i + (size_t)l * d.ldH];
    bool scaling = true;
    double prev_rel = 1e300;
    int iter = 0;
    bool converged = false;
    if (!group_sync(d, gen, cpm)) return;
    while (iter < d.max_iter) {
        iter++;
        // W = X for own rows, candidates for column 0
        for (int i = tid; i < n; i += NT) used[i] = 0;
        for (int i = g; i < n; i += cpm)
            for (int l = tid; l < n; l += NT) W[(size_t)i * n + l] = X[(size_t)i * n + l];
        __syncthreads();
        double logdet = 0.0;
        int bad = 0;
        for (int k = 0; k < n; k++) {
            // candidate of this CTA for column k among unused own rows
            {
                double best = -1.0;
                int bi = 0x7fffffff;
                for (int i = g + cpm * tid; i < n; i += cpm * NT)
                    if (!used[i]) {
                        double v = cabs2(W[(size_t)i * n + k]);
                        if (v > best || (v == best && i < bi)) {
                            best = v;
                            bi = i;
                        }
                    }
                best = warp_maxloc(best, bi);
                if (lane == 0) {
                    s_red[warp][0] = best;
                    s_idx[warp] = bi;
                }
                __syncthreads();
                if (tid == 0) {
                    for (int w = 1; w < NT / 32; w++)
                        if (s_red[w][0] > best || (s_red[w][0] == best && s_idx[w] < bi)) {
                            best = s_red[w][0];
                            bi = s_idx[w];
                        }
                    // two buffers by step parity: a CTA one step ahead cannot
                    // overwrite what a slower one is still reading
                    d.cand_val[(k & 1) * cpm + g] = best;
                    d.cand_row[(k & 1) * cpm + g] = bi;
                }
            }
            if (!group_sync(d, gen, cpm)) return;
            // global pivot (identical choice in every CTA)
            double best = -1.0;
            int pr = 0x7fffffff;
            for (int q = 0; q < cpm; q++) {
                double v = ((volatile double*)d.cand_val)[(k & 1) * cpm + q];
                int r = ((volatile int*)d.cand_row)[(k & 1) * cpm + q];
                if (v > best || (v == best && r < pr)) {
                    best = v;
                    pr = r;
                }
            }
            if (!(best > 0.0) || pr < 0 || pr >= n) {
                bad = 1;
                break;
            }
            const int buf = k & 1;
            // deferred write-back of the previous pivot row (its owner only)
            if (k > 0) {
                int pp = piv[k - 1];
                if (pp % cpm == g)
                    for (int l = tid; l < n; l += NT) W[(size_t)pp * n + l] = prow[buf ^ 1][l];
            }
            // FP64 is scarce on this GPU: the pivot reciprocal and log|pivot|
            // are formed once per CTA, not once per thread
            if (tid == 0) {
                double2 pv = W[(size_t)pr * n + k];
                s_inv = cinv(pv);
                logdet += 0.5 * log(cabs2(pv));
                used[pr] = 1;
                piv[k] = pr;
            }
            __syncthreads();
            const double2 inv = s_inv;
            for (int l = tid; l < n; l += NT) {
                double2 v = W[(size_t)pr * n + l];
                prow[buf][l] = (l == k) ? inv : cmul(v, inv);
            }
            __syncthreads();
            // eliminate own rows i != pr
            for (int i = g + cpm * warp; i < n; i += cpm * (NT / 32)) {
                if (i == pr) continue;
                double2* row = W + (size_t)i * n;
                double2 f = row[k];
                __syncwarp();
                for (int l = lane; l < n; l += 32) {
                    double2 pl = prow[buf][l];
                    if (l == k) {
                        row[l] = make_double2(-(f.x * pl.x - f.y * pl.y), -(f.x * pl.y + f.y * pl.x));
                    } else {
                        double2 v = row[l];
                        v.x -= f.x * pl.x - f.y * pl.y;
                        v.y -= f.x * pl.y + f.y * pl.x;
                        row[l] = v;
                    }
                }
            }
            __syncthreads();
        }
        if (bad) {
            if (tid == 0 && g == 0) atomicExch(d.status, OVL_ENOCONV);
            return;
        }
        // last pivot row write-back, then every row of the inverse is final
        {
            int pp = piv[n - 1];
            if (pp % cpm == g)
                for (int l = tid; l < n; l += NT) W[(size_t)pp * n + l] = prow[(n - 1) & 1][l];
        }
        if (!group_sync(d, gen, cpm)) return;
        // X_new[i][piv_j] = (c X[i][piv_j] + W[piv_i][j] / c) / 2
        if (tid == 0) s_c = scaling ? exp(-logdet / n) : 1.0;
        __syncthreads();
        const double c = s_c;
        const double ic = 1.0 / c;
        double dsum = 0.0, nsum = 0.0;
        for (int i = g + cpm * warp; i < n; i += cpm * (NT / 32)) {
            const double2* st = W + (size_t)piv[i] * n;
            double2* xr = X + (size_t)i * n;
            for (int j = lane; j < n; j += 32) {
                int l = piv[j];
                double2 xo = xr[l];
                double2 a = st[j];
                double2 xn = make_double2(0.5 * (c * xo.x + ic * a.x), 0.5 * (c * xo.y + ic * a.y));
                dsum += cabs2(csub(xn, xo));
                nsum += cabs2(xn);
                xr[l] = xn;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
            nsum += __shfl_xor_sync(0xffffffffu, nsum, o);
        }
        if (lane == 0) {
            s_red[warp][0] = dsum;
            s_red[warp][1] = nsum;
        }
        __syncthreads();
        if (tid == 0) {
            double a = 0.0, b = 0.0;
            for (int w = 0; w < NT / 32; w++) {
                a += s_red[w][0];
                b += s_red[w][1];
            }
            d.red[2 * g] = a;
            d.red[2 * g + 1] = b;
        }
        if (!group_sync(d, gen, cpm)) return;
        double D = 0.0, Nn = 0.0;
        for (int q = 0; q < cpm; q++) {
            D += ((volatile double*)d.red)[2 * q];
            Nn += ((volatile double*)d.red)[2 * q + 1];
        }
        const double diff = sqrt(D), nrm = sqrt(Nn);
        const double rel_step = diff / nrm;
        // stop at the tolerance; or one step after the relative step fell below
        // sqrt(tol) (quadratic convergence: this step is at the tolerance); or
        // when rounding stalls the unscaled iteration (step no longer halves)
        const bool unscaled = !scaling;
        if (rel_step <= d.tol || (unscaled && prev_rel <= 1e-10) ||
            (unscaled && prev_rel < 1e-8 && rel_step > 0.5 * prev_rel)) {
            converged = true;
            break;
        }
        if (rel_step < 1e-2) scaling = false;
        prev_rel = rel_step;
        if (!(nrm == nrm)) break;
    }
    if (g == 0 && tid == 0) {
        *d.iters = iter;
        if (!converged) atomicCAS(d.status, 0, OVL_ENOCONV);
    }
}

// y_s = F_s c_s for the coefficient vectors (F row-major n x n)
__global__ void __launch_bounds__(256) k_fmatvec(NewtonDev* nds, int nsolve) {
    const int s = blockIdx.y;
    NewtonDev& d = nds[s];
    if (!d.run) return;
    const int n = d.n;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int i = blockIdx.x * 8 + warp;
    if (i >= n) return;
    const double2* row = d.X + (size_t)i * n;
    const float4* rowf = (const float4*)row;
    double2 acc = make_double2(0.0, 0.0);
    for (int l = lane; l < n; l += 32) {
        double2 a, b = d.cvec[l];
        if (d.df) {
            float4 v = rowf[l];
            a = make_double2((double)v.x + (double)v.z, (double)v.y + (double)v.w);
        } else {
            a = row[l];
        }
        acc.x += a.x * b.x - a.y * b.y;
        acc.y += a.x * b.y + a.y * b.x;
    }
    for (int o = 16; o > 0; o >>= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    }
    if (lane == 0) d.gout[i] = acc;
}

}  // namespace

int ovl_newton_cpm(ovl_lattice lat, int nsolve, int nmax) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_newton, NT, 0);
    if (per_sm < 1) per_sm = 1;
    int cap = lat->num_sms * per_sm;
    int cpm = cap / (nsolve > 0 ? nsolve : 1);
    int want = (nmax + 7) / 8;  // at least 8 rows per CTA
    if (cpm > want) cpm = want;
    if (cpm > 64) cpm = 64;
    if (cpm < 1) cpm = 1;
    return cpm;
}

int ovl_newton_launch(ovl_lattice lat, NewtonDev* nd_dev, int nsolve, int cpm, cudaStream_t st) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_newton, NT, 0);
    if ((long)nsolve * cpm > (long)lat->num_sms * per_sm)
        return ovl_fail(lat, OVL_EINVAL, "Newton batch of %d x %d blocks exceeds co-residency (%d)", nsolve, cpm,
                        lat->num_sms * per_sm);
    void* args[] = {(void*)&nd_dev, (void*)&nsolve, (void*)&cpm};
    OVL_CUDA_TRY(lat, cudaLaunchCooperativeKernel((const void*)k_newton, dim3(nsolve * cpm), dim3(NT), args, 0, st));
    lat->launches++;
    return OVL_OK;
}

int ovl_fmatvec_launch(ovl_lattice lat, NewtonDev* nd_dev, int nsolve, int nmax, cudaStream_t st) {
    dim3 grid((nmax + 7) / 8, nsolve);
    k_fmatvec<<<grid, 256, 0, st>>>(nd_dev, nsolve);
    OVL_LAUNCH_CHECK(lat);
    return OVL_OK;
}

// ===========================================================================
// Double-float variant. GB300 issues FP64 at ~2 FMA/clock/SM and FP32 at 128,
// so the elimination runs in double-float (48-bit) arithmetic on the FP32
// pipes; only per-pivot scalars (reciprocal, log |pivot|) use FP64. Each CTA
// of a group keeps its rows of the work matrix in shared memory when they fit.
// Before every barrier each CTA publishes its best pivot candidate row to
// global memory, so the winning row is read by all CTAs right after the one
// barrier per pivot; the owner overwrites its copy with the scaled row.
// ===========================================================================
#include "df.cuh"

namespace {

constexpr int NTD = 512;  // threads of the double-float kernel (16 warps to hide FP32 chains)

template <bool SMEM>
__global__ void __launch_bounds__(NTD, 1) k_newton_df(NewtonDev* nds, int nsolve, int cpm) {
    extern __shared__ float4 dsm[];
    const int s = blockIdx.x / cpm;
    const int g = blockIdx.x % cpm;
    if (s >= nsolve) return;
    NewtonDev& d = nds[s];
    if (!d.run) return;
    const int n = d.n;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nr = (n - g + cpm - 1) / cpm;  // own rows: i = g + cpm * r
    float4* X = (float4*)d.X;
    float4* R = SMEM ? dsm : d.Wg + (size_t)g * (size_t)((n + cpm - 1) / cpm) * n;
    float4* prow = SMEM ? dsm + (size_t)nr * n : (float4*)(dsm);
    float4* fcol = prow + n;                          // nr values of column k
    int* piv = (int*)(fcol + ((nr + 1) & ~1));
    int* pinv = piv + n;
    unsigned char* used = (unsigned char*)(pinv + n);
    __shared__ float s_red[NTD / 32];
    __shared__ int s_idx[NTD / 32];
    __shared__ float4 s_inv;
    __shared__ double s_logdet, s_c;
    __shared__ float s_nrm[2][NTD / 32];
    __shared__ double s_cv[64];
    __shared__ int s_cr[64];
    unsigned gen = 0;
    // X_0 = H (column-major FP64 input); on resume X holds the iterate
    if (!d.resume)
        for (int r = 0; r < nr; r++) {
            int i = g + cpm * r;
            for (int l = tid; l < n; l += NTD) X[(size_t)i * n + l] = dfc_pack(dfc_from(d.H[i + (size_t)l * d.ldH]));
        }
    bool scaling = !d.resume, converged = false, handoff = false;
    double prev_rel = 1e300;
    int iter = 0;
    if (!group_sync(d, gen, cpm)) return;
    while (iter < d.max_iter) {
        iter++;
        for (int r = 0; r < nr; r++) {
            int i = g + cpm * r;
            for (int l = tid; l < n; l += NTD) R[(size_t)r * n + l] = __ldcg(X + (size_t)i * n + l);
        }
        for (int i = tid; i < n; i += NTD) used[i] = 0;
        if (tid == 0) s_logdet = 0.0;
        __syncthreads();
        int bad = 0;
        for (int k = 0; k < n; k++) {
            // best unused own row for column k (|hi|^2), published with its data
            float best = -1.f;
            int br = -1;
            for (int r = tid; r < nr; r += NTD) {
                int i = g + cpm * r;
                if (used[i]) continue;
                float4 v = R[(size_t)r * n + k];
                float a = v.x * v.x + v.y * v.y;
                if (a > best) {
                    best = a;
                    br = r;
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                float ov = __shfl_xor_sync(0xffffffffu, best, o);
                int oi = __shfl_xor_sync(0xffffffffu, br, o);
                if (ov > best || (ov == best && oi >= 0 && (br < 0 || oi < br))) {
                    best = ov;
                    br = oi;
                }
            }
            if (lane == 0) {
                s_red[warp] = best;
                s_idx[warp] = br;
            }
            __syncthreads();
            best = s_red[0];
            br = s_idx[0];
            for (int w = 1; w < NTD / 32; w++)
                if (s_red[w] > best || (s_red[w] == best && s_idx[w] >= 0 && (br < 0 || s_idx[w] < br))) {
                    best = s_red[w];
                    br = s_idx[w];
                }
            const int slot = (k & 1) * cpm + g;
            if (br >= 0)
                for (int l = tid; l < n; l += NTD) d.crow[(size_t)slot * n + l] = R[(size_t)br * n + l];
            if (tid == 0) {
                d.cand_val[slot] = br >= 0 ? (double)best : -1.0;
                d.cand_row[slot] = br >= 0 ? g + cpm * br : 0x7fffffff;
            }
            if (!group_sync(d, gen, cpm)) return;
            // candidates in parallel (one L2 read per thread), then the winner
            // (same choice in every CTA: largest |pivot|, then smallest row)
            if (tid < cpm) {
                s_cv[tid] = __ldcg(d.cand_val + (k & 1) * cpm + tid);
                s_cr[tid] = __ldcg(d.cand_row + (k & 1) * cpm + tid);
            }
            __syncthreads();
            double bv = -1.0;
            int pr = 0x7fffffff, q = -1;
            for (int c = 0; c < cpm; c++) {
                double v = s_cv[c];
                int rw = s_cr[c];
                if (v > bv || (v == bv && rw < pr)) {
                    bv = v;
                    pr = rw;
                    q = c;
                }
            }
            if (!(bv > 0.0) || q < 0) {
                bad = 1;
                break;
            }
            const float4* pw = d.crow + (size_t)((k & 1) * cpm + q) * n;
            if (tid == 0) {
                double2 pv = dfc_to(dfc_unpack(__ldcg(pw + k)));
                double2 inv = cinv(pv);
                s_inv = dfc_pack(dfc_from(inv));
                s_logdet += 0.5 * log(cabs2(pv));
                used[pr] = 1;
                piv[k] = pr;
            }
            // f values of own rows before they change
            for (int r = tid; r < nr; r += NTD) fcol[r] = R[(size_t)r * n + k];
            __syncthreads();
            const dfc inv = dfc_unpack(s_inv);
            for (int l = tid; l < n; l += NTD)
                prow[l] = l == k ? s_inv : dfc_pack(dfc_mul(dfc_unpack(__ldcg(pw + l)), inv));
            __syncthreads();
            const int rp = (pr % cpm == g) ? (pr - g) / cpm : -1;  // own index of the pivot row
            if (rp >= 0)
                for (int l = tid; l < n; l += NTD) R[(size_t)rp * n + l] = prow[l];
            // two rows per pass: independent dependency chains per thread
            for (int r0 = 0; r0 < nr; r0 += 2) {
                const bool two = r0 + 1 < nr;
                const bool a_on = r0 != rp, b_on = two && (r0 + 1 != rp);
                const dfc fa = dfc_unpack(fcol[r0]);
                const dfc fb = two ? dfc_unpack(fcol[r0 + 1]) : dfc_zero();
                float4* ra = R + (size_t)r0 * n;
                float4* rb = R + (size_t)(r0 + 1) * n;
                for (int l = tid; l < n; l += NTD) {
                    const dfc pl = dfc_unpack(prow[l]);
                    if (a_on) ra[l] = dfc_pack(dfc_fms(l == k ? dfc_zero() : dfc_unpack(ra[l]), fa, pl));
                    if (b_on) rb[l] = dfc_pack(dfc_fms(l == k ? dfc_zero() : dfc_unpack(rb[l]), fb, pl));
                }
            }
            __syncthreads();
        }
        if (bad) {
            if (tid == 0 && g == 0) atomicExch(d.status, OVL_ENOCONV);
            return;
        }
        for (int k = tid; k < n; k += NTD) pinv[piv[k]] = k;
        if (tid == 0) s_c = scaling ? exp(-s_logdet / n) : 1.0;
        __syncthreads();
        // inverse: Xinv[pinv(q)][piv[j]] = St[q][j] for the own stored rows q;
        // X_new row pinv(q) = (c X + Xinv / c) / 2, written by this CTA only
        const double c = s_c, ic = 1.0 / c;
        float dsum = 0.f, nsum = 0.f;
        for (int r = 0; r < nr; r++) {
            const int qrow = g + cpm * r;
            const int i = pinv[qrow];
            float4* xr = X + (size_t)i * n;
            for (int j = tid; j < n; j += NTD) {
                const int l = piv[j];
                dfc xo = dfc_unpack(__ldcg(xr + l));  // rows of X move between CTAs
                dfc a = dfc_unpack(R[(size_t)r * n + j]);
                dfc xn = dfc_axpby(0.5 * c, xo, 0.5 * ic, a);
                float dr = (xn.hi.x - xo.hi.x) + (xn.lo.x - xo.lo.x);
                float di = (xn.hi.y - xo.hi.y) + (xn.lo.y - xo.lo.y);
                dsum += dr * dr + di * di;
                nsum += xn.hi.x * xn.hi.x + xn.hi.y * xn.hi.y;
                xr[l] = dfc_pack(xn);
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
            nsum += __shfl_xor_sync(0xffffffffu, nsum, o);
        }
        if (lane == 0) {
            s_nrm[0][warp] = dsum;
            s_nrm[1][warp] = nsum;
        }
        __syncthreads();
        if (tid == 0) {
            double a = 0.0, b = 0.0;
            for (int w = 0; w < NTD / 32; w++) {
                a += s_nrm[0][w];
                b += s_nrm[1][w];
            }
            d.red[2 * g] = a;
            d.red[2 * g + 1] = b;
        }
        if (!group_sync(d, gen, cpm)) return;
        if (tid < cpm) {
            s_cv[tid] = __ldcg(d.red + 2 * tid);
            s_cr[tid] = 0;
        }
        __shared__ double s_nn[64];
        if (tid < cpm) s_nn[tid] = __ldcg(d.red + 2 * tid + 1);
        __syncthreads();
        double D = 0.0, Nn = 0.0;
        for (int c2 = 0; c2 < cpm; c2++) {
            D += s_cv[c2];
            Nn += s_nn[c2];
        }
        const double rel_step = sqrt(D) / sqrt(Nn);
        const bool unscaled = !scaling;
        if (rel_step <= d.tol || (unscaled && prev_rel <= 1e-10) ||
            (unscaled && prev_rel < 1e-8 && rel_step > 0.5 * prev_rel)) {
            converged = true;
            break;
        }
        if (d.ns_switch > 0.0 && rel_step < d.ns_switch) {  // Newton-Schulz takes over
            handoff = true;
            break;
        }
        if (rel_step < 1e-2) scaling = false;
        prev_rel = rel_step;
        if (!(Nn == Nn)) break;
    }
    if (g == 0 && tid == 0) {
        *d.iters = iter;
        if (handoff) *d.handoff = 1;
        else if (!converged) atomicCAS(d.status, 0, OVL_ENOCONV);
    }
}

size_t df_smem_bytes(int n, int nr, bool rows) {
    size_t b = 0;
    if (rows) b += (size_t)nr * n * sizeof(float4);
    b += (size_t)n * sizeof(float4);                  // prow
    b += (size_t)((nr + 1) & ~1) * sizeof(float4);    // fcol
    b += 2 * (size_t)n * sizeof(int) + (size_t)n + 64;  // piv, pinv, used
    return (b + 15) & ~(size_t)15;
}

}  // namespace

int ovl_newton_df_plan(ovl_lattice lat, int nsolve, int nmax, int* cpm_out, int* smem_rows) {
    int cpm = lat->num_sms / (nsolve > 0 ? nsolve : 1);
    int want = (nmax + 3) / 4;  // at least 4 rows per CTA
    if (cpm > want) cpm = want;
    if (cpm > 64) cpm = 64;
    if (cpm < 1) cpm = 1;
    int nr = (nmax + cpm - 1) / cpm;
    *smem_rows = df_smem_bytes(nmax, nr, true) <= 200 * 1024 ? 1 : 0;
    *cpm_out = cpm;
    return OVL_OK;
}

int ovl_newton_df_launch(ovl_lattice lat, NewtonDev* nd_dev, int nsolve, int nmax, int cpm, int smem_rows,
                         cudaStream_t st) {
    int nr = (nmax + cpm - 1) / cpm;
    size_t smem = df_smem_bytes(nmax, nr, smem_rows != 0);
    const void* fn = smem_rows ? (const void*)k_newton_df<true> : (const void*)k_newton_df<false>;
    OVL_CUDA_TRY(lat, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessorWithFlags(&per_sm, fn, NTD, smem, cudaOccupancyDefault);
    if (per_sm < 1 || (long)nsolve * cpm > (long)lat->num_sms * per_sm)
        return ovl_fail(lat, OVL_EINVAL, "Newton batch of %d x %d blocks exceeds co-residency (%d per SM)", nsolve,
                        cpm, per_sm);
    void* args[] = {(void*)&nd_dev, (void*)&nsolve, (void*)&cpm};
    OVL_CUDA_TRY(lat, cudaLaunchCooperativeKernel(fn, dim3(nsolve * cpm), dim3(NTD), args, smem, st));
    lat->launches++;
    return OVL_OK;
}

// ===========================================================================
// Cluster variant of the double-float Gauss-Jordan Newton. One thread-block
// cluster (16 CTAs, one per SM of a GPC) inverts one matrix; the rows live
// in the CTAs' shared memory (n^2 x 16 B fits 16 x 227 KB up to n of about
// 470). Per pivot: every CTA picks its best unused row for the column and
// copies it to a double-buffered candidate slot in its own shared memory,
// the cluster meets at one hardware barrier, and every CTA reads the
// candidates and then the winning row straight out of the owner's shared
// memory (distributed shared memory). The barrier is split (arrive, wait) with
// one step of lookahead: after the pivot row is known, a CTA first updates
// column k+1 of its rows, picks and fully updates its candidate for k+1,
// publishes it and arrives, and only then updates the rest of its rows, so
// the barrier and the candidate exchange overlap the bulk of the update.
// Candidate slots alternate by pivot parity: a slot is rewritten only after a
// barrier that every reader of its previous contents has passed.
// Clusters never wait on each other, so
// the launch is not cooperative: more matrices than resident clusters simply
// run in waves. All branches that skip a barrier (no work, singular pivot)
// are taken by every CTA of a cluster alike, since they depend only on data
// that every CTA reads identically, and each CTA passes one last barrier
// before it exits, so no CTA leaves while another still reads its memory.
// The scaling |det X|^(-1/n) accumulates |pivot|^2 as an FP32 mantissa and
// an integer exponent (the scale factor needs no more than FP32 accuracy),
// and the pivot reciprocal is formed in double-float, so the elimination
// uses no FP64 instruction.
// ===========================================================================
#include <cooperative_groups.h>

namespace {

namespace cg = cooperative_groups;

constexpr int NTC = 512;
constexpr int GPF = 4;  // prefetched L2-row elements per thread and pivot

// split cluster barrier (release on arrive, acquire on wait); every thread
// alternates arrive and wait, and cluster.sync() is one arrive plus one wait
__device__ __forceinline__ void cl_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory"); }
__device__ __forceinline__ void cl_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }

template <bool L2ROWS>
__global__ void __launch_bounds__(NTC, 1) k_newton_cl(NewtonDev* nds, int nsolve, int nrs_max) {
    extern __shared__ float4 csm[];
    cg::cluster_group cl = cg::this_cluster();
    const int CL = (int)cl.num_blocks();
    const int g = (int)cl.block_rank();
    const int s = blockIdx.x / CL;
    if (s >= nsolve) return;  // whole cluster
    NewtonDev& d = nds[s];
    if (!d.run) return;       // whole cluster
    const int n = d.n;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nr = (n - g + CL - 1) / CL;            // own rows: i = g + CL * r
    const int nrmax = (n + CL - 1) / CL;
    const int nrs = (L2ROWS && nrs_max < nrmax) ? nrs_max : nrmax;  // own rows kept in shared memory
    float4* X = (float4*)d.X;
    float4* R = csm;                                 // nrs x n
    // own rows nrs.. live in this CTA's private part of the work buffer (L2)
    float4* Rg = d.Wg + (size_t)g * (size_t)(nrmax - nrs) * n;
    auto rowp = [&](int r) -> float4* {
        return (!L2ROWS || r < nrs) ? R + (size_t)r * n : Rg + (size_t)(r - nrs) * n;
    };
    float4* crow = R + (size_t)nrs * n;              // 2 x n candidate rows (read by the cluster)
    float4* prow = crow + 2 * (size_t)n;             // n: scaled pivot row
    float4* fcol = prow + n;                         // nrmax: column k of own rows
    int* piv = (int*)(fcol + ((nrmax + 1) & ~1));
    int* pinv = piv + n;
    unsigned char* used = (unsigned char*)(pinv + n);
    __shared__ float s_red[NTC / 32];
    __shared__ int s_idx[NTC / 32];
    __shared__ float c_val[2];                       // candidate |pivot|^2 (read by the cluster)
    __shared__ int c_row[2];
    __shared__ float c_part[2];                      // per-iteration partial sums (read by the cluster)
    __shared__ int s_q, s_pr;
    __shared__ float s_bv;
    __shared__ float4 s_inv;
    __shared__ float s_mant;
    __shared__ int s_exp;
    // X_0 = H (column-major FP64 input), own rows; on resume X holds the iterate
    if (!d.resume)
        for (int r = 0; r < nr; r++) {
            const int i = g + CL * r;
            for (int l = tid; l < n; l += NTC) X[(size_t)i * n + l] = dfc_pack(dfc_from(d.H[i + (size_t)l * d.ldH]));
        }
    bool scaling = !d.resume, converged = false, bad = false, handoff = false;
    double prev_rel = 1e300;
    int iter = 0;
    // this CTA's best unused row for column col (largest |hi|^2, then smallest
    // row), brought up to date by row_update, copied to candidate slot `slot`
    // and published with its value; returns its own index (or -1)
    auto select_publish = [&](int col, int slot, auto&& row_update) -> int {
        float best = -1.f;
        int br = -1;
        for (int r = tid; r < nr; r += NTC) {
            if (used[g + CL * r]) continue;
            const float4 v = rowp(r)[col];
            const float a = v.x * v.x + v.y * v.y;
            if (a > best) {
                best = a;
                br = r;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float ov = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, br, o);
            if (ov > best || (ov == best && oi >= 0 && (br < 0 || oi < br))) {
                best = ov;
                br = oi;
            }
        }
        if (lane == 0) {
            s_red[warp] = best;
            s_idx[warp] = br;
        }
        __syncthreads();
        best = s_red[0];
        br = s_idx[0];
        for (int w = 1; w < NTC / 32; w++)
            if (s_red[w] > best || (s_red[w] == best && s_idx[w] >= 0 && (br < 0 || s_idx[w] < br))) {
                best = s_red[w];
                br = s_idx[w];
            }
        if (br >= 0)
            for (int l = tid; l < n; l += NTC) {
                row_update(br, l);
                crow[(size_t)slot * n + l] = rowp(br)[l];
            }
        if (tid == 0) {
            c_val[slot] = br >= 0 ? best : -1.f;
            c_row[slot] = br >= 0 ? g + CL * br : 0x7fffffff;
        }
        return br;
    };
    __syncthreads();
    while (iter < d.max_iter) {
        iter++;
        for (int r = 0; r < nr; r++) {
            const int i = g + CL * r;
            float4* rr = rowp(r);
            for (int l = tid; l < n; l += NTC) rr[l] = __ldcg(X + (size_t)i * n + l);
        }
        for (int i = tid; i < n; i += NTC) used[i] = 0;
        if (tid == 0) {
            s_mant = 1.f;
            s_exp = 0;
        }
        __syncthreads();
        // candidates for column 0 (rows fully current), then one split cluster
        // barrier per pivot: arrive once the next candidate is published,
        // wait before reading the candidates
        select_publish(0, 0, [](int, int) {});
        cl_arrive();
        for (int k = 0; k < n; k++) {
            const int slot = k & 1;
            cl_wait();
            // winner over the cluster: largest |pivot|^2, then smallest row
            if (warp == 0) {
                float v = -1.f;
                int rw = 0x7fffffff, q = -1;
                if (lane < CL) {
                    v = *cl.map_shared_rank(&c_val[slot], lane);
                    rw = *cl.map_shared_rank(&c_row[slot], lane);
                    q = lane;
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const float ov = __shfl_xor_sync(0xffffffffu, v, o);
                    const int orw = __shfl_xor_sync(0xffffffffu, rw, o);
                    const int oq = __shfl_xor_sync(0xffffffffu, q, o);
                    if (ov > v || (ov == v && orw < rw)) {
                        v = ov;
                        rw = orw;
                        q = oq;
                    }
                }
                if (lane == 0) {
                    s_bv = v;
                    s_pr = rw;
                    s_q = q;
                }
            }
            __syncthreads();
            if (!(s_bv > 0.f) || s_q < 0) {  // same decision in every CTA
                bad = true;
                break;
            }
            const int pr = s_pr;
            const float4* pw = cl.map_shared_rank(crow + (size_t)slot * n, s_q);
            if (tid == 0) {
                const dfc pv = dfc_unpack(pw[k]);
                s_inv = dfc_pack(dfc_inv(pv));
                int e;
                const float mnt = frexpf(s_mant * (pv.hi.x * pv.hi.x + pv.hi.y * pv.hi.y), &e);
                s_mant = mnt;
                s_exp += e;
                used[pr] = 1;
                piv[k] = pr;
            }
            for (int r = tid; r < nr; r += NTC) fcol[r] = rowp(r)[k];
            __syncthreads();
            const dfc inv = dfc_unpack(s_inv);
            for (int l = tid; l < n; l += NTC) prow[l] = l == k ? s_inv : dfc_pack(dfc_mul(dfc_unpack(pw[l]), inv));
            __syncthreads();
            const int rp = (pr % CL == g) ? (pr - g) / CL : -1;  // own index of the pivot row
            // x <- x - f p for own row r != rp at column l (column k: 0 - f p)
            auto upd_val = [&](int r, int l, float4 xin) -> float4 {
                if (r == rp) return prow[l];
                const dfc pl = dfc_unpack(prow[l]);
                const dfc f = dfc_unpack(fcol[r]);
                return dfc_pack(dfc_fms(l == k ? dfc_zero() : dfc_unpack(xin), f, pl));
            };
            auto upd = [&](int r, int l) {
                float4* x = rowp(r) + l;
                if (r == rp) {
                    *x = prow[l];
                } else {
                    const dfc pl = dfc_unpack(prow[l]);
                    const dfc f = dfc_unpack(fcol[r]);
                    *x = dfc_pack(dfc_fms(l == k ? dfc_zero() : dfc_unpack(*x), f, pl));
                }
            };
            int skip_r = -1, skip_l = -1;  // already updated: the published row, column k + 1
            if (k + 1 < n) {
                // lookahead: column k + 1, the next candidate row, publish, arrive
                for (int r = tid; r < nr; r += NTC) upd(r, k + 1);
                __syncthreads();
                skip_r = select_publish(k + 1, (k + 1) & 1, [&](int r, int l) { if (l != k + 1) upd(r, l); });
                skip_l = k + 1;
                cl_arrive();
            }
            // every remaining (own row, column) pair once, flattened over the
            // CTA: the first GPF elements of the rows in L2 are loaded before the
            // shared-memory rows are updated and written back after them
            const int gtot = L2ROWS ? (nr > nrs ? nr - nrs : 0) * n : 0;
            float4 gv[L2ROWS ? GPF : 1];
#pragma unroll
            for (int t = 0; t < (L2ROWS ? GPF : 0); t++) {
                const int e = tid + t * NTC;
                if (e < gtot) gv[t] = Rg[e];
            }
            {
                int r = tid / n, l = tid - (tid / n) * n;
                const int total = (nr < nrs ? nr : nrs) * n;
                for (int e = tid; e < total; e += NTC) {
                    if (r != skip_r && l != skip_l) upd(r, l);
                    l += NTC;
                    while (l >= n) {
                        l -= n;
                        r++;
                    }
                }
            }
#pragma unroll
            for (int t = 0; t < (L2ROWS ? GPF : 0); t++) {
                const int e = tid + t * NTC;
                if (e < gtot) {
                    const int r = nrs + e / n, l = e - (e / n) * n;
                    if (r != skip_r && l != skip_l) Rg[e] = upd_val(r, l, gv[t]);
                }
            }
            for (int e = tid + (L2ROWS ? GPF : 0) * NTC; e < gtot; e += NTC) {
                const int r = nrs + e / n, l = e - (e / n) * n;
                if (r != skip_r && l != skip_l) upd(r, l);
            }
            __syncthreads();
        }
        if (bad) break;
        for (int k = tid; k < n; k += NTC) pinv[piv[k]] = k;
        __syncthreads();
        const double logdet = 0.5 * (log((double)s_mant) + (double)s_exp * 0.69314718055994530942);
        const double c = scaling ? exp(-logdet / n) : 1.0, ic = 1.0 / c;
        // inverse: Xinv[pinv(q)][piv[j]] = St[q][j] for the own stored rows q;
        // X_new row pinv(q) = (c X + Xinv / c) / 2, written by this CTA only
        float dsum = 0.f, nsum = 0.f;
        for (int r = 0; r < nr; r++) {
            const int i = pinv[g + CL * r];
            float4* xr = X + (size_t)i * n;
            for (int j = tid; j < n; j += NTC) {
                const int l = piv[j];
                const dfc xo = dfc_unpack(__ldcg(xr + l));  // rows of X move between CTAs
                const dfc a = dfc_unpack(rowp(r)[j]);
                const dfc xn = dfc_axpby(0.5 * c, xo, 0.5 * ic, a);
                const float dr = (xn.hi.x - xo.hi.x) + (xn.lo.x - xo.lo.x);
                const float di = (xn.hi.y - xo.hi.y) + (xn.lo.y - xo.lo.y);
                dsum += dr * dr + di * di;
                nsum += xn.hi.x * xn.hi.x + xn.hi.y * xn.hi.y;
                xr[l] = dfc_pack(xn);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
            nsum += __shfl_xor_sync(0xffffffffu, nsum, o);
        }
        if (lane == 0) {
            s_red[warp] = dsum;
            s_idx[warp] = __float_as_int(nsum);
        }
        __syncthreads();
        if (tid == 0) {
            float a = 0.f, b = 0.f;
            for (int w = 0; w < NTC / 32; w++) {
                a += s_red[w];
                b += __int_as_float(s_idx[w]);
            }
            c_part[0] = a;
            c_part[1] = b;
        }
        cl.sync();  // also publishes this CTA's rows of X_new to the cluster
        double D = 0.0, Nn = 0.0;
        for (int q = 0; q < CL; q++) {  // same order in every CTA: same decision
            D += (double)*cl.map_shared_rank(&c_part[0], q);
            Nn += (double)*cl.map_shared_rank(&c_part[1], q);
        }
        const double rel_step = sqrt(D) / sqrt(Nn);
        const bool unscaled = !scaling;
        if (rel_step <= d.tol || (unscaled && prev_rel <= 1e-10) ||
            (unscaled && prev_rel < 1e-8 && rel_step > 0.5 * prev_rel)) {
            converged = true;
            break;
        }
        if (d.ns_switch > 0.0 && rel_step < d.ns_switch) {  // Newton-Schulz takes over
            handoff = true;
            break;
        }
        if (rel_step < 1e-2) scaling = false;
        prev_rel = rel_step;
        if (!(Nn == Nn)) break;
        // the partial sums are rewritten only after n more cluster barriers,
        // which every CTA reaches after these reads
    }
    if (g == 0 && tid == 0) {
        *d.iters = iter;
        if (bad) atomicExch(d.status, OVL_ENOCONV);
        else if (handoff) *d.handoff = 1;
        else if (!converged) atomicCAS(d.status, 0, OVL_ENOCONV);
    }
    cl.sync();  // no CTA leaves while another may read its shared memory
}

// shared memory of a CTA keeping nrs rows of an order-n matrix
size_t cl_smem_bytes(int n, int CL, int nrs) {
    const size_t nrmax = (size_t)((n + CL - 1) / CL);
    size_t b = (size_t)nrs * n * sizeof(float4);        // rows
    b += 3 * (size_t)n * sizeof(float4);                // 2 candidate rows + pivot row
    b += (size_t)((nrmax + 1) & ~(size_t)1) * sizeof(float4);
    b += 2 * (size_t)n * sizeof(int) + (size_t)n + 64;
    return (b + 15) & ~(size_t)15;
}

}  // namespace

int ovl_newton_cl_plan(ovl_lattice lat, int nsolve, int nmax, int* cl_size, size_t* smem_out, int* nrs_out,
                       int* l2rows_out) {
    // Cluster size and rows per CTA in shared memory. A GPC hosts one cluster
    // of 13..16 CTAs at most and a floor-swept GPC none, so a smaller cluster
    // can keep every matrix of a batch resident in one wave; rows that do not
    // fit a CTA's shared memory stay in its part of the work buffer (L2).
    // Rows in L2 put their latency on the per-pivot path (measured: one wave
    // of 12-CTA clusters with 7 of 36 rows in L2 is 1.4x slower than two
    // waves of 16-CTA clusters with every row in shared memory at n = 430),
    // so a shape with every row in shared memory is always preferred; among
    // those, and among the others, the cost is waves x rows per CTA.
    *cl_size = 0;
    *smem_out = 0;
    *nrs_out = 0;
    *l2rows_out = 0;
    int optin = 0, dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return OVL_OK;
    const size_t avail = (size_t)optin - 1024;  // static shared memory of the kernel
    for (const void* fn : {(const void*)k_newton_cl<false>, (const void*)k_newton_cl<true>})
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess ||
            cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)avail) != cudaSuccess) {
            cudaGetLastError();
            return OVL_OK;
        }
    long best_cost = -1;
    for (int CL = 16; CL >= 2; CL--) {
        const int nrmax = (nmax + CL - 1) / CL;
        const size_t fixed = cl_smem_bytes(nmax, CL, 0);
        if (fixed >= avail) continue;
        const size_t fit = (avail - fixed) / ((size_t)nmax * sizeof(float4));
        const int nrs = (int)std::min<size_t>((size_t)nrmax, fit);
        const int ng = nrmax - nrs;
        if (nrs < 1 || 2 * ng > nrmax) continue;
        const size_t smem = cl_smem_bytes(nmax, CL, nrs);
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = CL;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(CL);
        cfg.blockDim = dim3(NTC);
        cfg.dynamicSmemBytes = smem;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int active = 0;
        const void* fn = ng > 0 ? (const void*)k_newton_cl<true> : (const void*)k_newton_cl<false>;
        if (cudaOccupancyMaxActiveClusters(&active, fn, &cfg) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        if (active < 1) continue;
        const long waves = (nsolve + active - 1) / active;
        const long cost = (ng > 0 ? (1L << 40) : 0L) + waves * (long)(nrs + ng);
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            *cl_size = CL;
            *smem_out = smem;
            *nrs_out = nrs;
            *l2rows_out = ng > 0 ? 1 : 0;
        }
    }
    (void)lat;
    return OVL_OK;
}

int ovl_newton_cl_launch(ovl_lattice lat, NewtonDev* nd_dev, int nsolve, int cl_size, size_t smem, int nrs,
                         int l2rows, cudaStream_t st) {
    const void* fn = l2rows ? (const void*)k_newton_cl<true> : (const void*)k_newton_cl<false>;
    OVL_CUDA_TRY(lat, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cl_size;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(nsolve * cl_size);
    cfg.blockDim = dim3(NTC);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (l2rows)
        OVL_CUDA_TRY(lat, cudaLaunchKernelEx(&cfg, k_newton_cl<true>, nd_dev, nsolve, nrs));
    else
        OVL_CUDA_TRY(lat, cudaLaunchKernelEx(&cfg, k_newton_cl<false>, nd_dev, nsolve, nrs));
    lat->launches++;
    return OVL_OK;
}
