// Newton-Schulz finish of the sign of the small projected matrix.
//
// The scaled Newton iteration (Gauss-Jordan inverse per step, newton.cu)
// brings X_i close to the involution sgn(H); from there the inverse-free
// Newton-Schulz step
//     X <- X (3 I - X^2) / 2 = X + (X - X Y) / 2,   Y = X^2,
// converges quadratically to the same limit (Higham, Functions of Matrices,
// 2008, Sec. 5.3) and needs only two matrix products, which spread over the
// whole GPU instead of one cluster per matrix with a barrier per pivot. It
// is taken only while |I - X^2|_F < 1/2 (sufficient for convergence); a
// matrix that leaves that region goes back to the Gauss-Jordan iteration.
//
// Products are complex double-float GEMMs: 64 x 64 output tiles, 16-deep k
// slabs staged in shared memory, 4 x 4 outputs per thread accumulated with
// error-free transformations (df.cuh) and renormalised after every slab.
#include "df.cuh"
#include "newton.cuh"

namespace {

constexpr int NS_T = 64;         // output tile edge
constexpr int NS_K = 16;         // k slab
constexpr int NS_THREADS = 256;  // 16 x 16 threads, 4 x 4 outputs each

__device__ __forceinline__ void dfacc_renorm(dfacc& a) {
    float s, e;
    two_sum(a.s.x, a.t.x, s, e);
    a.s.x = s;
    a.t.x = e;
    two_sum(a.s.y, a.t.y, s, e);
    a.s.y = s;
    a.t.y = e;
}

__device__ __forceinline__ double block_sum(double v, double* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < NS_THREADS / 32; w++) t += red[w];
    return t;  // valid in thread 0
}

// MODE 0: Y = X X and |I - Y|_F^2.
// MODE 1: P = X Y, X_new = X + (X - P) / 2 into the other buffer, and
//         |X_new - X|_F^2, |X_new|_F^2 (skipped outside the region).
template <int MODE>
__global__ void __launch_bounds__(NS_THREADS) k_ns_gemm(const NsDev* __restrict__ nds) {
    const NsDev& d = nds[blockIdx.z];
    if (!d.on) return;
    const int n = d.n;
    const int i0 = blockIdx.y * NS_T, j0 = blockIdx.x * NS_T;
    if (i0 >= n || j0 >= n) return;
    const int tn = gridDim.x, t2 = tn * tn, tile = blockIdx.y * tn + blockIdx.x;
    const int tns = (n + NS_T - 1) / NS_T;  // tiles per edge of this matrix
    __shared__ double s_ry;
    if (MODE == 1) {  // |I - X^2|_F^2 from the tile partials, in tile order (same in every CTA)
        if (threadIdx.x == 0) {
            double ry = 0.0;
            for (int ty0 = 0; ty0 < tns; ty0++)
                for (int tx0 = 0; tx0 < tns; tx0++) ry += d.acc[ty0 * tn + tx0];
            s_ry = ry;
        }
        __syncthreads();
        if (!(s_ry < d.region)) return;
    }
    const float4* __restrict__ A = d.cur ? d.W : d.X;
    const float4* __restrict__ B = MODE == 0 ? A : d.Y;
    __shared__ float4 As[NS_K][NS_T + 1];  // As[k][i] = A[i0 + i][k0 + k]
    __shared__ float4 Bs[NS_K][NS_T];      // Bs[k][j] = B[k0 + k][j0 + j]
    __shared__ double red[NS_THREADS / 32];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    dfacc acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) dfacc_zero(acc[i][j]);
    for (int k0 = 0; k0 < n; k0 += NS_K) {
        for (int q = tid; q < NS_T * NS_K; q += NS_THREADS) {
            const int r = q / NS_K, c = q % NS_K;
            const int gi = i0 + r, gk = k0 + c;
            As[c][r] = (gi < n && gk < n) ? A[(size_t)gi * n + gk] : z4;
            const int rb = q / NS_T, cb = q % NS_T;
            const int gkb = k0 + rb, gj = j0 + cb;
            Bs[rb][cb] = (gkb < n && gj < n) ? B[(size_t)gkb * n + gj] : z4;
        }
        __syncthreads();
#pragma unroll 2
        for (int kk = 0; kk < NS_K; kk++) {
            float4 a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; i++) a[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; j++) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++)
                    dfacc_mac(acc[i][j], make_float2(a[i].x, a[i].y), make_float2(a[i].z, a[i].w),
                              make_float2(b[j].x, b[j].y), make_float2(b[j].z, b[j].w));
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
            for (int j = 0; j < 4; j++) dfacc_renorm(acc[i][j]);
    }
    double p0 = 0.0, p1 = 0.0;
    float4* __restrict__ out = MODE == 0 ? d.Y : (d.cur ? d.X : d.W);
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int gi = i0 + ty * 4 + i, gj = j0 + tx * 4 + j;
            if (gi >= n || gj >= n) continue;
            float hr, lr, hi, li;
            two_sum(acc[i][j].s.x, acc[i][j].t.x, hr, lr);
            two_sum(acc[i][j].s.y, acc[i][j].t.y, hi, li);
            if (MODE == 0) {
                out[(size_t)gi * n + gj] = make_float4(hr, hi, lr, li);
                const float dr = (hr - (gi == gj ? 1.f : 0.f)) + lr, di = hi + li;
                p0 += (double)dr * dr + (double)di * di;
            } else {
                const dfc x = dfc_unpack(A[(size_t)gi * n + gj]);
                const dfc pv = dfc_make(make_float2(hr, hi), make_float2(lr, li));
                const dfc one = dfc_make(make_float2(1.f, 0.f), make_float2(0.f, 0.f));
                const dfc mhalf = dfc_make(make_float2(-0.5f, 0.f), make_float2(0.f, 0.f));
                const dfc diff = dfc_fms(x, one, pv);     // X - P
                const dfc xn = dfc_fms(x, mhalf, diff);   // X + (X - P) / 2
                out[(size_t)gi * n + gj] = dfc_pack(xn);
                const float sr = diff.hi.x + diff.lo.x, si = diff.hi.y + diff.lo.y;
                p0 += 0.25 * ((double)sr * sr + (double)si * si);
                p1 += (double)xn.hi.x * xn.hi.x + (double)xn.hi.y * xn.hi.y;
            }
        }
    // one partial per tile (summed in tile order by the readers: deterministic)
    const double t0 = block_sum(p0, red);
    if (tid == 0) d.acc[(MODE == 0 ? 0 : t2) + tile] = t0;
    if (MODE == 1) {
        const double t1 = block_sum(p1, red);
        if (tid == 0) d.acc[2 * t2 + tile] = t1;
    }
}

// per matrix: region test, step, convergence (the Gauss-Jordan kernels' rule,
// plus: stop once a step is <= 1e-8); tile partials summed in tile order
__global__ void k_ns_check(NsDev* nds, int nsolve, int max_iter, int tn) {
    const int t2 = tn * tn;
    for (int s = threadIdx.x; s < nsolve; s += blockDim.x) {
        NsDev& d = nds[s];
        if (!d.on) continue;
        const int tns = (d.n + NS_T - 1) / NS_T;
        double ry = 0.0, D = 0.0, Nn = 0.0;
        for (int ty0 = 0; ty0 < tns; ty0++)
            for (int tx0 = 0; tx0 < tns; tx0++) {
                ry += d.acc[ty0 * tn + tx0];
                D += d.acc[t2 + ty0 * tn + tx0];
                Nn += d.acc[2 * t2 + ty0 * tn + tx0];
            }
        if (!(ry < d.region)) {
            d.fallback = 1;  // X unchanged (the update was skipped)
            d.on = 0;
        } else {
            const double rel = sqrt(D) / sqrt(Nn);
            d.cur ^= 1;
            d.iters++;
            if (!(rel == rel)) {
                d.fallback = 1;
                d.on = 0;
            } else if (rel <= d.tol || rel <= 1e-8 || d.prev <= 1e-10 || (d.prev < 1e-8 && rel > 0.5 * d.prev)) {
                // rel <= 1e-8: the step is quadratic, so the new iterate's error is
                // about rel^2, at the rounding level of the double-float products
                d.done = 1;
                d.on = 0;
            } else if (d.iters >= max_iter) {
                d.fallback = 1;
                d.on = 0;
            }
            d.prev = rel;
        }
    }
}

// the final iterate back into X where it ended in W
__global__ void __launch_bounds__(256) k_ns_final(NsDev* nds) {
    NsDev& d = nds[blockIdx.y];
    if (d.cur != 1) return;
    const size_t nn = (size_t)d.n * d.n;
    for (size_t e = blockIdx.x * (size_t)256 + threadIdx.x; e < nn; e += (size_t)gridDim.x * 256) d.X[e] = d.W[e];
}

}  // namespace

int ovl_newton_schulz(ovl_lattice lat, NsDev* d_ns, NsDev* h_ns, int nsolve, int nmax, int max_iter,
                      cudaStream_t st) {
    if (nsolve < 1 || nmax < 1) return OVL_OK;
    OVL_CUDA_TRY(lat, cudaMemcpyAsync(d_ns, h_ns, nsolve * sizeof(NsDev), cudaMemcpyHostToDevice, st));
    const dim3 grid((nmax + NS_T - 1) / NS_T, (nmax + NS_T - 1) / NS_T, nsolve);
    for (int it = 0; it < max_iter; it++) {
        k_ns_gemm<0><<<grid, NS_THREADS, 0, st>>>(d_ns);
        OVL_LAUNCH_CHECK(lat);
        k_ns_gemm<1><<<grid, NS_THREADS, 0, st>>>(d_ns);
        OVL_LAUNCH_CHECK(lat);
        k_ns_check<<<1, 32, 0, st>>>(d_ns, nsolve, max_iter, (int)grid.x);
        OVL_LAUNCH_CHECK(lat);
        OVL_CUDA_TRY(lat, cudaMemcpyAsync(h_ns, d_ns, nsolve * sizeof(NsDev), cudaMemcpyDeviceToHost, st));
        OVL_CUDA_TRY(lat, cudaStreamSynchronize(st));
        bool any = false;
        for (int s = 0; s < nsolve; s++) any = any || h_ns[s].on;
        if (!any) break;
    }
    k_ns_final<<<dim3(64, nsolve), 256, 0, st>>>(d_ns);
    OVL_LAUNCH_CHECK(lat);
    OVL_CUDA_TRY(lat, cudaMemcpyAsync(h_ns, d_ns, nsolve * sizeof(NsDev), cudaMemcpyDeviceToHost, st));
    OVL_CUDA_TRY(lat, cudaStreamSynchronize(st));
    return OVL_OK;
}
