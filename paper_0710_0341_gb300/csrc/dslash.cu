// H_w(mu) = gamma_5 D_w(mu): the 4D nearest-neighbour stencil of Eq. 2.
//
// The site arithmetic (spin projection, SU(3) mat-vecs, expansion, gamma_5)
// is in dslash_site.cuh; this file holds the kernels and their launcher.
// One thread per (site, right-hand side); links are shared by every
// right-hand side of a launch (they are re-read through L2, which holds them
// for every lattice this library targets).
#include "dd.cuh"
#include "dslash_site.cuh"
#include "ovl_common.cuh"

namespace {

using namespace ovl_stencil;

template <typename T, typename VT, int LINKS, bool TILED>
__device__ __forceinline__ void dslash_site(const KArgs& a) {
    const int r = blockIdx.y;
    if (a.active && !a.active[(size_t)r * a.stride]) return;  // whole CTA (one right-hand side)
    if (a.klim && a.j > a.klim[(size_t)r * a.stride]) return;
    // e^{+-mu} of this right-hand side. FP32 spinors: every thread takes the
    // FP32 exponentials itself (no barrier; the FP32 weights carry the FP32
    // kernel's own rounding). FP64 spinors: one thread per CTA in FP64 (an FP64
    // exp per thread would add to the FP64 pipe that bounds that kernel).
    T w_fw, w_bw;
    if constexpr (sizeof(T) == sizeof(float)) {
        const float mu = (float)a.mu[r];
        w_fw = expf(mu);
        w_bw = expf(-mu);
    } else {
        __shared__ T s_w[2];
        if (threadIdx.x == 0) {
            const double mu = a.mu[r];
            s_w[0] = (T)exp(mu);
            s_w[1] = (T)exp(-mu);
        }
        __syncthreads();
        w_fw = s_w[0];
        w_bw = s_w[1];
    }
    size_t site;
    if constexpr (TILED) {  // block -> (tile x, y, z, t), thread -> site in the tile
        unsigned b = blockIdx.x;
        const unsigned nbx = a.Lx / a.tx, nby = a.Ly / a.ty, nbz = a.Lz / a.tz;
        const unsigned bx = b % nbx;
        b /= nbx;
        const unsigned by = b % nby;
        b /= nby;
        const unsigned bz = b % nbz, t = b / nbz;
        const unsigned th = threadIdx.x;
        const unsigned x = bx * a.tx + th % a.tx, y = by * a.ty + (th / a.tx) % a.ty, z = bz * a.tz + th / (a.tx * a.ty);
        site = x + (size_t)a.Lx * (y + (size_t)a.Ly * (z + (size_t)a.Lz * t));
    } else {
        site = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    }
    if (site >= a.V) return;
    site_compute<T, VT, LINKS>(a, (const VT*)a.in[r], (VT*)a.out[r], site, w_fw, w_bw);
}

// FP64 spinors: the compiler's register choice (140 for FP64 links, 168 for the
// double-float arithmetic on FP64 data; no spills)
template <typename T, typename VT, int LINKS, bool TILED = false>
__global__ void __launch_bounds__(128) k_dslash(KArgs a) {
    dslash_site<T, VT, LINKS, TILED>(a);
}

// FP32 spinors: at most 64 registers, 8 CTAs per SM (measured 13 % faster
// than 96 registers with 12-real links at 24^3x48, in spite of a few spills)
template <typename T, typename VT, int LINKS, bool TILED = false, int MINB = 8>
__global__ void __launch_bounds__(128, MINB) k_dslash32(KArgs a) {
    dslash_site<T, VT, LINKS, TILED>(a);
}

// ---------------------------------------------------------------------------
// FP32 stencil with the neighbour data staged by asynchronous copies
// (cp.async, Ampere and later): each thread copies the next hop's neighbour
// spinor (6 x 16 B) and link (3 x 16 B for 12-real links, 4 x 16 B + 8 B for
// 18-real links) into its own slots of shared memory while it computes the
// current hop from the previous slots. A thread so keeps a whole hop of loads
// in flight without holding them in registers (the register-resident kernel
// spills at its 64-register cap). Slots are laid out [buffer][item][thread]:
// consecutive threads read consecutive 16-byte words (no bank conflicts).
// Same arithmetic, in the same order, as site_compute: results are identical.
// ---------------------------------------------------------------------------
constexpr int AS_T = 128;

__device__ __forceinline__ void cp_async16(float4* dst, const void* src) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(float4* dst, const void* src) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <int LINKS>
struct AsyncHop {
    static constexpr int NL = LINKS == OVL_LINKS_R12 ? 3 : 5;  // link words per hop
    static constexpr int ITEMS = 6 + NL;
    // copy the spinor at nb and the link (nu, ls) into buffer b of this thread
    static __device__ __forceinline__ void issue(const KArgs& a, const float4* in, float4* buf, int b, size_t nb,
                                                 int nu, size_t ls) {
        const size_t V = a.V;
        float4* s = buf + (size_t)b * ITEMS * AS_T + threadIdx.x;
#pragma unroll
        for (int cp = 0; cp < 6; cp++) cp_async16(s + cp * AS_T, in + (size_t)cp * V + nb);
        if constexpr (LINKS == OVL_LINKS_R12) {
#pragma unroll
            for (int p = 0; p < 3; p++) cp_async16(s + (6 + p) * AS_T, a.u12 + ((size_t)nu * 3 + p) * V + ls);
        } else {
#pragma unroll
            for (int p = 0; p < 4; p++) cp_async16(s + (6 + p) * AS_T, a.u32q + ((size_t)nu * 4 + p) * V + ls);
            cp_async8(s + 10 * AS_T, a.u32r + (size_t)nu * V + ls);
        }
        cp_commit();
    }
    // one hop from buffer b (as hop() of dslash_site.cuh)
    template <int NU, bool FWD>
    static __device__ __forceinline__ void run(const float4* buf, int b, float w, C<float> (&acc)[12]) {
        const float4* s = buf + (size_t)b * ITEMS * AS_T + threadIdx.x;
        C<float> psi[12];
#pragma unroll
        for (int cp = 0; cp < 6; cp++) {
            const float4 v = s[cp * AS_T];
            psi[2 * cp] = mk<float>(v.x, v.y);
            psi[2 * cp + 1] = mk<float>(v.z, v.w);
        }
        C<float> h[6];
        project<float, NU, FWD>(psi, h);
        C<float> u[9];
        if constexpr (LINKS == OVL_LINKS_R12) {
#pragma unroll
            for (int p = 0; p < 3; p++) {
                const float4 v = s[(6 + p) * AS_T];
                u[2 * p] = mk<float>(v.x, v.y);
                u[2 * p + 1] = mk<float>(v.z, v.w);
            }
            u[6] = conj(u[1] * u[5] - u[2] * u[4]);
            u[7] = conj(u[2] * u[3] - u[0] * u[5]);
            u[8] = conj(u[0] * u[4] - u[1] * u[3]);
        } else {
#pragma unroll
            for (int p = 0; p < 4; p++) {
                const float4 v = s[(6 + p) * AS_T];
                u[2 * p] = mk<float>(v.x, v.y);
                u[2 * p + 1] = mk<float>(v.z, v.w);
            }
            const float4 v = s[10 * AS_T];
            u[8] = mk<float>(v.x, v.y);
        }
        C<float> g[6];
        LinkMul<float>::template run<FWD>(u, h, g);
        expand_add<float, NU, FWD>(g, w, acc);
    }
};

template <int LINKS>
__global__ void __launch_bounds__(AS_T, 5) k_dslash32a(KArgs a) {
    using H = AsyncHop<LINKS>;
    extern __shared__ float4 as_buf[];  // [2][ITEMS][AS_T]
    const int r = blockIdx.y;
    if (a.active && !a.active[(size_t)r * a.stride]) return;
    if (a.klim && a.j > a.klim[(size_t)r * a.stride]) return;
    const float mu_r = (float)a.mu[r];  // as in dslash_site: FP32 weights per thread
    const float w_fw = expf(mu_r), w_bw = expf(-mu_r);
    const size_t site = blockIdx.x * (size_t)AS_T + threadIdx.x;
    if (site >= a.V) return;
    const float4* in = (const float4*)a.in[r];
    const int Lx = a.Lx, Ly = a.Ly, Lz = a.Lz, Lt = a.Lt;
    const size_t sy = Lx, sz = (size_t)Lx * Ly, stt = sz * Lz;
    unsigned q = (unsigned)site;
    const int x = (int)(q % (unsigned)Lx);
    q /= (unsigned)Lx;
    const int y = (int)(q % (unsigned)Ly);
    q /= (unsigned)Ly;
    const int z = (int)(q % (unsigned)Lz);
    const int t = (int)(q / (unsigned)Lz);
    const size_t xp = x + 1 == Lx ? site - (Lx - 1) : site + 1;
    const size_t xm = x == 0 ? site + (Lx - 1) : site - 1;
    const size_t yp = y + 1 == Ly ? site - (Ly - 1) * sy : site + sy;
    const size_t ym = y == 0 ? site + (Ly - 1) * sy : site - sy;
    const size_t zp = z + 1 == Lz ? site - (Lz - 1) * sz : site + sz;
    const size_t zm = z == 0 ? site + (Lz - 1) * sz : site - sz;
    const size_t tp = t + 1 == Lt ? site - (Lt - 1) * stt : site + stt;
    const size_t tm = t == 0 ? site + (Lt - 1) * stt : site - stt;
    float wtp = w_fw, wtm = w_bw;
    if (a.apbc) {
        if (t + 1 == Lt) wtp = -wtp;
        if (t == 0) wtm = -wtm;
    }
    C<float> acc[12];
#pragma unroll
    for (int i = 0; i < 12; i++) acc[i] = mk<float>(0.f, 0.f);
    // two buffers: hop h + 1 is in flight while hop h is computed
    H::issue(a, in, as_buf, 0, xp, 0, site);
    H::issue(a, in, as_buf, 1, xm, 0, xm);
    cp_wait<1>();
    H::template run<0, true>(as_buf, 0, 1.f, acc);
    H::issue(a, in, as_buf, 0, yp, 1, site);
    cp_wait<1>();
    H::template run<0, false>(as_buf, 1, 1.f, acc);
    H::issue(a, in, as_buf, 1, ym, 1, ym);
    cp_wait<1>();
    H::template run<1, true>(as_buf, 0, 1.f, acc);
    H::issue(a, in, as_buf, 0, zp, 2, site);
    cp_wait<1>();
    H::template run<1, false>(as_buf, 1, 1.f, acc);
    H::issue(a, in, as_buf, 1, zm, 2, zm);
    cp_wait<1>();
    H::template run<2, true>(as_buf, 0, 1.f, acc);
    H::issue(a, in, as_buf, 0, tp, 3, site);
    cp_wait<1>();
    H::template run<2, false>(as_buf, 1, 1.f, acc);
    H::issue(a, in, as_buf, 1, tm, 3, tm);
    cp_wait<1>();
    H::template run<3, true>(as_buf, 0, wtp, acc);
    cp_wait<0>();
    H::template run<3, false>(as_buf, 1, wtm, acc);
    C<float> psi[12];
    load_spinor<float, float2>((const float2*)in, a.V, site, psi);
    const float kap = (float)a.kappa;
    C<float> o[12];
#pragma unroll
    for (int i = 0; i < 12; i++) {
        C<float> dd = psi[i] - kap * acc[i];
        o[i] = i < 6 ? dd : mk<float>(-dd.r, -dd.i);  // gamma_5 = diag(1,1,-1,-1)
    }
    store_spinor<float, float2>((float2*)a.out[r], a.V, site, o);
}

}  // namespace

int ovl_dslash_launch(ovl_lattice lat, const DslashArgs& d, int fmt, int links, cudaStream_t st) {
    KArgs a;
    a.in = d.in;
    a.out = d.out;
    a.mu = d.mu;
    a.active = d.active;
    a.klim = d.klim;
    a.stride = d.stride;
    a.j = d.j;
    a.Lx = lat->dims[0];
    a.Ly = lat->dims[1];
    a.Lz = lat->dims[2];
    a.Lt = lat->dims[3];
    a.V = lat->V;
    a.kappa = d.kappa;
    a.apbc = lat->apbc;
    a.u64 = lat->links.u64;
    a.u32q = lat->links.u32q;
    a.u32r = lat->links.u32r;
    a.u12 = lat->links.u12;
    // launch shape: the autotuner's choice for this format and link type (see
    // ovl_autotune), else 128 consecutive sites per CTA
    const OvlStenShape sh = lat->sten_shape[fmt == OVL_VEC_F64 ? 0 : 1][links & 3];
    a.tx = sh.tx;
    a.ty = sh.ty;
    a.tz = sh.tz;
    const unsigned ntile = sh.tx ? (unsigned)((lat->V / ((size_t)sh.tx * sh.ty * sh.tz))) : 0;
    dim3 grid(sh.tx ? ntile : (unsigned)((lat->V + 127) / 128), (unsigned)d.nrhs);
    const int tpb32 = sh.tx ? sh.tx * sh.ty * sh.tz : 128;
    if (fmt == OVL_VEC_F64) {
        // FP64 is bound by the FP64 pipe of each SM: on small launches one-warp
        // CTAs spread the work evenly over the SMs (measured at 8^4 with 8
        // right-hand sides: 62 us per launch with 32 threads, 70 us with 64 or 128)
        const int tpb = sh.tx ? tpb32 : sh.tpb ? sh.tpb
                                               : (lat->V * (size_t)d.nrhs < (size_t)1024 * lat->num_sms ? 32 : 128);
        dim3 g64(sh.tx ? ntile : (unsigned)((lat->V + tpb - 1) / tpb), (unsigned)d.nrhs);
        const bool t = sh.tx != 0;  // tiled variants are separate instantiations (no extra registers otherwise)
        if (links == OVL_LINKS_F64DF) {  // same shapes as FP64 (at 8^4 x 8 rhs: 81 us with 32 or 128 threads)
            if (t)
                k_dslash<dd, double2, OVL_LINKS_F64, true><<<g64, tpb, 0, st>>>(a);
            else
                k_dslash<dd, double2, OVL_LINKS_F64><<<g64, tpb, 0, st>>>(a);
        } else if (links == OVL_LINKS_F64) {
            if (t)
                k_dslash<double, double2, OVL_LINKS_F64, true><<<g64, tpb, 0, st>>>(a);
            else
                k_dslash<double, double2, OVL_LINKS_F64><<<g64, tpb, 0, st>>>(a);
        } else if (links == OVL_LINKS_F32) {
            k_dslash<float, double2, OVL_LINKS_F32><<<g64, tpb, 0, st>>>(a);
        } else {
            k_dslash<float, double2, OVL_LINKS_R12><<<g64, tpb, 0, st>>>(a);
        }
    } else {
        const bool t = sh.tx != 0;
        if (links == OVL_LINKS_F64 || links == OVL_LINKS_F64DF)
            return ovl_fail(lat, OVL_ENOTSUP, "F32 spinors with F64 links are not built");
        if (sh.async) {  // staged by cp.async (consecutive sites, 128 threads)
            const int items = links == OVL_LINKS_R12 ? AsyncHop<OVL_LINKS_R12>::ITEMS : AsyncHop<OVL_LINKS_F32>::ITEMS;
            const size_t smem = (size_t)2 * items * AS_T * sizeof(float4);
            if (!lat->sten_async_attr) {
                OVL_CUDA_TRY(lat, cudaFuncSetAttribute(k_dslash32a<OVL_LINKS_R12>,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024));
                OVL_CUDA_TRY(lat, cudaFuncSetAttribute(k_dslash32a<OVL_LINKS_F32>,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024));
                lat->sten_async_attr = true;
            }
            dim3 ga((unsigned)((lat->V + AS_T - 1) / AS_T), (unsigned)d.nrhs);
            if (links == OVL_LINKS_R12)
                k_dslash32a<OVL_LINKS_R12><<<ga, AS_T, smem, st>>>(a);
            else
                k_dslash32a<OVL_LINKS_F32><<<ga, AS_T, smem, st>>>(a);
            OVL_LAUNCH_CHECK(lat);
            return OVL_OK;
        }
        else if (links == OVL_LINKS_F32 && t)
            k_dslash32<float, float2, OVL_LINKS_F32, true><<<grid, tpb32, 0, st>>>(a);
        else if (links == OVL_LINKS_F32 && sh.minb == 6)
            k_dslash32<float, float2, OVL_LINKS_F32, false, 6><<<grid, tpb32, 0, st>>>(a);
        else if (links == OVL_LINKS_F32 && sh.minb == 4)
            k_dslash32<float, float2, OVL_LINKS_F32, false, 4><<<grid, tpb32, 0, st>>>(a);
        else if (links == OVL_LINKS_F32)
            k_dslash32<float, float2, OVL_LINKS_F32><<<grid, tpb32, 0, st>>>(a);
        else if (t)
            k_dslash32<float, float2, OVL_LINKS_R12, true><<<grid, tpb32, 0, st>>>(a);
        else if (sh.minb == 6)
            k_dslash32<float, float2, OVL_LINKS_R12, false, 6><<<grid, tpb32, 0, st>>>(a);
        else if (sh.minb == 4)
            k_dslash32<float, float2, OVL_LINKS_R12, false, 4><<<grid, tpb32, 0, st>>>(a);
        else
            k_dslash32<float, float2, OVL_LINKS_R12><<<grid, tpb32, 0, st>>>(a);
    }
    OVL_LAUNCH_CHECK(lat);
    return OVL_OK;
}
