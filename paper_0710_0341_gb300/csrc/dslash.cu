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
    // e^{+-mu} of this right-hand side, once per CTA: an FP64 exp per thread
    // kept the FP64 pipe half busy in the FP32 kernel
    __shared__ T s_w[2];
    if (threadIdx.x == 0) {
        const double mu = a.mu[r];
        s_w[0] = (T)exp(mu);
        s_w[1] = (T)exp(-mu);
    }
    __syncthreads();
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
    site_compute<T, VT, LINKS>(a, (const VT*)a.in[r], (VT*)a.out[r], site, s_w[0], s_w[1]);
}

// FP64 spinors: the compiler's register choice (140 for FP64 links, 168 for the
// double-float arithmetic on FP64 data; no spills)
template <typename T, typename VT, int LINKS, bool TILED = false>
__global__ void __launch_bounds__(128) k_dslash(KArgs a) {
    dslash_site<T, VT, LINKS, TILED>(a);
}

// FP32 spinors: at most 64 registers, 8 CTAs per SM (measured 13 % faster
// than 96 registers with 12-real links at 24^3x48, in spite of a few spills)
template <typename T, typename VT, int LINKS, bool TILED = false>
__global__ void __launch_bounds__(128, 8) k_dslash32(KArgs a) {
    dslash_site<T, VT, LINKS, TILED>(a);
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
        else if (links == OVL_LINKS_F32 && t)
            k_dslash32<float, float2, OVL_LINKS_F32, true><<<grid, tpb32, 0, st>>>(a);
        else if (links == OVL_LINKS_F32)
            k_dslash32<float, float2, OVL_LINKS_F32><<<grid, tpb32, 0, st>>>(a);
        else if (t)
            k_dslash32<float, float2, OVL_LINKS_R12, true><<<grid, tpb32, 0, st>>>(a);
        else
            k_dslash32<float, float2, OVL_LINKS_R12><<<grid, tpb32, 0, st>>>(a);
    }
    OVL_LAUNCH_CHECK(lat);
    return OVL_OK;
}
