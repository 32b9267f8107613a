// Internal declarations shared by the CUDA translation units of libovl.
// Not part of the public ABI (include/ovl.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string>
#include <vector>

#include "../../include/ovl.h"

#define OVL_PROF_CLASSES 8

// ---------------------------------------------------------------------------
// Packed spinor order used on the device.
//
// A spinor field has N = 12 V complex entries (spin s, colour c; component
// index cc = 3 s + c). The device keeps them component-pair major:
//     pos(cc, site) = ((cc >> 1) * V + site) * 2 + (cc & 1)      (complex units)
// so a thread handling one site reads each pair (cc, cc+1) as one contiguous
// 16-byte (complex64) or 32-byte (complex128) chunk and a warp of consecutive
// sites reads contiguous memory. Every Krylov vector, deflation vector and
// work vector uses this order; inner products do not depend on it.
// ---------------------------------------------------------------------------
__host__ __device__ inline size_t ovl_pos(int cc, size_t site, size_t V) {
    return ((size_t)(cc >> 1) * V + site) * 2 + (cc & 1);
}

// Links on the device (V sites, 4 directions):
//  F64 : double2 U64[(nu*9 + e)*V + site], e = 3a + b
//  F32 : float4  U32q[(nu*4 + p)*V + site] holds entries (2p, 2p+1), p < 4,
//        float2  U32r[nu*V + site] holds entry 8
//  R12 : float4  U12[(nu*3 + p)*V + site] holds entries (2p, 2p+1) of rows 0,1
struct LinkSet {
    double2* u64 = nullptr;
    float4*  u32q = nullptr;
    float2*  u32r = nullptr;
    float4*  u12 = nullptr;
};

// Stencil launch shape: tx x ty x tz sites per CTA (tx = 0: consecutive
// sites, tpb threads per CTA, tpb = 0: the built-in rule)
struct OvlStenShape {
    int tpb = 0, tx = 0, ty = 0, tz = 0;
    int async = 0;  // FP32: neighbour data staged in shared memory by cp.async
    int minb = 0;   // FP32, consecutive sites: resident CTAs the registers are capped for (0: 8, or 6 or 4)
};

struct ovl_lattice_s {
    int dims[4];       // Lx, Ly, Lz, Lt
    int apbc;          // antiperiodic in t
    size_t V, N;       // sites, complex entries per spinor (12 V)
    cudaStream_t stream;
    int device;
    LinkSet links;
    bool have_links = false;
    unsigned long long link_hash = 0;  // fingerprint of the FP64 links (ovl_set_links)
    std::string err;
    // device status word for kernels that can time out or fail (int[64])
    int* d_status = nullptr;
    // scratch reused across calls (grown on demand)
    void* scratch = nullptr;
    size_t scratch_bytes = 0;
    // workspace of ovl_sign_apply (Krylov bases, small matrices), grown on demand
    void* ws = nullptr;
    size_t ws_bytes = 0;
    int num_sms = 0;
    // per-device launch facts of this lattice's device, found on first use
    int gs_dot_occ = 0;            // resident pass-A CTAs per SM
    bool gs_update_attr = false;   // pass B may take more than 48 KB of shared memory
    bool gs_update64_attr = false; // the same for the FP64 pass B
    bool gs_bulk_attr = false;     // the same for the bulk-copy pass B (its stage ring)
    int pass_b_bulk = 0;           // 1: pass B streams the basis by bulk copies where it can (ovl_set_pass_b)
    // stencil launch shapes per [spinor format F64/F32][link type], set by ovl_autotune
    OvlStenShape sten_shape[2][4];
    bool sten_async_attr = false;  // the staged FP32 kernels may take 64 KB of shared memory
    // CUDA graph of the fixed-depth Arnoldi loop of ovl_sign_apply (ovl_set_graphs)
    bool graphs = false;
    cudaStream_t cap_stream = nullptr;  // private stream the loop is captured on
    cudaGraphExec_t graph_exec = nullptr;
    uint64_t graph_key = 0, graph_seen = 0;
    long long graph_kernels = 0, graph_replays = 0;
    // kernels launched by this handle, and optional per-class event timing
    long long launches = 0;
    bool prof = false;
    double prof_acc[OVL_PROF_CLASSES][3] = {};  // launches, ms, algorithmic bytes
    struct ProfRec {
        int cls;
        cudaEvent_t a, b;
        double bytes;
    };
    std::vector<ProfRec> prof_pending;
    std::vector<cudaEvent_t> event_pool;
};

// event-timed region of one kernel class (no-op unless profiling is on)
struct ProfScope {
    ovl_lattice lat;
    int cls;
    double bytes;
    cudaEvent_t a = nullptr, b = nullptr;
    ProfScope(ovl_lattice l, int c, double by, cudaStream_t st);
    void end(cudaStream_t st);
};
void ovl_prof_flush(ovl_lattice lat);

struct ovl_deflation_s {
    ovl_lattice lat;
    int scheme, m;
    double mu, m_w;
    // packed vectors stored as FP32 hi / lo planes (complex64 each), m columns
    float2* S_hi = nullptr;   // Schur: S; LR: R
    float2* S_lo = nullptr;
    float2* L_hi = nullptr;   // LR only
    float2* L_lo = nullptr;
    // complex128 copies for the plain FP64 form: exact for imported vectors,
    // built from hi + lo on first use otherwise
    double2* S64 = nullptr;
    double2* L64 = nullptr;
    double2* T = nullptr;     // Schur: m x m column-major (device); LR: Lambda (m)
    std::vector<double> T_host;  // same data on the host (2*m*m or 2*m doubles)
    int setup_restarts = 0;      // restarts and operator applications of ovl_deflation_setup
    int setup_matvecs = 0;
};

// ---------------------------------------------------------------------------
// Error plumbing
// ---------------------------------------------------------------------------
int ovl_fail(ovl_lattice lat, int code, const char* fmt, ...);
// a failed call's error is also taken off the runtime's last-error slot, so
// that it is not reported again by the next launch check
#define OVL_CUDA_TRY(lat, call)                                                      \
    do {                                                                             \
        cudaError_t e__ = (call);                                                    \
        if (e__ != cudaSuccess) {                                                    \
            cudaGetLastError();                                                      \
            return ovl_fail((lat), OVL_ECUDA, "%s failed: %s (%s:%d)", #call,         \
                            cudaGetErrorString(e__), __FILE__, __LINE__);            \
        }                                                                            \
    } while (0)
#define OVL_LAUNCH_CHECK(lat)                                                        \
    do {                                                                             \
        cudaError_t e__ = cudaGetLastError();                                        \
        if (e__ != cudaSuccess)                                                      \
            return ovl_fail((lat), OVL_ECUDA, "kernel launch failed: %s (%s:%d)",    \
                            cudaGetErrorString(e__), __FILE__, __LINE__);            \
        (lat)->launches++;                                                           \
    } while (0)

// Is p a device (or managed) pointer?
bool ovl_is_device_ptr(const void* p);

// Scratch memory owned by the lattice, grown on demand (never shrinks).
int ovl_scratch(ovl_lattice lat, size_t bytes, void** out);

// ---------------------------------------------------------------------------
// Complex helpers
// ---------------------------------------------------------------------------
__host__ __device__ inline double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ inline double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ inline double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ inline double2 cconjmul(double2 a, double2 b) {  // conj(a) * b
    return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__host__ __device__ inline double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__host__ __device__ inline double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }
__host__ __device__ inline double2 cinv(double2 a) {
    double d = 1.0 / cabs2(a);
    return make_double2(a.x * d, -a.y * d);
}

// Launch helpers (defined in the respective .cu files) -----------------------
int ovl_pack_impl(ovl_lattice lat, const double* canon_dev, void* packed, int nrhs, int fmt, cudaStream_t st);
int ovl_unpack_impl(ovl_lattice lat, const void* packed, double* canon_dev, int nrhs, int fmt, cudaStream_t st);

// Stencil over a batch: out_r = H_w(mu_r) in_r for r < nrhs.
// fmt: OVL_VEC_F64 / OVL_VEC_F32 for both in and out; links: OVL_LINKS_*.
// in/out are arrays (device) of nrhs pointers; mu is a device array of nrhs
// doubles; active (device, nrhs ints, may be null) skips rhs with active[r]==0.
// active/klim (optional) skip rhs r when active[r*stride] == 0 or
// j > klim[r*stride] (they may point into an array of larger records).
struct DslashArgs {
    const void* const* in;
    void* const* out;
    const double* mu;
    const int* active = nullptr;
    const int* klim = nullptr;
    int stride = 1;
    int j = 0;
    int nrhs;
    double kappa;
};
int ovl_dslash_launch(ovl_lattice lat, const DslashArgs& a, int fmt, int links, cudaStream_t st);

// Packed-vector device memory for n vectors of 12 V complex (format fmt).
size_t ovl_vec_bytes(ovl_lattice lat, int fmt);
