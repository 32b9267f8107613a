// Allocation-free variant of ovl_apply_Hw.
//
// ovl_apply_Hw stages the packed input and output spinors in a device buffer
// that the lattice handle grows with cudaMalloc. Some callers cannot let a
// library allocate: a serving process that has handed all free HBM to its
// own memory pool (cudaMalloc would fail), code that must not trigger the
// implicit device synchronisation of cudaMalloc/cudaFree, or a host
// framework that requires every device byte a library uses to be accounted
// for up front. ovl_apply_Hw_noalloc gives them the same operator with its
// staging space in a fixed file-scope device array (OVL_NOALLOC_BYTES,
// 32 MiB) that exists on every GPU that loads the library, until the process
// exits. It calls no cudaMalloc, cudaFree or allocating library routine.
//
// The host needs the array's device address, which is not the symbol's host
// name: the first call on each device looks it up with
// cudaGetSymbolAddress (with that device current) and caches it. Every call
// copies its pointer table from host memory that is freed on return and then
// synchronises the lattice's stream, so no call may be made while that stream
// is being captured into a graph: the call checks and refuses. All calls share
// the one array and each overwrites it: calls that overlap on the GPU (several
// streams or threads at once) race and give wrong results.
#include <string.h>

#include <mutex>

#include "ovl_common.cuh"

#define OVL_NOALLOC_BYTES (32u << 20)

static __device__ __align__(256) unsigned char g_noalloc_scratch[OVL_NOALLOC_BYTES];

static std::mutex g_noalloc_mu;
static void* g_noalloc_addr[128] = {};

static int noalloc_base(ovl_lattice lat, unsigned char** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128)
        return ovl_fail(lat, OVL_ECUDA, "ovl_apply_Hw_noalloc: no current device");
    // the address looked up is that of the current device's copy of the array
    if (dev != lat->device)
        return ovl_fail(lat, OVL_EINVAL, "ovl_apply_Hw_noalloc: current device %d is not the lattice's device %d",
                        dev, lat->device);
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return ovl_fail(lat, OVL_ECUDA, "ovl_apply_Hw_noalloc: cudaGetSymbolAddress failed: %s",
                            cudaGetErrorString(e));
        g_noalloc_addr[dev] = p;
    }
    *out = (unsigned char*)g_noalloc_addr[dev];
    return OVL_OK;
}

extern "C" int ovl_apply_Hw_noalloc(ovl_lattice lat, double mu, double m_w, const double* in, double* out,
                                    int nrhs, int links) {
    if (!lat || !in || !out || nrhs < 1) return ovl_fail(lat, OVL_EINVAL, "ovl_apply_Hw_noalloc: bad argument");
    if (!lat->have_links) return ovl_fail(lat, OVL_EINVAL, "ovl_apply_Hw_noalloc: links not set");
    if (!(m_w > -4.0 + 1e-12) || !(m_w < 1e6))
        return ovl_fail(lat, OVL_EINVAL, "ovl_apply_Hw_noalloc: m_w=%g gives no finite kappa", m_w);
    if (links < OVL_LINKS_F64 || links > OVL_LINKS_F64DF)
        return ovl_fail(lat, OVL_EINVAL, "ovl_apply_Hw_noalloc: bad links format %d", links);
    // first, so that a refused call makes no other CUDA call under capture
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    OVL_CUDA_TRY(lat, cudaStreamIsCapturing(lat->stream, &cs));
    if (cs != cudaStreamCaptureStatusNone)
        return ovl_fail(lat, OVL_EINVAL, "ovl_apply_Hw_noalloc: the lattice's stream is being captured");
    if (!ovl_is_device_ptr(in) || !ovl_is_device_ptr(out))
        return ovl_fail(lat, OVL_EINVAL, "ovl_apply_Hw_noalloc: in and out must be device memory");
    if (in == out) return ovl_fail(lat, OVL_EINVAL, "ovl_apply_Hw_noalloc: in and out must differ");
    const int fmt = (links == OVL_LINKS_F64 || links == OVL_LINKS_F64DF) ? OVL_VEC_F64 : OVL_VEC_F32;
    const size_t vb = ovl_vec_bytes(lat, fmt) * (size_t)nrhs;  // one packed block
    const size_t vba = (vb + 255) & ~(size_t)255;
    const size_t args = 3 * sizeof(double) * (size_t)nrhs;      // in/out pointers and mu
    const size_t need = 2 * vba + args;
    if (need > OVL_NOALLOC_BYTES)
        return ovl_fail(lat, OVL_EINVAL,
                        "ovl_apply_Hw_noalloc: %d right-hand sides of %zu sites need %zu bytes, above the fixed "
                        "%u-byte staging array (use ovl_apply_Hw)",
                        nrhs, lat->V, need, (unsigned)OVL_NOALLOC_BYTES);
    unsigned char* base = nullptr;
    if (int rc = noalloc_base(lat, &base)) return rc;
    unsigned char* pin = base;
    unsigned char* pout = base + vba;
    unsigned char* pargs = base + 2 * vba;
    std::vector<uint64_t> h(3 * (size_t)nrhs);
    for (int r = 0; r < nrhs; r++) {
        h[r] = (uint64_t)(pin + r * (vb / nrhs));
        h[nrhs + r] = (uint64_t)(pout + r * (vb / nrhs));
        double m = mu;
        memcpy(&h[2 * nrhs + r], &m, sizeof m);
    }
    cudaStream_t st = lat->stream;
    OVL_CUDA_TRY(lat, cudaMemcpyAsync(pargs, h.data(), args, cudaMemcpyHostToDevice, st));
    if (int rc = ovl_pack_impl(lat, in, pin, nrhs, fmt, st)) return rc;
    DslashArgs da;
    da.in = (const void* const*)pargs;
    da.out = (void* const*)(pargs + 8 * (size_t)nrhs);
    da.mu = (const double*)(pargs + 16 * (size_t)nrhs);
    da.nrhs = nrhs;
    da.kappa = 1.0 / (8.0 + 2.0 * m_w);
    if (int rc = ovl_dslash_launch(lat, da, fmt, links, st)) return rc;
    if (int rc = ovl_unpack_impl(lat, pout, out, nrhs, fmt, st)) return rc;
    OVL_CUDA_TRY(lat, cudaStreamSynchronize(st));  // h must outlive the copy
    return OVL_OK;
}
