// Lattice handle, links upload, packed/canonical spinor conversion and the
// operator entry points of the C ABI (Sec. 1, Eq. 2).
#include <stdarg.h>
#include <string.h>

#include "ovl_common.cuh"

static thread_local std::string g_noh_err;

int ovl_fail(ovl_lattice lat, int code, const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (lat)
        lat->err = buf;
    else
        g_noh_err = buf;
    return code;
}

bool ovl_is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int ovl_scratch(ovl_lattice lat, size_t bytes, void** out) {
    if (bytes > lat->scratch_bytes) {
        if (lat->scratch) {
            cudaStreamSynchronize(lat->stream);
            cudaFree(lat->scratch);
            lat->scratch = nullptr;
            lat->scratch_bytes = 0;
        }
        size_t nb = bytes + bytes / 4 + 4096;
        if (cudaMalloc(&lat->scratch, nb) != cudaSuccess) {
            cudaGetLastError();
            return ovl_fail(lat, OVL_ENOMEM, "scratch allocation of %zu bytes failed", nb);
        }
        lat->scratch_bytes = nb;
    }
    *out = lat->scratch;
    return OVL_OK;
}

size_t ovl_vec_bytes(ovl_lattice lat, int fmt) {
    return lat->N * (fmt == OVL_VEC_F64 ? sizeof(double2) : sizeof(float2));
}

extern "C" const char* ovl_last_error(ovl_lattice lat) {
    return lat ? lat->err.c_str() : g_noh_err.c_str();
}

extern "C" const char* ovl_version(void) { return "ovl 0.1.0 sm_103a"; }

extern "C" int ovl_create_lattice(const int dims[4], int antiperiodic_t, void* stream, ovl_lattice* out) {
    if (!dims || !out) return ovl_fail(nullptr, OVL_EINVAL, "ovl_create_lattice: null argument");
    for (int i = 0; i < 4; i++)
        if (dims[i] < 2 || dims[i] > 4096)
            return ovl_fail(nullptr, OVL_EINVAL, "ovl_create_lattice: dims[%d]=%d out of [2,4096]", i, dims[i]);
    size_t V = (size_t)dims[0] * dims[1] * dims[2] * dims[3];
    if (V > (size_t)1 << 28) return ovl_fail(nullptr, OVL_EINVAL, "ovl_create_lattice: volume %zu too large", V);
    ovl_lattice L = new ovl_lattice_s();
    for (int i = 0; i < 4; i++) L->dims[i] = dims[i];
    L->apbc = antiperiodic_t ? 1 : 0;
    L->V = V;
    L->N = 12 * V;
    L->stream = (cudaStream_t)stream;
    if (cudaGetDevice(&L->device) != cudaSuccess) {
        cudaGetLastError();
        delete L;
        return ovl_fail(nullptr, OVL_ECUDA, "ovl_create_lattice: no CUDA device");
    }
    cudaDeviceGetAttribute(&L->num_sms, cudaDevAttrMultiProcessorCount, L->device);
    if (cudaMalloc(&L->d_status, 64 * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        delete L;
        return ovl_fail(nullptr, OVL_ENOMEM, "ovl_create_lattice: status word allocation failed");
    }
    cudaMemset(L->d_status, 0, 64 * sizeof(int));
    *out = L;
    return OVL_OK;
}

static void free_links(LinkSet& s) {
    cudaFree(s.u64);
    cudaFree(s.u32q);
    cudaFree(s.u32r);
    cudaFree(s.u12);
    s = LinkSet();
}

extern "C" int ovl_destroy_lattice(ovl_lattice lat) {
    if (!lat) return OVL_OK;
    cudaStreamSynchronize(lat->stream);
    if (lat->graph_exec) cudaGraphExecDestroy(lat->graph_exec);
    if (lat->cap_stream) cudaStreamDestroy(lat->cap_stream);
    free_links(lat->links);
    ovl_prof_flush(lat);
    for (cudaEvent_t e : lat->event_pool) cudaEventDestroy(e);
    cudaFree(lat->scratch);
    cudaFree(lat->ws);
    cudaFree(lat->d_status);
    delete lat;
    return OVL_OK;
}

// canonical U[site][nu][a][b] complex128 -> the three device formats
__global__ void k_links_convert(const double2* __restrict__ Uc, size_t V, double2* __restrict__ u64,
                                float4* __restrict__ u32q, float2* __restrict__ u32r, float4* __restrict__ u12) {
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= V * 4) return;
    size_t site = i >> 2;
    int nu = (int)(i & 3);
    const double2* src = Uc + (site * 4 + nu) * 9;
    double2 e[9];
#pragma unroll
    for (int k = 0; k < 9; k++) e[k] = src[k];
#pragma unroll
    for (int k = 0; k < 9; k++) u64[((size_t)nu * 9 + k) * V + site] = e[k];
#pragma unroll
    for (int p = 0; p < 4; p++)
        u32q[((size_t)nu * 4 + p) * V + site] =
            make_float4((float)e[2 * p].x, (float)e[2 * p].y, (float)e[2 * p + 1].x, (float)e[2 * p + 1].y);
    u32r[(size_t)nu * V + site] = make_float2((float)e[8].x, (float)e[8].y);
#pragma unroll
    for (int p = 0; p < 3; p++)
        u12[((size_t)nu * 3 + p) * V + site] =
            make_float4((float)e[2 * p].x, (float)e[2 * p].y, (float)e[2 * p + 1].x, (float)e[2 * p + 1].y);
}

// 64-bit fingerprint of the FP64 link field: the sum (mod 2^64) over its
// doubles of a SplitMix64 mix of (bits + index * golden ratio), so that the
// same field gives the same value on any launch shape; used to tie saved
// deflation data to the links they were computed for.
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}
__global__ void k_link_hash(const double* __restrict__ u, size_t n, unsigned long long* out) {
    unsigned long long acc = 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        acc += mix64((unsigned long long)__double_as_longlong(u[i]) + i * 0x9e3779b97f4a7c15ull);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, acc);
}

extern "C" int ovl_set_links(ovl_lattice lat, const double* U) {
    if (!lat || !U) return ovl_fail(lat, OVL_EINVAL, "ovl_set_links: null argument");
    size_t V = lat->V;
    size_t bytes = V * 4 * 9 * sizeof(double2);
    if (!lat->links.u64) {
        LinkSet s;
        bool ok = cudaMalloc(&s.u64, bytes) == cudaSuccess && cudaMalloc(&s.u32q, V * 16 * sizeof(float4)) == cudaSuccess &&
                  cudaMalloc(&s.u32r, V * 4 * sizeof(float2)) == cudaSuccess &&
                  cudaMalloc(&s.u12, V * 12 * sizeof(float4)) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            free_links(s);
            return ovl_fail(lat, OVL_ENOMEM, "ovl_set_links: link allocation failed");
        }
        lat->links = s;
    }
    const double2* src = (const double2*)U;
    double2* tmp = nullptr;
    if (!ovl_is_device_ptr(U)) {
        void* p;
        int rc = ovl_scratch(lat, bytes, &p);
        if (rc) return rc;
        tmp = (double2*)p;
        OVL_CUDA_TRY(lat, cudaMemcpyAsync(tmp, U, bytes, cudaMemcpyHostToDevice, lat->stream));
        src = tmp;
    }
    unsigned nb = (unsigned)((V * 4 + 255) / 256);
    k_links_convert<<<nb, 256, 0, lat->stream>>>(src, V, lat->links.u64, lat->links.u32q, lat->links.u32r,
                                                  lat->links.u12);
    OVL_LAUNCH_CHECK(lat);
    {
        void* p;
        if (int rc = ovl_scratch(lat, bytes + sizeof(unsigned long long), &p)) return rc;
        unsigned long long* hd = (unsigned long long*)((char*)p + bytes);  // after the staged links
        OVL_CUDA_TRY(lat, cudaMemsetAsync(hd, 0, sizeof *hd, lat->stream));
        k_link_hash<<<(unsigned)lat->num_sms * 4, 256, 0, lat->stream>>>((const double*)lat->links.u64, V * 4 * 18, hd);
        OVL_LAUNCH_CHECK(lat);
        OVL_CUDA_TRY(lat, cudaMemcpyAsync(&lat->link_hash, hd, sizeof *hd, cudaMemcpyDeviceToHost, lat->stream));
    }
    OVL_CUDA_TRY(lat, cudaStreamSynchronize(lat->stream));
    lat->have_links = true;
    return OVL_OK;
}

// ---------------------------------------------------------------------------
// canonical (site-major, 12 complex per site) <-> packed (component-pair major)
// ---------------------------------------------------------------------------
template <typename VT>
__global__ void k_pack(const double2* __restrict__ canon, VT* __restrict__ packed, size_t V, int nrhs) {
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= V * 6 * (size_t)nrhs) return;
    size_t r = i / (V * 6);
    size_t rem = i - r * V * 6;
    int cp = (int)(rem / V);
    size_t site = rem - (size_t)cp * V;
    const double2* src = canon + r * 12 * V + site * 12 + 2 * cp;
    VT* dst = packed + r * 12 * V + ((size_t)cp * V + site) * 2;
    double2 a = src[0], b = src[1];
    if constexpr (sizeof(VT) == sizeof(double2)) {
        dst[0] = a;
        dst[1] = b;
    } else {
        *(float4*)dst = make_float4((float)a.x, (float)a.y, (float)b.x, (float)b.y);
    }
}

template <typename VT>
__global__ void k_unpack(const VT* __restrict__ packed, double2* __restrict__ canon, size_t V, int nrhs) {
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= V * 6 * (size_t)nrhs) return;
    size_t r = i / (V * 6);
    size_t rem = i - r * V * 6;
    int cp = (int)(rem / V);
    size_t site = rem - (size_t)cp * V;
    double2* dst = canon + r * 12 * V + site * 12 + 2 * cp;
    const VT* src = packed + r * 12 * V + ((size_t)cp * V + site) * 2;
    if constexpr (sizeof(VT) == sizeof(double2)) {
        dst[0] = src[0];
        dst[1] = src[1];
    } else {
        float4 v = *(const float4*)src;
        dst[0] = make_double2(v.x, v.y);
        dst[1] = make_double2(v.z, v.w);
    }
}

int ovl_pack_impl(ovl_lattice lat, const double* canon_dev, void* packed, int nrhs, int fmt, cudaStream_t st) {
    size_t n = lat->V * 6 * (size_t)nrhs;
    unsigned nb = (unsigned)((n + 255) / 256);
    if (fmt == OVL_VEC_F64)
        k_pack<double2><<<nb, 256, 0, st>>>((const double2*)canon_dev, (double2*)packed, lat->V, nrhs);
    else
        k_pack<float2><<<nb, 256, 0, st>>>((const double2*)canon_dev, (float2*)packed, lat->V, nrhs);
    OVL_LAUNCH_CHECK(lat);
    return OVL_OK;
}

int ovl_unpack_impl(ovl_lattice lat, const void* packed, double* canon_dev, int nrhs, int fmt, cudaStream_t st) {
    size_t n = lat->V * 6 * (size_t)nrhs;
    unsigned nb = (unsigned)((n + 255) / 256);
    if (fmt == OVL_VEC_F64)
        k_unpack<double2><<<nb, 256, 0, st>>>((const double2*)packed, (double2*)canon_dev, lat->V, nrhs);
    else
        k_unpack<float2><<<nb, 256, 0, st>>>((const float2*)packed, (double2*)canon_dev, lat->V, nrhs);
    OVL_LAUNCH_CHECK(lat);
    return OVL_OK;
}

static int check_fmt(ovl_lattice lat, int fmt) {
    if (fmt != OVL_VEC_F64 && fmt != OVL_VEC_F32) return ovl_fail(lat, OVL_EINVAL, "bad spinor format %d", fmt);
    return OVL_OK;
}

extern "C" int ovl_pack_spinor(ovl_lattice lat, const double* canon, void* packed, int nrhs, int fmt) {
    if (!lat || !canon || !packed || nrhs < 1) return ovl_fail(lat, OVL_EINVAL, "ovl_pack_spinor: bad argument");
    if (int rc = check_fmt(lat, fmt)) return rc;
    if (!ovl_is_device_ptr(packed)) return ovl_fail(lat, OVL_EINVAL, "ovl_pack_spinor: packed must be device memory");
    size_t cb = lat->N * sizeof(double2) * nrhs;
    const double* src = canon;
    if (!ovl_is_device_ptr(canon)) {
        void* p;
        if (int rc = ovl_scratch(lat, cb, &p)) return rc;
        OVL_CUDA_TRY(lat, cudaMemcpyAsync(p, canon, cb, cudaMemcpyHostToDevice, lat->stream));
        src = (const double*)p;
    }
    if (int rc = ovl_pack_impl(lat, src, packed, nrhs, fmt, lat->stream)) return rc;
    OVL_CUDA_TRY(lat, cudaStreamSynchronize(lat->stream));
    return OVL_OK;
}

extern "C" int ovl_unpack_spinor(ovl_lattice lat, const void* packed, double* canon, int nrhs, int fmt) {
    if (!lat || !canon || !packed || nrhs < 1) return ovl_fail(lat, OVL_EINVAL, "ovl_unpack_spinor: bad argument");
    if (int rc = check_fmt(lat, fmt)) return rc;
    if (!ovl_is_device_ptr(packed)) return ovl_fail(lat, OVL_EINVAL, "ovl_unpack_spinor: packed must be device memory");
    size_t cb = lat->N * sizeof(double2) * nrhs;
    if (ovl_is_device_ptr(canon)) {
        if (int rc = ovl_unpack_impl(lat, packed, canon, nrhs, fmt, lat->stream)) return rc;
    } else {
        void* p;
        if (int rc = ovl_scratch(lat, cb, &p)) return rc;
        if (int rc = ovl_unpack_impl(lat, packed, (double*)p, nrhs, fmt, lat->stream)) return rc;
        OVL_CUDA_TRY(lat, cudaMemcpyAsync(canon, p, cb, cudaMemcpyDeviceToHost, lat->stream));
    }
    OVL_CUDA_TRY(lat, cudaStreamSynchronize(lat->stream));
    return OVL_OK;
}

static int check_mw(ovl_lattice lat, double m_w) {
    if (!(m_w > -4.0 + 1e-12) || !(m_w < 1e6)) return ovl_fail(lat, OVL_EINVAL, "m_w=%g gives no finite kappa", m_w);
    return OVL_OK;
}

// stencil on packed device vectors; builds the pointer / mu arrays in scratch
static int dslash_packed(ovl_lattice lat, const double* mu_host, double m_w, const void* in, void* out, int nrhs,
                         int fmt, int links, void* argspace) {
    size_t vb = ovl_vec_bytes(lat, fmt);
    std::vector<const void*> pin(nrhs);
    std::vector<void*> pout(nrhs);
    for (int r = 0; r < nrhs; r++) {
        pin[r] = (const char*)in + r * vb;
        pout[r] = (char*)out + r * vb;
    }
    char* a = (char*)argspace;
    OVL_CUDA_TRY(lat, cudaMemcpyAsync(a, pin.data(), nrhs * sizeof(void*), cudaMemcpyHostToDevice, lat->stream));
    OVL_CUDA_TRY(lat, cudaMemcpyAsync(a + 8 * nrhs, pout.data(), nrhs * sizeof(void*), cudaMemcpyHostToDevice,
                                      lat->stream));
    OVL_CUDA_TRY(lat, cudaMemcpyAsync(a + 16 * nrhs, mu_host, nrhs * sizeof(double), cudaMemcpyHostToDevice,
                                      lat->stream));
    DslashArgs da;
    da.in = (const void* const*)a;
    da.out = (void* const*)(a + 8 * nrhs);
    da.mu = (const double*)(a + 16 * nrhs);
    da.active = nullptr;
    da.nrhs = nrhs;
    da.kappa = 1.0 / (8.0 + 2.0 * m_w);
    const double sb = fmt == OVL_VEC_F64 ? 16.0 : 8.0;
    const double lb = (links == OVL_LINKS_F64 || links == OVL_LINKS_F64DF) ? 144.0 : links == OVL_LINKS_F32 ? 72.0 : 48.0;
    ProfScope ps(lat, 0, nrhs * (double)lat->V * (24.0 * sb + 4.0 * lb), lat->stream);
    int rc = ovl_dslash_launch(lat, da, fmt, links, lat->stream);
    ps.end(lat->stream);
    // the host vectors above must outlive the async copies
    cudaStreamSynchronize(lat->stream);
    return rc;
}

extern "C" int ovl_apply_Hw_packed(ovl_lattice lat, const double* mu, double m_w, const void* in, void* out, int nrhs,
                                   int fmt, int links) {
    if (!lat || !mu || !in || !out || nrhs < 1) return ovl_fail(lat, OVL_EINVAL, "ovl_apply_Hw_packed: bad argument");
    if (!lat->have_links) return ovl_fail(lat, OVL_EINVAL, "ovl_apply_Hw_packed: links not set");
    if (int rc = check_fmt(lat, fmt)) return rc;
    if (int rc = check_mw(lat, m_w)) return rc;
    if (links < OVL_LINKS_F64 || links > OVL_LINKS_F64DF) return ovl_fail(lat, OVL_EINVAL, "bad links format %d", links);
    if ((fmt == OVL_VEC_F64) != (links == OVL_LINKS_F64 || links == OVL_LINKS_F64DF))
        return ovl_fail(lat, OVL_EINVAL, "ovl_apply_Hw_packed: F64 vectors go with F64/F64DF links, F32 with F32/R12");
    if (!ovl_is_device_ptr(in) || !ovl_is_device_ptr(out))
        return ovl_fail(lat, OVL_EINVAL, "ovl_apply_Hw_packed: in/out must be device memory");
    if (in == out) return ovl_fail(lat, OVL_EINVAL, "ovl_apply_Hw_packed: in and out must differ");
    void* args;
    if (int rc = ovl_scratch(lat, 32 * (size_t)nrhs + 256, &args)) return rc;
    return dslash_packed(lat, mu, m_w, in, out, nrhs, fmt, links, args);
}

extern "C" int ovl_apply_Hw(ovl_lattice lat, double mu, double m_w, const double* in, double* out, int nrhs,
                            int links) {
    if (!lat || !in || !out || nrhs < 1) return ovl_fail(lat, OVL_EINVAL, "ovl_apply_Hw: bad argument");
    if (!lat->have_links) return ovl_fail(lat, OVL_EINVAL, "ovl_apply_Hw: links not set");
    if (int rc = check_mw(lat, m_w)) return rc;
    if (links < OVL_LINKS_F64 || links > OVL_LINKS_F64DF) return ovl_fail(lat, OVL_EINVAL, "bad links format %d", links);
    int fmt = (links == OVL_LINKS_F64 || links == OVL_LINKS_F64DF) ? OVL_VEC_F64 : OVL_VEC_F32;
    size_t cb = lat->N * sizeof(double2) * nrhs;  // canonical bytes
    size_t pb = ovl_vec_bytes(lat, fmt) * nrhs;   // packed bytes
    size_t off_in = 0, off_pin = cb, off_pout = off_pin + pb, off_args = off_pout + pb;
    size_t total = off_args + 32 * (size_t)nrhs + 256;
    void* s;
    if (int rc = ovl_scratch(lat, total, &s)) return rc;
    char* base = (char*)s;
    const double* cin = in;
    if (!ovl_is_device_ptr(in)) {
        OVL_CUDA_TRY(lat, cudaMemcpyAsync(base + off_in, in, cb, cudaMemcpyHostToDevice, lat->stream));
        cin = (const double*)(base + off_in);
    }
    if (int rc = ovl_pack_impl(lat, cin, base + off_pin, nrhs, fmt, lat->stream)) return rc;
    std::vector<double> mus(nrhs, mu);
    if (int rc = dslash_packed(lat, mus.data(), m_w, base + off_pin, base + off_pout, nrhs, fmt, links,
                               base + off_args))
        return rc;
    if (ovl_is_device_ptr(out)) {
        if (int rc = ovl_unpack_impl(lat, base + off_pout, out, nrhs, fmt, lat->stream)) return rc;
    } else {
        if (int rc = ovl_unpack_impl(lat, base + off_pout, (double*)(base + off_in), nrhs, fmt, lat->stream)) return rc;
        OVL_CUDA_TRY(lat, cudaMemcpyAsync(out, base + off_in, cb, cudaMemcpyDeviceToHost, lat->stream));
    }
    OVL_CUDA_TRY(lat, cudaStreamSynchronize(lat->stream));
    return OVL_OK;
}

// ---------------------------------------------------------------------------
// kernel accounting
// ---------------------------------------------------------------------------
static cudaEvent_t take_event(ovl_lattice lat) {
    if (!lat->event_pool.empty()) {
        cudaEvent_t e = lat->event_pool.back();
        lat->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

ProfScope::ProfScope(ovl_lattice l, int c, double by, cudaStream_t st) : lat(l), cls(c), bytes(by) {
    if (!lat->prof) return;
    a = take_event(lat);
    b = take_event(lat);
    cudaEventRecord(a, st);
}

void ProfScope::end(cudaStream_t st) {
    if (!lat->prof || !a) return;
    cudaEventRecord(b, st);
    lat->prof_pending.push_back({cls, a, b, bytes});
    a = b = nullptr;
}

void ovl_prof_flush(ovl_lattice lat) {
    if (lat->prof_pending.empty()) return;
    cudaStreamSynchronize(lat->stream);
    for (auto& r : lat->prof_pending) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, r.a, r.b);
        lat->prof_acc[r.cls][0] += 1;
        lat->prof_acc[r.cls][1] += ms;
        lat->prof_acc[r.cls][2] += r.bytes;
        lat->event_pool.push_back(r.a);
        lat->event_pool.push_back(r.b);
    }
    lat->prof_pending.clear();
}

extern "C" int ovl_launch_count(ovl_lattice lat, long long* n) {
    if (!lat || !n) return ovl_fail(lat, OVL_EINVAL, "ovl_launch_count: null argument");
    *n = lat->launches;
    return OVL_OK;
}

extern "C" int ovl_profile(ovl_lattice lat, int enable, double* stats) {
    if (!lat) return ovl_fail(lat, OVL_EINVAL, "ovl_profile: null handle");
    ovl_prof_flush(lat);
    if (stats)
        for (int c = 0; c < OVL_PROF_CLASSES; c++)
            for (int k = 0; k < 3; k++) stats[3 * c + k] = lat->prof_acc[c][k];
    if (enable) {
        for (int c = 0; c < OVL_PROF_CLASSES; c++)
            for (int k = 0; k < 3; k++) lat->prof_acc[c][k] = 0.0;
    }
    lat->prof = enable != 0;
    return OVL_OK;
}
