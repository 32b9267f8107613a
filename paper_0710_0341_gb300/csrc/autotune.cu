// Autotuner of the stencil's launch shape (not in the paper).
//
// The stencil's result does not depend on how sites are assigned to threads,
// only its speed does: with consecutive sites per CTA most neighbour spinors
// (the y, z, t hops) are loaded by other CTAs and come from L2; with a CTA
// covering a tx x ty x tz tile of sites at one t, the x, y and z neighbours
// are mostly loaded by the CTA itself and hit L1. Which shape is fastest
// depends on the lattice, the arithmetic and the number of right-hand sides,
// so ovl_autotune times every candidate on the lattice's own links and keeps
// the fastest per (spinor format, link type) in the handle. For FP32 spinors a
// further candidate stages each hop's neighbour data in shared memory with
// asynchronous copies (k_dslash32a).
#include <string.h>

#include <vector>

#include "ovl_common.cuh"

namespace {

__global__ void k_fill(double* x, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        x[i] = 0.25 * (double)((i * 2654435761ull >> 7) % 1024) / 1024.0 - 0.125;
}

struct Cand {
    OvlStenShape s;
};

std::vector<Cand> candidates(const ovl_lattice lat, int fp64) {
    std::vector<Cand> out;
    const int* L = lat->dims;
    Cand c;
    c.s = OvlStenShape();  // the built-in rule
    out.push_back(c);
    if (fp64) {
        c.s.tpb = 32;
        out.push_back(c);
        c.s.tpb = 128;
        out.push_back(c);
    } else {
        c.s = OvlStenShape();  // neighbour data staged by cp.async
        c.s.tpb = 128;
        c.s.async = 1;
        out.push_back(c);
        for (int mb : {6, 4}) {  // register caps of 85 and 128 (fewer spills, fewer warps)
            c.s = OvlStenShape();
            c.s.tpb = 128;
            c.s.minb = mb;
            out.push_back(c);
        }
    }
    const int sizes[] = {128, 32};
    for (int sz : sizes) {
        if (sz == 32 && !fp64) continue;
        for (int tx = 4; tx <= 32; tx *= 2)
            for (int ty = 1; ty <= 16; ty *= 2) {
                if (sz % (tx * ty)) continue;
                const int tz = sz / (tx * ty);
                if (tz < 1 || L[0] % tx || L[1] % ty || L[2] % tz) continue;
                c.s = OvlStenShape();
                c.s.tpb = sz;
                c.s.tx = tx;
                c.s.ty = ty;
                c.s.tz = tz;
                out.push_back(c);
            }
    }
    return out;
}

}  // namespace

extern "C" int ovl_autotune(ovl_lattice lat, int nrhs, double* report, int max_report, int* n_report) {
    if (!lat || nrhs < 1 || nrhs > 64) return ovl_fail(lat, OVL_EINVAL, "ovl_autotune: bad argument");
    if (!lat->have_links) return ovl_fail(lat, OVL_EINVAL, "ovl_autotune: links not set");
    const size_t N = lat->N;
    cudaStream_t st = lat->stream;
    void *buf = nullptr, *ptrs = nullptr;
    double* mu = nullptr;
    const size_t vb = N * sizeof(double2) * (size_t)nrhs;
    if (cudaMalloc(&buf, 2 * vb) != cudaSuccess || cudaMalloc(&ptrs, 2 * nrhs * sizeof(void*)) != cudaSuccess ||
        cudaMalloc(&mu, nrhs * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(buf);
        cudaFree(ptrs);
        cudaFree(mu);
        return ovl_fail(lat, OVL_ENOMEM, "ovl_autotune: work buffers do not fit");
    }
    int rc = OVL_OK;
    int nrep = 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_fill<<<lat->num_sms * 4, 256, 0, st>>>((double*)buf, 2 * vb / sizeof(double));
    {
        std::vector<double> hm(nrhs, 0.3);
        cudaMemcpyAsync(mu, hm.data(), nrhs * sizeof(double), cudaMemcpyHostToDevice, st);
    }
    const int kinds[3][2] = {{OVL_VEC_F32, OVL_LINKS_R12}, {OVL_VEC_F32, OVL_LINKS_F32}, {OVL_VEC_F64, OVL_LINKS_F64}};
    for (int kd = 0; kd < 3 && !rc; kd++) {
        const int fmt = kinds[kd][0], links = kinds[kd][1];
        const size_t eb = fmt == OVL_VEC_F64 ? sizeof(double2) : sizeof(float2);
        std::vector<void*> hp(2 * nrhs);
        for (int r = 0; r < nrhs; r++) {
            hp[r] = (char*)buf + (size_t)r * N * eb;
            hp[nrhs + r] = (char*)buf + vb + (size_t)r * N * eb;
        }
        if (cudaMemcpyAsync(ptrs, hp.data(), hp.size() * sizeof(void*), cudaMemcpyHostToDevice, st) != cudaSuccess) {
            rc = ovl_fail(lat, OVL_ECUDA, "ovl_autotune: copy failed");
            break;
        }
        DslashArgs da;
        da.in = (const void* const*)ptrs;
        da.out = (void* const*)((void**)ptrs + nrhs);
        da.mu = mu;
        da.nrhs = nrhs;
        da.kappa = 1.0 / 6.0;
        OvlStenShape& slot = lat->sten_shape[fmt == OVL_VEC_F64 ? 0 : 1][links];
        const OvlStenShape keep = slot;
        double best = 1e300;
        OvlStenShape best_s = keep;
        for (const Cand& c : candidates(lat, fmt == OVL_VEC_F64)) {
            slot = c.s;
            for (int w = 0; w < 2 && !rc; w++) rc = ovl_dslash_launch(lat, da, fmt, links, st);
            const int reps = 5;
            cudaEventRecord(e0, st);
            for (int w = 0; w < reps && !rc; w++) rc = ovl_dslash_launch(lat, da, fmt, links, st);
            cudaEventRecord(e1, st);
            if (rc) break;
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                rc = ovl_fail(lat, OVL_ECUDA, "ovl_autotune: timing failed");
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            const double us = 1e3 * ms / reps;
            if (report && nrep < max_report) {
                double* q = report + 8 * (size_t)nrep;
                q[0] = fmt;
                q[1] = links;
                q[2] = c.s.tpb;
                q[3] = c.s.tx;
                q[4] = c.s.ty;
                q[5] = c.s.tz;
                q[6] = c.s.async + 10 * c.s.minb;  // async flag; register cap as 10 x resident CTAs
                q[7] = us;
                nrep++;
            }
            if (us < best) {
                best = us;
                best_s = c.s;
            }
        }
        slot = rc ? keep : best_s;
        if (!rc && fmt == OVL_VEC_F64) {
            // the double-float arithmetic on FP64 data takes the FP64 kernel's shape
            lat->sten_shape[0][OVL_LINKS_F64DF] = best_s;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamSynchronize(st);
    cudaFree(buf);
    cudaFree(ptrs);
    cudaFree(mu);
    if (n_report) *n_report = nrep;
    return rc;
}

extern "C" int ovl_autotune_shape(ovl_lattice lat, int fmt, int links, int shape[5]) {
    if (!lat || !shape || (fmt != OVL_VEC_F64 && fmt != OVL_VEC_F32) || links < 0 || links > 3)
        return ovl_fail(lat, OVL_EINVAL, "ovl_autotune_shape: bad argument");
    const OvlStenShape& s = lat->sten_shape[fmt == OVL_VEC_F64 ? 0 : 1][links];
    shape[0] = s.tpb;
    shape[1] = s.tx;
    shape[2] = s.ty;
    shape[3] = s.tz;
    shape[4] = s.async + 10 * s.minb;
    return OVL_OK;
}

extern "C" int ovl_autotune_set_shape(ovl_lattice lat, int fmt, int links, const int shape[5]) {
    if (!lat || !shape || (fmt != OVL_VEC_F64 && fmt != OVL_VEC_F32) || links < 0 || links > 3)
        return ovl_fail(lat, OVL_EINVAL, "ovl_autotune_set_shape: bad argument");
    OvlStenShape s;
    s.tpb = shape[0];
    s.tx = shape[1];
    s.ty = shape[2];
    s.tz = shape[3];
    s.async = shape[4] % 10;
    s.minb = shape[4] / 10;
    const int* L = lat->dims;
    const bool builtin = !s.tpb && !s.tx && !s.ty && !s.tz && !s.async && !s.minb;
    bool ok = builtin;
    if (!builtin && s.minb)
        ok = fmt == OVL_VEC_F32 && (s.minb == 4 || s.minb == 6) && s.tpb == 128 && !s.tx && !s.async &&
             links != OVL_LINKS_F64 && links != OVL_LINKS_F64DF;
    else if (!builtin && s.async)
        ok = fmt == OVL_VEC_F32 && links != OVL_LINKS_F64 && links != OVL_LINKS_F64DF && s.tpb == 128 && !s.tx &&
             !s.ty && !s.tz;
    else if (!builtin && !s.tx)
        ok = fmt == OVL_VEC_F64 && (s.tpb == 32 || s.tpb == 128) && !s.ty && !s.tz;
    else if (!builtin)
        ok = s.tx > 0 && s.ty > 0 && s.tz > 0 && s.tx * s.ty * s.tz == s.tpb &&
             (s.tpb == 128 || (s.tpb == 32 && fmt == OVL_VEC_F64)) && L[0] % s.tx == 0 && L[1] % s.ty == 0 &&
             L[2] % s.tz == 0;
    if (!ok)
        return ovl_fail(lat, OVL_EINVAL, "ovl_autotune_set_shape: shape {%d,%d,%d,%d,%d} does not fit this lattice/format",
                        s.tpb, s.tx, s.ty, s.tz, s.async);
    lat->sten_shape[fmt == OVL_VEC_F64 ? 0 : 1][links] = s;
    return OVL_OK;
}
