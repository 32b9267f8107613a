// The overlap operator at nonzero chemical potential (Sec. 1, Eq. 1):
//     D_ov(mu) x = x + gamma_5 sgn(H_w(mu)) x,
// and its adjoint D_ov(mu)^dag x = x + sgn(H_w(mu))^dag gamma_5 x with
// sgn(H_w(mu))^dag = sgn(H_w(mu)^dag) = sgn(H_w(-mu)) (H_w(mu)^dag = H_w(-mu)
// follows from Eq. 2). The sign runs through ovl_sign_apply; this file adds
// the gamma_5 combinations (canonical layout: spin index 2, 3 negated) and the
// LR deflation data of the adjoint operator: the left and right eigenvectors
// of H_w(mu) are the right and left eigenvectors of H_w(-mu), with conjugated
// eigenvalues (Eq. 20), so one eigenvector computation serves both (Sec. 5).
#include <string.h>

#include <vector>

#include "ovl_common.cuh"

namespace {

// canonical layout: complex index i = site * 12 + spin * 3 + colour
__device__ __forceinline__ bool lower_spin(size_t i) { return (i / 3) % 4 >= 2; }

// mode 0: y = x + gamma5 s;  mode 1: y = gamma5 x;  mode 2: y = x + s
__global__ void __launch_bounds__(256) k_overlap_combine(const double2* __restrict__ x, const double2* __restrict__ s,
                                                        double2* __restrict__ y, size_t n, int mode) {
    for (size_t i = blockIdx.x * (size_t)256 + threadIdx.x; i < n; i += (size_t)gridDim.x * 256) {
        const double sg = lower_spin(i) ? -1.0 : 1.0;
        const double2 a = x[i];
        if (mode == 1) {
            y[i] = make_double2(sg * a.x, sg * a.y);
        } else {
            const double2 b = s[i];
            const double f = mode == 0 ? sg : 1.0;
            y[i] = make_double2(a.x + f * b.x, a.y + f * b.y);
        }
    }
}

int combine(ovl_lattice lat, const double2* x, const double2* s, double2* y, size_t n, int mode) {
    size_t blocks = (n + 255) / 256, cap = (size_t)lat->num_sms * 8;
    k_overlap_combine<<<(unsigned)(blocks < cap ? blocks : cap), 256, 0, lat->stream>>>(x, s, y, n, mode);
    OVL_LAUNCH_CHECK(lat);
    return OVL_OK;
}

}  // namespace

extern "C" int ovl_overlap_apply(ovl_lattice lat, int nsolve, const ovl_sign_params* params,
                                 const ovl_deflation* defl, const double* x, double* y, int adjoint,
                                 ovl_sign_info* info) {
    if (!lat || nsolve < 1 || !params || !x || !y) return ovl_fail(lat, OVL_EINVAL, "ovl_overlap_apply: bad argument");
    if (adjoint != 0 && adjoint != 1) return ovl_fail(lat, OVL_EINVAL, "ovl_overlap_apply: adjoint must be 0 or 1");
    const size_t n = lat->N * (size_t)nsolve;  // complex entries of the batch
    const size_t bytes = n * sizeof(double2);
    double2* buf = nullptr;  // x (device copy), s, t
    if (cudaMalloc(&buf, 3 * bytes) != cudaSuccess) {
        cudaGetLastError();
        return ovl_fail(lat, OVL_ENOMEM, "ovl_overlap_apply: %zu bytes of work space", 3 * bytes);
    }
    double2 *dx = buf, *ds = buf + n, *dt = buf + 2 * n;
    int rc = OVL_OK;
    std::vector<ovl_sign_params> p(params, params + nsolve);
    const bool ydev = ovl_is_device_ptr(y);
    do {
        if (cudaMemcpyAsync(dx, x, bytes, cudaMemcpyDefault, lat->stream) != cudaSuccess) {
            rc = ovl_fail(lat, OVL_ECUDA, "ovl_overlap_apply: copying x failed");
            break;
        }
        const double2* sign_in = dx;
        if (adjoint) {
            // sgn(H_w(-mu)) (gamma5 x): the solves run at -mu with the adjoint deflation data
            for (auto& q : p) q.mu = -q.mu;
            if ((rc = combine(lat, dx, nullptr, dt, n, 1))) break;
            sign_in = dt;
        }
        if ((rc = ovl_sign_apply(lat, nsolve, p.data(), defl, (const double*)sign_in, (double*)ds, info))) break;
        double2* out = ydev ? (double2*)y : dt;
        if ((rc = combine(lat, dx, ds, out, n, adjoint ? 2 : 0))) break;
        if (!ydev && cudaMemcpyAsync(y, dt, bytes, cudaMemcpyDeviceToHost, lat->stream) != cudaSuccess) {
            rc = ovl_fail(lat, OVL_ECUDA, "ovl_overlap_apply: copying y failed");
            break;
        }
        if (cudaStreamSynchronize(lat->stream) != cudaSuccess)
            rc = ovl_fail(lat, OVL_ECUDA, "ovl_overlap_apply: %s", cudaGetErrorString(cudaGetLastError()));
    } while (0);
    cudaStreamSynchronize(lat->stream);
    cudaFree(buf);
    return rc;
}

extern "C" int ovl_deflation_adjoint(ovl_deflation d, ovl_deflation* out) {
    if (!d || !out) return ovl_fail(d ? d->lat : nullptr, OVL_EINVAL, "ovl_deflation_adjoint: null argument");
    ovl_lattice lat = d->lat;
    if (d->scheme != OVL_DEFL_LR)
        return ovl_fail(lat, OVL_ENOTSUP, "ovl_deflation_adjoint: only LR deflation data serve the adjoint");
    const size_t vb = lat->N * (size_t)d->m * sizeof(float2);
    ovl_deflation a = new ovl_deflation_s();
    a->lat = lat;
    a->scheme = OVL_DEFL_LR;
    a->m = d->m;
    a->mu = -d->mu;
    a->m_w = d->m_w;
    a->T_host.resize(2 * (size_t)d->m);
    for (int i = 0; i < d->m; i++) {  // conj(Lambda)
        a->T_host[2 * i] = d->T_host[2 * i];
        a->T_host[2 * i + 1] = -d->T_host[2 * i + 1];
    }
    bool ok = cudaMalloc(&a->S_hi, vb) == cudaSuccess && cudaMalloc(&a->S_lo, vb) == cudaSuccess &&
              cudaMalloc(&a->L_hi, vb) == cudaSuccess && cudaMalloc(&a->L_lo, vb) == cudaSuccess &&
              cudaMalloc(&a->T, (size_t)d->m * sizeof(double2)) == cudaSuccess;
    // right vectors of the adjoint = left vectors of the operator, and back
    ok = ok && cudaMemcpy(a->S_hi, d->L_hi, vb, cudaMemcpyDeviceToDevice) == cudaSuccess &&
         cudaMemcpy(a->S_lo, d->L_lo, vb, cudaMemcpyDeviceToDevice) == cudaSuccess &&
         cudaMemcpy(a->L_hi, d->S_hi, vb, cudaMemcpyDeviceToDevice) == cudaSuccess &&
         cudaMemcpy(a->L_lo, d->S_lo, vb, cudaMemcpyDeviceToDevice) == cudaSuccess &&
         cudaMemcpy(a->T, a->T_host.data(), (size_t)d->m * sizeof(double2), cudaMemcpyHostToDevice) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        ovl_destroy_deflation(a);
        return ovl_fail(lat, OVL_ENOMEM, "ovl_deflation_adjoint: allocation or copy failed");
    }
    *out = a;
    return OVL_OK;
}
