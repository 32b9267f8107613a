// Small MLP that predicts the Krylov depth k and the deflation count m
// (not in the paper: a learned front end that sizes the Krylov basis before
// a solve; the adaptive depth of ovl_sign_apply stays its fallback).
//
// Network x (n_in) -> ReLU(W1 x + b1) -> ReLU(W2 h1 + b2) -> W3 h2 + b3 (n_out),
// FP32, parameters in one flat vector [W1 (row-major), b1, W2, b2, W3, b3].
// Loss: mean of w (y - t)^2 with w = under_weight where y < t.
//
// k_mlp_grad: one CTA per tile of samples, one thread per hidden unit; the
// weights sit in shared memory, each thread keeps its rows of the gradient
// in registers and the CTA writes one partial gradient; k_mlp_reduce sums the
// partials in a fixed order (deterministic); k_mlp_adam applies Adam.
#include <algorithm>

#include "ovl_common.cuh"

#define MLP_MAX_IN 32
#define MLP_MAX_H 128
#define MLP_MAX_OUT 4
#define MLP_TILE 32  // samples per CTA

struct ovl_mlp_s {
    int n_in, n_h, n_out, np;
    float *theta = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr, *part = nullptr, *loss = nullptr;
    float *X = nullptr, *T = nullptr, *Y = nullptr;
    int cap = 0;  // samples the X/T/Y/part buffers hold
    int step = 0;
    std::string err;
};

namespace {

__device__ __forceinline__ int off_b1(int ni, int nh) { return nh * ni; }
__device__ __forceinline__ int off_W2(int ni, int nh) { return nh * ni + nh; }
__device__ __forceinline__ int off_b2(int ni, int nh) { return nh * ni + nh + nh * nh; }
__device__ __forceinline__ int off_W3(int ni, int nh) { return nh * ni + 2 * nh + nh * nh; }
__device__ __forceinline__ int off_b3(int ni, int nh, int no) { return nh * ni + 2 * nh + nh * nh + no * nh; }

// forward only (grad == nullptr) or forward + backward with partial gradients
__global__ void k_mlp(const float* __restrict__ theta, int ni, int nh, int no, const float* __restrict__ X,
                      const float* __restrict__ T, int B, float uw, float* __restrict__ Y, float* __restrict__ part,
                      float* __restrict__ lpart, int np) {
    extern __shared__ float sm[];
    float* sW = sm;                   // all parameters
    float* sx = sW + np;              // x of the current sample
    float* sh1 = sx + MLP_MAX_IN;     // h1
    float* sh2 = sh1 + MLP_MAX_H;     // h2
    float* sdz2 = sh2 + MLP_MAX_H;    // dz2
    float* sy = sdz2 + MLP_MAX_H;     // y, dy
    const int t = threadIdx.x;        // hidden unit (blockDim.x == nh)
    for (int i = t; i < np; i += blockDim.x) sW[i] = theta[i];
    const float* W1 = sW;
    const float* b1 = sW + off_b1(ni, nh);
    const float* W2 = sW + off_W2(ni, nh);
    const float* b2 = sW + off_b2(ni, nh);
    const float* W3 = sW + off_W3(ni, nh);
    const float* b3 = sW + off_b3(ni, nh, no);
    float gW1[MLP_MAX_IN], gW2[MLP_MAX_H], gW3[MLP_MAX_OUT];
    float gb1 = 0.f, gb2 = 0.f, gb3 = 0.f, lsum = 0.f;
    const bool grad = part != nullptr;
    for (int i = 0; i < MLP_MAX_IN; i++) gW1[i] = 0.f;
    for (int i = 0; i < MLP_MAX_H; i++) gW2[i] = 0.f;
    for (int i = 0; i < MLP_MAX_OUT; i++) gW3[i] = 0.f;
    __syncthreads();
    const int s0 = blockIdx.x * MLP_TILE;
    for (int si = s0; si < min(B, s0 + MLP_TILE); si++) {
        for (int i = t; i < ni; i += blockDim.x) sx[i] = X[(size_t)si * ni + i];
        __syncthreads();
        float z1 = b1[t];
        for (int i = 0; i < ni; i++) z1 = fmaf(W1[t * ni + i], sx[i], z1);
        sh1[t] = fmaxf(z1, 0.f);
        __syncthreads();
        float z2 = b2[t];
        for (int i = 0; i < nh; i++) z2 = fmaf(W2[t * nh + i], sh1[i], z2);
        sh2[t] = fmaxf(z2, 0.f);
        __syncthreads();
        if (t < no) {
            float y = b3[t];
            for (int i = 0; i < nh; i++) y = fmaf(W3[t * nh + i], sh2[i], y);
            if (Y) Y[(size_t)si * no + t] = y;
            if (grad) {
                float d = y - T[(size_t)si * no + t];
                float w = d < 0.f ? uw : 1.f;
                lsum += w * d * d;
                sy[t] = 2.f * w * d / (float)(B * no);  // dL/dy
            }
        }
        __syncthreads();
        if (grad) {
            // layer 3
            float dh2 = 0.f;
            for (int o = 0; o < no; o++) {
                gW3[o] = fmaf(sy[o], sh2[t], gW3[o]);
                dh2 = fmaf(W3[o * nh + t], sy[o], dh2);
            }
            if (t < no) gb3 += sy[t];
            float dz2 = z2 > 0.f ? dh2 : 0.f;
            sdz2[t] = dz2;
            gb2 += dz2;
            for (int i = 0; i < nh; i++) gW2[i] = fmaf(dz2, sh1[i], gW2[i]);
            __syncthreads();
            float dh1 = 0.f;
            for (int u = 0; u < nh; u++) dh1 = fmaf(W2[u * nh + t], sdz2[u], dh1);
            float dz1 = z1 > 0.f ? dh1 : 0.f;
            gb1 += dz1;
            for (int i = 0; i < ni; i++) gW1[i] = fmaf(dz1, sx[i], gW1[i]);
        }
        __syncthreads();
    }
    if (!grad) return;
    float* g = part + (size_t)blockIdx.x * np;
    for (int i = 0; i < ni; i++) g[t * ni + i] = gW1[i];
    g[off_b1(ni, nh) + t] = gb1;
    for (int i = 0; i < nh; i++) g[off_W2(ni, nh) + t * nh + i] = gW2[i];
    g[off_b2(ni, nh) + t] = gb2;
    for (int o = 0; o < no; o++) g[off_W3(ni, nh) + o * nh + t] = gW3[o];
    if (t < no) g[off_b3(ni, nh, no) + t] = gb3;
    if (t < no) lpart[blockIdx.x * MLP_MAX_OUT + t] = lsum;
    else if (t < MLP_MAX_OUT) lpart[blockIdx.x * MLP_MAX_OUT + t] = 0.f;
}

__global__ void k_mlp_reduce(const float* __restrict__ part, int nblk, int np, float* __restrict__ grad,
                             const float* __restrict__ lpart, float* __restrict__ loss, int B, int no) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < np) {
        float s = 0.f;
        for (int b = 0; b < nblk; b++) s += part[(size_t)b * np + i];
        grad[i] = s;
    }
    if (i == 0 && loss) {
        float s = 0.f;
        for (int b = 0; b < nblk * MLP_MAX_OUT; b++) s += lpart[b];
        *loss = s / (float)(B * no);
    }
}

// Adam (Kingma & Ba 2015) with bias correction
__global__ void k_mlp_adam(float* __restrict__ theta, float* __restrict__ m, float* __restrict__ v,
                           const float* __restrict__ g, int np, float lr, float b1, float b2, float eps, float c1,
                           float c2) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    float gi = g[i];
    float mi = b1 * m[i] + (1.f - b1) * gi;
    float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    theta[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

int fail(ovl_mlp net, int code, const char* msg) {
    if (net) net->err = msg;
    return ovl_fail(nullptr, code, "%s", msg);
}

int ensure(ovl_mlp net, int B) {
    if (B <= net->cap) return OVL_OK;
    cudaFree(net->X);
    cudaFree(net->T);
    cudaFree(net->Y);
    cudaFree(net->part);
    cudaFree(net->loss);
    int nblk = (B + MLP_TILE - 1) / MLP_TILE;
    bool ok = cudaMalloc(&net->X, sizeof(float) * (size_t)B * net->n_in) == cudaSuccess &&
              cudaMalloc(&net->T, sizeof(float) * (size_t)B * net->n_out) == cudaSuccess &&
              cudaMalloc(&net->Y, sizeof(float) * (size_t)B * net->n_out) == cudaSuccess &&
              cudaMalloc(&net->part, sizeof(float) * (size_t)nblk * net->np) == cudaSuccess &&
              cudaMalloc(&net->loss, sizeof(float) * ((size_t)nblk * MLP_MAX_OUT + 1)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        net->cap = 0;
        return fail(net, OVL_ENOMEM, "ovl_mlp: allocation failed");
    }
    net->cap = B;
    return OVL_OK;
}

size_t smem_bytes(ovl_mlp net) { return sizeof(float) * ((size_t)net->np + MLP_MAX_IN + 3 * MLP_MAX_H + 8); }

int copy_in(ovl_mlp net, float* dst, const float* src, size_t n) {
    cudaMemcpyKind k = ovl_is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (cudaMemcpy(dst, src, n * sizeof(float), k) != cudaSuccess) return fail(net, OVL_ECUDA, "ovl_mlp: copy failed");
    return OVL_OK;
}
int copy_out(ovl_mlp net, float* dst, const float* src, size_t n) {
    cudaMemcpyKind k = ovl_is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (cudaMemcpy(dst, src, n * sizeof(float), k) != cudaSuccess) return fail(net, OVL_ECUDA, "ovl_mlp: copy failed");
    return OVL_OK;
}

int grad_pass(ovl_mlp net, int B, float uw) {
    int nblk = (B + MLP_TILE - 1) / MLP_TILE;
    k_mlp<<<nblk, net->n_h, smem_bytes(net)>>>(net->theta, net->n_in, net->n_h, net->n_out, net->X, net->T, B, uw,
                                                nullptr, net->part, net->loss + 1, net->np);
    k_mlp_reduce<<<(net->np + 255) / 256, 256>>>(net->part, nblk, net->np, net->grad, net->loss + 1, net->loss, B,
                                                  net->n_out);
    if (cudaGetLastError() != cudaSuccess) return fail(net, OVL_ECUDA, "ovl_mlp: kernel launch failed");
    return OVL_OK;
}

}  // namespace

extern "C" int ovl_mlp_create(int n_in, int n_hidden, int n_out, ovl_mlp* out) {
    if (!out || n_in < 1 || n_in > MLP_MAX_IN || n_hidden < n_out || n_hidden > MLP_MAX_H || n_hidden < 32 ||
        n_hidden % 32 || n_out < 1 || n_out > MLP_MAX_OUT)
        return ovl_fail(nullptr, OVL_EINVAL, "ovl_mlp_create: sizes (in %d, hidden %d multiple of 32, out %d) out of range",
                        n_in, n_hidden, n_out);
    ovl_mlp net = new ovl_mlp_s();
    net->n_in = n_in;
    net->n_h = n_hidden;
    net->n_out = n_out;
    net->np = n_hidden * n_in + n_hidden + n_hidden * n_hidden + n_hidden + n_out * n_hidden + n_out;
    size_t b = sizeof(float) * net->np;
    if (cudaMalloc(&net->theta, b) != cudaSuccess || cudaMalloc(&net->m, b) != cudaSuccess ||
        cudaMalloc(&net->v, b) != cudaSuccess || cudaMalloc(&net->grad, b) != cudaSuccess) {
        cudaGetLastError();
        delete net;
        return ovl_fail(nullptr, OVL_ENOMEM, "ovl_mlp_create: allocation failed");
    }
    cudaMemset(net->theta, 0, b);
    cudaMemset(net->m, 0, b);
    cudaMemset(net->v, 0, b);
    cudaFuncSetAttribute(k_mlp, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
    *out = net;
    return OVL_OK;
}

extern "C" int ovl_mlp_destroy(ovl_mlp net) {
    if (!net) return OVL_OK;
    cudaDeviceSynchronize();
    for (float* p : {net->theta, net->m, net->v, net->grad, net->part, net->loss, net->X, net->T, net->Y}) cudaFree(p);
    delete net;
    return OVL_OK;
}

extern "C" int ovl_mlp_num_params(ovl_mlp net, int* np) {
    if (!net || !np) return ovl_fail(nullptr, OVL_EINVAL, "ovl_mlp_num_params: null argument");
    *np = net->np;
    return OVL_OK;
}

extern "C" int ovl_mlp_set_params(ovl_mlp net, const float* theta) {
    if (!net || !theta) return ovl_fail(nullptr, OVL_EINVAL, "ovl_mlp_set_params: null argument");
    if (int rc = copy_in(net, net->theta, theta, net->np)) return rc;
    cudaMemset(net->m, 0, sizeof(float) * net->np);
    cudaMemset(net->v, 0, sizeof(float) * net->np);
    net->step = 0;
    return OVL_OK;
}

extern "C" int ovl_mlp_get_params(ovl_mlp net, float* theta) {
    if (!net || !theta) return ovl_fail(nullptr, OVL_EINVAL, "ovl_mlp_get_params: null argument");
    return copy_out(net, theta, net->theta, net->np);
}

extern "C" int ovl_mlp_forward(ovl_mlp net, const float* X, int batch, float* Y) {
    if (!net || !X || !Y || batch < 1) return ovl_fail(nullptr, OVL_EINVAL, "ovl_mlp_forward: bad argument");
    if (int rc = ensure(net, batch)) return rc;
    if (int rc = copy_in(net, net->X, X, (size_t)batch * net->n_in)) return rc;
    int nblk = (batch + MLP_TILE - 1) / MLP_TILE;
    k_mlp<<<nblk, net->n_h, smem_bytes(net)>>>(net->theta, net->n_in, net->n_h, net->n_out, net->X, nullptr, batch,
                                                1.f, net->Y, nullptr, nullptr, net->np);
    if (cudaGetLastError() != cudaSuccess) return fail(net, OVL_ECUDA, "ovl_mlp_forward: launch failed");
    return copy_out(net, Y, net->Y, (size_t)batch * net->n_out);
}

extern "C" int ovl_mlp_loss_grad(ovl_mlp net, const float* X, const float* T, int batch, float under_weight,
                                 float* loss, float* grad) {
    if (!net || !X || !T || batch < 1) return ovl_fail(nullptr, OVL_EINVAL, "ovl_mlp_loss_grad: bad argument");
    if (int rc = ensure(net, batch)) return rc;
    if (int rc = copy_in(net, net->X, X, (size_t)batch * net->n_in)) return rc;
    if (int rc = copy_in(net, net->T, T, (size_t)batch * net->n_out)) return rc;
    if (int rc = grad_pass(net, batch, under_weight)) return rc;
    if (loss)
        if (int rc = copy_out(net, loss, net->loss, 1)) return rc;
    if (grad)
        if (int rc = copy_out(net, grad, net->grad, net->np)) return rc;
    return OVL_OK;
}

extern "C" int ovl_mlp_train(ovl_mlp net, const float* X, const float* T, int batch, int steps, float lr,
                             float under_weight, float* final_loss) {
    if (!net || !X || !T || batch < 1 || steps < 0 || !(lr > 0.f))
        return ovl_fail(nullptr, OVL_EINVAL, "ovl_mlp_train: bad argument");
    if (int rc = ensure(net, batch)) return rc;
    if (int rc = copy_in(net, net->X, X, (size_t)batch * net->n_in)) return rc;
    if (int rc = copy_in(net, net->T, T, (size_t)batch * net->n_out)) return rc;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (int s = 0; s < steps; s++) {
        if (int rc = grad_pass(net, batch, under_weight)) return rc;
        net->step++;
        float c1 = 1.f - powf(b1, (float)net->step), c2 = 1.f - powf(b2, (float)net->step);
        k_mlp_adam<<<(net->np + 255) / 256, 256>>>(net->theta, net->m, net->v, net->grad, net->np, lr, b1, b2, eps, c1,
                                                    c2);
    }
    if (int rc = grad_pass(net, batch, under_weight)) return rc;
    if (final_loss)
        if (int rc = copy_out(net, final_loss, net->loss, 1)) return rc;
    if (cudaDeviceSynchronize() != cudaSuccess) return fail(net, OVL_ECUDA, "ovl_mlp_train: kernel failed");
    return OVL_OK;
}

extern "C" const char* ovl_mlp_last_error(ovl_mlp net) { return net ? net->err.c_str() : ""; }
