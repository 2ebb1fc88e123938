// Learned router: per-quartet features, a 3-layer MLP (20 -> 64 -> 64 -> 2, FP16 weights)
// predicting log10 of the quartet's largest |integral| (output 0) and log10 of the split
// path's error on it (output 1), and its training kernels (forward, backward with the
// gradient of the mean over samples of the summed squared errors, Adam).
//
// Parameter layout (LX_MLP_NPARAM floats): W1[64][20], b1[64], W2[64][64], b2[64],
// W3[2][64], b3[2].  Activations are ReLU.  The forward pass always uses the FP16-rounded
// weights; training keeps FP32 master weights and takes the gradient of the FP16 forward
// (straight through the rounding).
#include <cmath>
#include <cuda_fp16.h>

#include "lx_internal.cuh"

namespace lx {

namespace {

constexpr int NIN = LX_MLP_NIN, NW = LX_MLP_WIDTH, NOUT = LX_MLP_NOUT;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + NW * NIN, OFF_W2 = OFF_B1 + NW, OFF_B2 = OFF_W2 + NW * NW,
              OFF_W3 = OFF_B2 + NW, OFF_B3 = OFF_W3 + NOUT * NW, NPARAM = OFF_B3 + NOUT;
static_assert(NPARAM == LX_MLP_NPARAM, "parameter layout");

constexpr float PI_F = 3.14159265358979f;

// Features of one quartet (all FP32; the routing decision needs no more):
//  0-3  l of each shell / 6          4-7  ln(min exponent) / 4      8-11 ln(max exponent) / 4
//  12   |AB| / 10   13 |CD| / 10     14   |Pbar - Qbar| / 30 (centers of the most diffuse products)
//  15   mu_ab |AB|^2 / 20 (min exponents)   16 mu_cd |CD|^2 / 20     17 ln(1 + rho |Pbar Qbar|^2) / 3
//  18   ln(Ka Kb Kc Kd) / 6
//  19   log10 of an (ss|ss)-type magnitude estimate with the most diffuse primitives / 10
__global__ void features_kernel(const DShell* __restrict__ sh, const double* __restrict__ exps,
                                const int* __restrict__ q4, int64_t nq, float* __restrict__ feat) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nq) return;
    float zmin[4], zmax[4], c[4][3];
    int lsum = 0, lk[4];
    float lnK = 0.f;
    for (int k = 0; k < 4; ++k) {
        const DShell s = sh[q4[4 * i + k]];
        lk[k] = s.l;
        lsum += s.l;
        float mn = 1e30f, mx = 0.f;
        for (int j = 0; j < s.K; ++j) {
            const float z = (float)exps[s.prim_off + j];
            mn = fminf(mn, z);
            mx = fmaxf(mx, z);
        }
        zmin[k] = mn;
        zmax[k] = mx;
        lnK += logf((float)s.K);
        for (int d = 0; d < 3; ++d) c[k][d] = (float)s.A[d];
    }
    (void)lsum;
    float ab2 = 0.f, cd2 = 0.f, pq2 = 0.f;
    const float zp = zmin[0] + zmin[1], zq = zmin[2] + zmin[3];
    for (int d = 0; d < 3; ++d) {
        const float dab = c[0][d] - c[1][d], dcd = c[2][d] - c[3][d];
        ab2 += dab * dab;
        cd2 += dcd * dcd;
        const float P = (zmin[0] * c[0][d] + zmin[1] * c[1][d]) / zp, Q = (zmin[2] * c[2][d] + zmin[3] * c[3][d]) / zq;
        pq2 += (P - Q) * (P - Q);
    }
    const float mu = zmin[0] * zmin[1] / zp, nu = zmin[2] * zmin[3] / zq, rho = zp * zq / (zp + zq);
    const float T = rho * pq2;
    // 2 pi^{5/2} / (zp zq sqrt(zp + zq)) exp(-mu AB^2 - nu CD^2) F0(T), F0 ~ min(1, sqrt(pi / 4T))
    const float f0 = T < 1e-6f ? 1.f : fminf(1.f, sqrtf(PI_F / (4.f * T)));
    const float lest = logf(2.f * powf(PI_F, 2.5f) / (zp * zq * sqrtf(zp + zq))) - mu * ab2 - nu * cd2 + logf(f0);
    float* f = feat + i * NIN;
    for (int k = 0; k < 4; ++k) {
        f[k] = lk[k] / 6.f;
        f[4 + k] = logf(zmin[k]) / 4.f;
        f[8 + k] = logf(zmax[k]) / 4.f;
    }
    f[12] = sqrtf(ab2) / 10.f;
    f[13] = sqrtf(cd2) / 10.f;
    f[14] = sqrtf(pq2) / 30.f;
    f[15] = fminf(mu * ab2 / 20.f, 10.f);
    f[16] = fminf(nu * cd2 / 20.f, 10.f);
    f[17] = log1pf(T) / 3.f;
    f[18] = lnK / 6.f;
    f[19] = fmaxf(lest * 0.4342945f / 10.f, -10.f);
}

__device__ inline float relu(float x) { return x > 0.f ? x : 0.f; }

// Inference: one thread per sample, FP16 weights staged in shared memory as FP32.
__global__ void mlp_forward_kernel(const __half* __restrict__ p16, const float* __restrict__ feat, int64_t n,
                                   float* __restrict__ out) {
    __shared__ float P[NPARAM];
    for (int j = threadIdx.x; j < NPARAM; j += blockDim.x) P[j] = __half2float(p16[j]);
    __syncthreads();
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    float x[NIN], h1[NW];
    for (int k = 0; k < NIN; ++k) x[k] = feat[i * NIN + k];
    for (int j = 0; j < NW; ++j) {
        float a = P[OFF_B1 + j];
        for (int k = 0; k < NIN; ++k) a += P[OFF_W1 + j * NIN + k] * x[k];
        h1[j] = relu(a);
    }
    float y[NOUT];
    for (int o = 0; o < NOUT; ++o) y[o] = P[OFF_B3 + o];
    for (int j = 0; j < NW; ++j) {
        float a = P[OFF_B2 + j];
        for (int k = 0; k < NW; ++k) a += P[OFF_W2 + j * NW + k] * h1[k];
        const float h2 = relu(a);
        for (int o = 0; o < NOUT; ++o) y[o] += P[OFF_W3 + o * NW + j] * h2;
    }
    for (int o = 0; o < NOUT; ++o) out[i * NOUT + o] = y[o];
}

constexpr int TB = 128;  // samples per training block

// Loss and gradient of (1/n) sum_i sum_o (y_io - t_io)^2 over n samples (targets t[n][NOUT]),
// forward with FP16-rounded weights.  grad (NPARAM floats) and loss (1 float) must be zero on
// entry; blocks add into them.
constexpr size_t GRAD_SMEM = sizeof(float) * (NPARAM + TB * (NIN + 1) + 3 * TB * (NW + 1) + TB * NOUT);

__global__ void __launch_bounds__(TB) mlp_grad_kernel(const float* __restrict__ params,
                                                       const float* __restrict__ feat,
                                                       const float* __restrict__ target, int64_t n,
                                                       float* __restrict__ grad, float* __restrict__ loss) {
    extern __shared__ float sm[];
    float* P = sm;
    float (*X)[NIN + 1] = reinterpret_cast<float (*)[NIN + 1]>(P + NPARAM);
    float (*H1)[NW + 1] = reinterpret_cast<float (*)[NW + 1]>(&X[TB][0]);
    float (*D2)[NW + 1] = H1 + TB;  // dL/d(pre-activation 2), then reused for layer 1
    float (*H2)[NW + 1] = D2 + TB;
    float (*DY)[NOUT] = reinterpret_cast<float (*)[NOUT]>(&H2[TB][0]);
    for (int j = threadIdx.x; j < NPARAM; j += TB) P[j] = __half2float(__float2half_rn(params[j]));
    const int t = threadIdx.x;
    const int64_t i = blockIdx.x * (int64_t)TB + t;
    const bool live = i < n;
    for (int k = 0; k < NIN; ++k) X[t][k] = live ? feat[i * NIN + k] : 0.f;
    __syncthreads();
    // forward
    for (int j = 0; j < NW; ++j) {
        float a = P[OFF_B1 + j];
        for (int k = 0; k < NIN; ++k) a += P[OFF_W1 + j * NIN + k] * X[t][k];
        H1[t][j] = relu(a);
    }
    float y[NOUT];
    for (int o = 0; o < NOUT; ++o) y[o] = P[OFF_B3 + o];
    for (int j = 0; j < NW; ++j) {
        float a = P[OFF_B2 + j];
        for (int k = 0; k < NW; ++k) a += P[OFF_W2 + j * NW + k] * H1[t][k];
        H2[t][j] = relu(a);
        for (int o = 0; o < NOUT; ++o) y[o] += P[OFF_W3 + o * NW + j] * H2[t][j];
    }
    float l2 = 0.f;
    for (int o = 0; o < NOUT; ++o) {
        const float r = live ? y[o] - target[i * NOUT + o] : 0.f;
        DY[t][o] = live ? 2.f * r / (float)n : 0.f;
        l2 += r * r;
    }
    if (live) atomicAdd(loss, l2 / (float)n);
    // dL/d(pre2)_j = sum_o dy_o W3[o][j] [pre2_j > 0]
    for (int j = 0; j < NW; ++j) {
        float a = 0.f;
        for (int o = 0; o < NOUT; ++o) a += DY[t][o] * P[OFF_W3 + o * NW + j];
        D2[t][j] = H2[t][j] > 0.f ? a : 0.f;
    }
    __syncthreads();
    // layer-3 and layer-2 gradients, reduced over the block's samples
    for (int j = t; j < NW; j += TB) {
        float gw3[NOUT], gb2 = 0.f;
        for (int o = 0; o < NOUT; ++o) gw3[o] = 0.f;
        for (int s = 0; s < TB; ++s) {
            for (int o = 0; o < NOUT; ++o) gw3[o] += DY[s][o] * H2[s][j];
            gb2 += D2[s][j];
        }
        for (int o = 0; o < NOUT; ++o) atomicAdd(&grad[OFF_W3 + o * NW + j], gw3[o]);
        atomicAdd(&grad[OFF_B2 + j], gb2);
    }
    if (t < NOUT) {
        float gb3 = 0.f;
        for (int s = 0; s < TB; ++s) gb3 += DY[s][t];
        atomicAdd(&grad[OFF_B3 + t], gb3);
    }
    for (int e = t; e < NW * NW; e += TB) {
        const int j = e / NW, k = e - j * NW;
        float g = 0.f;
        for (int s = 0; s < TB; ++s) g += D2[s][j] * H1[s][k];
        atomicAdd(&grad[OFF_W2 + e], g);
    }
    __syncthreads();
    // dL/d(pre1)_k = sum_j dL/d(pre2)_j W2[j][k] [pre1_k > 0], overwriting D2 after use
    float d1[NW];
    for (int k = 0; k < NW; ++k) {
        float a = 0.f;
        for (int j = 0; j < NW; ++j) a += D2[t][j] * P[OFF_W2 + j * NW + k];
        d1[k] = H1[t][k] > 0.f ? a : 0.f;
    }
    __syncthreads();
    for (int k = 0; k < NW; ++k) D2[t][k] = d1[k];
    __syncthreads();
    for (int e = t; e < NW * NIN; e += TB) {
        const int j = e / NIN, k = e - j * NIN;
        float g = 0.f;
        for (int s = 0; s < TB; ++s) g += D2[s][j] * X[s][k];
        atomicAdd(&grad[OFF_W1 + e], g);
    }
    for (int j = t; j < NW; j += TB) {
        float g = 0.f;
        for (int s = 0; s < TB; ++s) g += D2[s][j];
        atomicAdd(&grad[OFF_B1 + j], g);
    }
}

// Adam on the FP32 master weights; refreshes the FP16 copy and clears the gradient.
__global__ void mlp_adam_kernel(float* __restrict__ params, float* __restrict__ m, float* __restrict__ v,
                                float* __restrict__ grad, __half* __restrict__ p16, int step, float lr, float b1,
                                float b2, float eps) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= NPARAM) return;
    const float g = grad[j];
    const float mj = b1 * m[j] + (1.f - b1) * g, vj = b2 * v[j] + (1.f - b2) * g * g;
    m[j] = mj;
    v[j] = vj;
    const float mh = mj / (1.f - powf(b1, (float)step)), vh = vj / (1.f - powf(b2, (float)step));
    const float w = params[j] - lr * mh / (sqrtf(vh) + eps);
    params[j] = w;
    p16[j] = __float2half_rn(w);
    grad[j] = 0.f;
}

}  // namespace

cudaError_t init_router_kernels() {
    return cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GRAD_SMEM);
}

cudaError_t launch_features(const DShell* sh, const double* exps, const int* q4, int64_t nq, float* feat,
                            cudaStream_t st) {
    if (nq <= 0) return cudaSuccess;
    features_kernel<<<(unsigned)((nq + 127) / 128), 128, 0, st>>>(sh, exps, q4, nq, feat);
    return cudaGetLastError();
}

cudaError_t launch_mlp_forward(const void* p16, const float* feat, int64_t n, float* out, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    mlp_forward_kernel<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(static_cast<const __half*>(p16), feat, n, out);
    return cudaGetLastError();
}

cudaError_t launch_mlp_grad(const float* params, const float* feat, const float* target, int64_t n, float* grad,
                            float* loss, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(grad, 0, sizeof(float) * NPARAM, st);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(loss, 0, sizeof(float), st)) != cudaSuccess) return e;
    if (n <= 0) return cudaSuccess;
    mlp_grad_kernel<<<(unsigned)((n + TB - 1) / TB), TB, GRAD_SMEM, st>>>(params, feat, target, n, grad, loss);
    return cudaGetLastError();
}

cudaError_t launch_mlp_adam(float* params, float* m, float* v, float* grad, void* p16, int step, float lr, float b1,
                            float b2, float eps, cudaStream_t st) {
    mlp_adam_kernel<<<(NPARAM + 127) / 128, 128, 0, st>>>(params, m, v, grad, static_cast<__half*>(p16), step, lr,
                                                          b1, b2, eps);
    return cudaGetLastError();
}

}  // namespace lx
