// Cost-model network (config selection of the contraction steps): an MLP
// with two hidden ReLU layers of TN_MLP_HIDDEN units over TN_MLP_IN step
// features, one output (predicted log2 of a step's time per pass).
//
//   z1 = W1 x + b1,  a1 = relu(z1)
//   z2 = W2 a1 + b2, a2 = relu(z2)
//   y  = w3 . a2 + b3
//
// Parameters are one flat FP32 array: W1 [H][D] (row j = hidden unit j),
// b1 [H], W2 [H][H] (row j = unit j of the second layer), b2 [H], w3 [H],
// b3 [1].  Training minimises L = (1/n) sum_i (y_i - t_i)^2.
//
// Kernels (one CTA = H threads, thread j owns hidden unit j of both layers):
//   k_mlp_pass<TRAIN>  forward (and, when training, backward) over a
//                      contiguous chunk of rows per CTA.  W2 sits in shared
//                      memory with a padded row stride of H+1 floats, so both
//                      the row walk (thread j over k: z2) and the column walk
//                      (thread j over i: dA1) are free of bank conflicts; the
//                      CTA's dW2 accumulator uses the same layout.  Per-CTA
//                      gradient partials go to caller scratch.
//   k_mlp_reduce       sums the partials over CTAs in a fixed order
//                      (deterministic gradients and loss).
//   k_mlp_adam         Adam update (Kingma & Ba, bias-corrected moments).
//   k_mlp_f16          inference with FP16 weights and activations
//                      (half2 FMAs, summed in FP32 every 8 pairs).
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "../../include/tn.h"

namespace {

constexpr int D = TN_MLP_IN;
constexpr int H = TN_MLP_HIDDEN;
constexpr int HP = H + 1;  // padded row stride of W2 in shared memory
constexpr int NP = TN_MLP_NPARAMS;
constexpr int OFF_W1 = 0, OFF_B1 = H * D, OFF_W2 = OFF_B1 + H, OFF_B2 = OFF_W2 + H * H, OFF_W3 = OFF_B2 + H,
              OFF_B3 = OFF_W3 + H;
static_assert(OFF_B3 + 1 == NP, "parameter layout");
constexpr int MAX_CTAS = 304;  // 2 per SM on 152 SMs
constexpr size_t PASS_SMEM = size_t(2) * H * HP * sizeof(float);

__device__ __forceinline__ float block_sum(float v, float *red) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[w] = v;
    __syncthreads();
    float s = 0.f;
#pragma unroll
    for (int q = 0; q < H / 32; ++q) s += red[q];  // fixed order
    __syncthreads();
    return s;
}

template <bool TRAIN>
__global__ void __launch_bounds__(H) k_mlp_pass(const float *__restrict__ P, const float *__restrict__ X,
                                               const float *__restrict__ T, int64_t n, int64_t chunk,
                                               float *__restrict__ y_out, float *__restrict__ partial) {
    extern __shared__ float sm[];
    float *W2s = sm;            // [H][HP]
    float *G2s = sm + H * HP;   // [H][HP] (training)
    __shared__ float xs[D], a1s[H], dz2s[H], red[H / 32];
    const int j = threadIdx.x;
    float w1[D];
#pragma unroll
    for (int d = 0; d < D; ++d) w1[d] = P[OFF_W1 + j * D + d];
    const float b1 = P[OFF_B1 + j], b2 = P[OFF_B2 + j], w3 = P[OFF_W3 + j], b3 = P[OFF_B3];
    for (int k = 0; k < H; ++k) {
        W2s[j * HP + k] = P[OFF_W2 + j * H + k];
        if (TRAIN) G2s[j * HP + k] = 0.f;
    }
    float gw1[D];
#pragma unroll
    for (int d = 0; d < D; ++d) gw1[d] = 0.f;
    float gb1 = 0.f, gb2 = 0.f, gw3 = 0.f, gb3 = 0.f, loss = 0.f;
    __syncthreads();
    const int64_t r0 = int64_t(blockIdx.x) * chunk;
    const int64_t r1 = r0 + chunk < n ? r0 + chunk : n;
    for (int64_t i = r0; i < r1; ++i) {
        if (j < D) xs[j] = X[i * D + j];
        __syncthreads();
        float z1 = b1;
#pragma unroll
        for (int d = 0; d < D; ++d) z1 = fmaf(w1[d], xs[d], z1);
        a1s[j] = fmaxf(z1, 0.f);
        __syncthreads();
        float z2 = b2;
#pragma unroll 8
        for (int k = 0; k < H; ++k) z2 = fmaf(W2s[j * HP + k], a1s[k], z2);
        const float a2 = fmaxf(z2, 0.f);
        const float y = b3 + block_sum(w3 * a2, red);
        if (!TRAIN) {
            if (j == 0) y_out[i] = y;
            continue;
        }
        const float e = y - T[i];
        const float dy = 2.f * e / float(n);
        loss = fmaf(e, e, loss);
        gw3 = fmaf(dy, a2, gw3);
        gb3 += dy;
        const float dz2 = z2 > 0.f ? dy * w3 : 0.f;
        dz2s[j] = dz2;
        gb2 += dz2;
#pragma unroll 8
        for (int k = 0; k < H; ++k) G2s[j * HP + k] = fmaf(dz2, a1s[k], G2s[j * HP + k]);
        __syncthreads();
        float da1 = 0.f;
#pragma unroll 8
        for (int q = 0; q < H; ++q) da1 = fmaf(dz2s[q], W2s[q * HP + j], da1);
        const float dz1 = z1 > 0.f ? da1 : 0.f;
        gb1 += dz1;
#pragma unroll
        for (int d = 0; d < D; ++d) gw1[d] = fmaf(dz1, xs[d], gw1[d]);
        __syncthreads();  // xs, a1s and dz2s are rewritten by the next row
    }
    if (!TRAIN) return;
    float *out = partial + int64_t(blockIdx.x) * (NP + 1);
#pragma unroll
    for (int d = 0; d < D; ++d) out[OFF_W1 + j * D + d] = gw1[d];
    out[OFF_B1 + j] = gb1;
    for (int k = 0; k < H; ++k) out[OFF_W2 + j * H + k] = G2s[j * HP + k];
    out[OFF_B2 + j] = gb2;
    out[OFF_W3 + j] = gw3;
    if (j == 0) {
        out[OFF_B3] = gb3;
        out[NP] = loss;
    }
}

__global__ void k_mlp_reduce(const float *__restrict__ partial, int ctas, int64_t n, float *__restrict__ grad,
                             float *__restrict__ loss) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > NP) return;
    float s = 0.f;
    for (int c = 0; c < ctas; ++c) s += partial[int64_t(c) * (NP + 1) + p];  // fixed order
    if (p < NP) grad[p] = s;
    else if (loss) *loss = s / float(n);
}

// (1 - beta) and the bias corrections 1 - beta^t come from the host in
// double precision: in FP32, 1 - 0.999f alone is off by 1.3e-5 relative.
__global__ void k_mlp_adam(float *__restrict__ P, const float *__restrict__ G, float *__restrict__ M,
                           float *__restrict__ V, float lr, float b1, float omb1, float b2, float omb2, float eps,
                           float c1, float c2) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NP) return;
    const float g = G[p];
    const float m = b1 * M[p] + omb1 * g;
    const float v = b2 * V[p] + omb2 * g * g;
    M[p] = m;
    V[p] = v;
    P[p] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
}

__global__ void k_mlp_to_half(const float *__restrict__ P, __half *__restrict__ Q) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < NP) Q[p] = __float2half_rn(P[p]);
}

// FP16 inference.  W2 rows in shared memory with a stride of H+2 halves
// (an odd number of 32-bit words), so half2 pairs stay aligned and the row
// walk is free of bank conflicts.
constexpr int HP2 = H + 2;
__global__ void __launch_bounds__(H) k_mlp_f16(const __half *__restrict__ Q, const float *__restrict__ X, int64_t n,
                                              int64_t chunk, float *__restrict__ y_out) {
    __shared__ __align__(16) __half W2s[H * HP2];
    __shared__ __align__(16) __half a1s[H];
    __shared__ __half xs[D];
    __shared__ float red[H / 32];
    const int j = threadIdx.x;
    __half2 w1[D / 2];
#pragma unroll
    for (int d = 0; d < D / 2; ++d) w1[d] = __halves2half2(Q[OFF_W1 + j * D + 2 * d], Q[OFF_W1 + j * D + 2 * d + 1]);
    const float b1 = __half2float(Q[OFF_B1 + j]), b2 = __half2float(Q[OFF_B2 + j]);
    const float w3 = __half2float(Q[OFF_W3 + j]), b3 = __half2float(Q[OFF_B3]);
    for (int k = 0; k < H; ++k) W2s[j * HP2 + k] = Q[OFF_W2 + j * H + k];
    __syncthreads();
    const int64_t r0 = int64_t(blockIdx.x) * chunk;
    const int64_t r1 = r0 + chunk < n ? r0 + chunk : n;
    for (int64_t i = r0; i < r1; ++i) {
        if (j < D) xs[j] = __float2half_rn(X[i * D + j]);
        __syncthreads();
        __half2 acc = __float2half2_rn(0.f);
#pragma unroll
        for (int d = 0; d < D / 2; ++d) acc = __hfma2(w1[d], __halves2half2(xs[2 * d], xs[2 * d + 1]), acc);
        const float z1 = b1 + __low2float(acc) + __high2float(acc);
        a1s[j] = __float2half_rn(fmaxf(z1, 0.f));
        __syncthreads();
        float z2 = b2;
        const __half2 *wr = reinterpret_cast<const __half2 *>(W2s + j * HP2);
        const __half2 *ar = reinterpret_cast<const __half2 *>(a1s);
        for (int k8 = 0; k8 < H / 2; k8 += 8) {
            __half2 s = __float2half2_rn(0.f);
#pragma unroll
            for (int q = 0; q < 8; ++q) s = __hfma2(wr[k8 + q], ar[k8 + q], s);
            z2 += __low2float(s) + __high2float(s);
        }
        const float a2 = __half2float(__float2half_rn(fmaxf(z2, 0.f)));
        const float y = b3 + block_sum(w3 * a2, red);
        if (j == 0) y_out[i] = y;
    }
}

int ctas_for(int64_t n) {
    int64_t c = (n + 31) / 32;
    return int(c < 1 ? 1 : (c > MAX_CTAS ? MAX_CTAS : c));
}

}  // namespace

namespace tnk {

size_t mlp_grad_scratch_bytes(int64_t n) { return size_t(ctas_for(n)) * (NP + 1) * sizeof(float); }

cudaError_t mlp_forward(const float *params, const float *X, int64_t n, float *y, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_mlp_pass<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PASS_SMEM);
    if (e != cudaSuccess) return e;
    const int ctas = ctas_for(n);
    const int64_t chunk = (n + ctas - 1) / ctas;
    k_mlp_pass<false><<<ctas, H, PASS_SMEM, st>>>(params, X, nullptr, n, chunk, y, nullptr);
    return cudaGetLastError();
}

cudaError_t mlp_grad(const float *params, const float *X, const float *t, int64_t n, float *grad, float *loss,
                     float *scratch, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(k_mlp_pass<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PASS_SMEM);
    if (e != cudaSuccess) return e;
    const int ctas = ctas_for(n);
    const int64_t chunk = (n + ctas - 1) / ctas;
    k_mlp_pass<true><<<ctas, H, PASS_SMEM, st>>>(params, X, t, n, chunk, nullptr, scratch);
    k_mlp_reduce<<<(NP + 1 + 255) / 256, 256, 0, st>>>(scratch, ctas, n, grad, loss);
    return cudaGetLastError();
}

cudaError_t mlp_adam(float *params, const float *grad, float *m, float *v, int32_t step, float lr, float beta1,
                     float beta2, float eps, cudaStream_t st) {
    const double b1 = beta1, b2 = beta2;
    const float c1 = float(1.0 - std::pow(b1, double(step))), c2 = float(1.0 - std::pow(b2, double(step)));
    k_mlp_adam<<<(NP + 255) / 256, 256, 0, st>>>(params, grad, m, v, lr, beta1, float(1.0 - b1), beta2,
                                                 float(1.0 - b2), eps, c1, c2);
    return cudaGetLastError();
}

cudaError_t mlp_to_half(const float *params, uint16_t *params16, cudaStream_t st) {
    k_mlp_to_half<<<(NP + 255) / 256, 256, 0, st>>>(params, reinterpret_cast<__half *>(params16));
    return cudaGetLastError();
}

cudaError_t mlp_forward_f16(const uint16_t *params16, const float *X, int64_t n, float *y, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int ctas = ctas_for(n);
    const int64_t chunk = (n + ctas - 1) / ctas;
    k_mlp_f16<<<ctas, H, 0, st>>>(reinterpret_cast<const __half *>(params16), X, n, chunk, y);
    return cudaGetLastError();
}

}  // namespace tnk
