// The learned Q' guess network shared by the training kernels (mlp.cu) and
// the Newton kernel's inline inference (kernels_qprime.cu).
//
// Parameters, one flat FP32 array (row-major [fan_in][fan_out] matrices):
//   W1[9][64] b1[64] W2[64][64] b2[64] W3[64][5] b3[5]        (MLP_NPARAM)
// Normalisation, one flat FP32 array:
//   x_mean[9] x_std[9] t_mean[5] t_std[5]                       (MLP_NNORM)
// Features x: rho, U1..3, theta, I1, I2, I3 of A = Pi/(rho theta), and the
// local mean free path lambda = mu/rho sqrt(pi/(2 theta)).  Target Delta:
// rho'/rho - 1, (U' - U)/sqrt(theta), theta'/theta - 1.
#pragma once

#include <cuda_bf16.h>

#define MLP_IN 9
#define MLP_H 64
#define MLP_OUT 5
#define MLP_NPARAM (MLP_IN * MLP_H + MLP_H + MLP_H * MLP_H + MLP_H + MLP_H * MLP_OUT + MLP_OUT)
#define MLP_NNORM (2 * MLP_IN + 2 * MLP_OUT)
#define MLP_LOG_STRIDE (MLP_IN + MLP_OUT)

struct MlpParams {
    const float *w;          // MLP_NPARAM FP32 master weights
    const float *norm;       // MLP_NNORM
    const float *w16;        // the weights rounded to BF16 once (or null): BF16 inference reads them as they are
};

__device__ __forceinline__ float mlp_round(float x, int bf16) {
    return bf16 ? __bfloat162float(__float2bfloat16_rn(x)) : x;
}

// One warp evaluates the network for one point; every lane passes the same
// features and receives Delta.  Lane l owns hidden units l and l + 32.
__device__ __forceinline__ void mlp_infer_warp(const MlpParams &p, const float x[MLP_IN], float delta[MLP_OUT],
                                               int bf16, int lane) {
    // with the pre-rounded copy the weights need no rounding here (the same
    // values: BF16 rounding of a value is a fixed function of it)
    const bool pre = bf16 && p.w16 != nullptr;
    const float *W1 = pre ? p.w16 : p.w, *b1 = W1 + MLP_IN * MLP_H, *W2 = b1 + MLP_H, *b2 = W2 + MLP_H * MLP_H;
    const float *W3 = b2 + MLP_H, *b3 = W3 + MLP_H * MLP_OUT;
    const int wr = pre ? 0 : bf16;
    float xn[MLP_IN];
#pragma unroll
    for (int f = 0; f < MLP_IN; ++f) xn[f] = mlp_round((x[f] - __ldg(p.norm + f)) / __ldg(p.norm + MLP_IN + f), bf16);
    float h1[2], h2[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int j = lane + 32 * r;
        float z = __ldg(b1 + j);
#pragma unroll
        for (int f = 0; f < MLP_IN; ++f) z = fmaf(xn[f], mlp_round(__ldg(W1 + f * MLP_H + j), wr), z);
        h1[r] = mlp_round(z / (1.f + __expf(-z)), bf16);
    }
    float z2[2] = {__ldg(b2 + lane), __ldg(b2 + lane + 32)};
    for (int k = 0; k < MLP_H; ++k) {
        const float hk = __shfl_sync(0xffffffffu, h1[k >> 5], k & 31);
        z2[0] = fmaf(hk, mlp_round(__ldg(W2 + k * MLP_H + lane), wr), z2[0]);
        z2[1] = fmaf(hk, mlp_round(__ldg(W2 + k * MLP_H + lane + 32), wr), z2[1]);
    }
#pragma unroll
    for (int r = 0; r < 2; ++r) h2[r] = mlp_round(z2[r] / (1.f + __expf(-z2[r])), bf16);
#pragma unroll
    for (int o = 0; o < MLP_OUT; ++o) {
        float y = h2[0] * mlp_round(__ldg(W3 + lane * MLP_OUT + o), wr) +
                  h2[1] * mlp_round(__ldg(W3 + (lane + 32) * MLP_OUT + o), wr);
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) y += __shfl_xor_sync(0xffffffffu, y, s);
        y += __ldg(b3 + o);
        delta[o] = y * __ldg(p.norm + 2 * MLP_IN + MLP_OUT + o) + __ldg(p.norm + 2 * MLP_IN + o);
    }
}

// batched inference on tensor cores (mlp_tc.cu): delta[n][5] from raw features x[n][9]
cudaError_t launch_mlp_infer_tc(const MlpParams &p, const float *x, long long n, float *delta, unsigned int *status,
                                cudaStream_t s);
size_t mlp_train_smem();
cudaError_t launch_mlp_train(const MlpParams &p, const float *x, const float *t, const int *idx, int nb,
                             float *grad, double *loss, int bf16, cudaStream_t s);
// w16[i] = w[i] rounded to BF16 (held in FP32), the copy BF16 inference reads
cudaError_t launch_mlp_round(const float *w, float *w16, int n, cudaStream_t s);
cudaError_t launch_mlp_adam(float *w, float *m, float *v, float *grad, int n, float lr, float b1, float b2,
                            float eps, int step, cudaStream_t s);
