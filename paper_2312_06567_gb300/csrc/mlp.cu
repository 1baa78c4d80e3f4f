// Learned initial guess for the Q' Newton solve: a 9 -> 64 -> 64 -> 5 SiLU
// network trained on the GPU on (features, Delta) pairs that the solver's own
// converged Newton solves log.  The paper has the Newton solve only; the
// guess is this project's addition (features, target and network as in
// mlp_features / the header's MLP entry points).
//
// Precision: weights and layer inputs are rounded to BF16 (the operands of
// every product), all sums accumulate in FP32, the optimiser keeps FP32
// master weights (Adam).  With bf16 = 0 the same kernels run on FP32
// operands (used by the gradient check against the FP64 reference).
//
// Training kernel: one block of 256 threads per chunk of 64 samples; the
// block computes the three layers as small GEMMs through shared memory, the
// backward pass likewise, and adds its partial weight gradients into the
// global FP32 gradient with atomics.
#include "bgk_internal.cuh"
#include "bgk_mlp.cuh"

namespace {

constexpr int SB = 64;       // samples per training block
constexpr int NT = 256;      // threads per training block

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }
__device__ __forceinline__ float rnd(float x, int bf16) { return bf16 ? bf16r(x) : x; }
__device__ __forceinline__ float silu(float z) { return z / (1.f + __expf(-z)); }
__device__ __forceinline__ float silu_grad(float z) {
    const float s = 1.f / (1.f + __expf(-z));
    return s * (1.f + z * (1.f - s));
}

struct TrainSmem {
    float xn[SB][MLP_IN];
    float z1[SB][MLP_H], h1[SB][MLP_H];
    float z2[SB][MLP_H], h2[SB][MLP_H];
    float dy[SB][MLP_OUT];
    float w2[MLP_H][MLP_H];
    float red[NT / 32];
};

// x[n][9] raw features, t[n][5] raw targets; idx[b] sample indices of this batch.
__global__ void __launch_bounds__(NT) k_mlp_train(MlpParams prm, const float *x, const float *t,
                                                  const int *idx, int nb, float *grad, double *loss,
                                                  int bf16) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TrainSmem &sm = *reinterpret_cast<TrainSmem *>(smem_raw);
    const int tid = threadIdx.x;
    const int s0 = blockIdx.x * SB;
    const int ns = min(SB, nb - s0);
    const float *W1 = prm.w, *b1 = W1 + MLP_IN * MLP_H, *W2 = b1 + MLP_H, *b2 = W2 + MLP_H * MLP_H;
    const float *W3 = b2 + MLP_H, *b3 = W3 + MLP_H * MLP_OUT;
    // stage the samples (normalised) and W2
    for (int i = tid; i < SB * MLP_IN; i += NT) {
        const int s = i / MLP_IN, f = i % MLP_IN;
        float v = 0.f;
        if (s < ns) v = (x[(size_t)idx[s0 + s] * MLP_IN + f] - prm.norm[f]) / prm.norm[MLP_IN + f];
        sm.xn[s][f] = rnd(v, bf16);
    }
    for (int i = tid; i < MLP_H * MLP_H; i += NT) sm.w2[i / MLP_H][i % MLP_H] = rnd(W2[i], bf16);
    __syncthreads();
    // layer 1
    for (int i = tid; i < SB * MLP_H; i += NT) {
        const int s = i / MLP_H, j = i % MLP_H;
        float z = b1[j];
        for (int f = 0; f < MLP_IN; ++f) z = fmaf(sm.xn[s][f], rnd(W1[f * MLP_H + j], bf16), z);
        sm.z1[s][j] = z;
        sm.h1[s][j] = rnd(silu(z), bf16);
    }
    __syncthreads();
    // layer 2
    for (int i = tid; i < SB * MLP_H; i += NT) {
        const int s = i / MLP_H, j = i % MLP_H;
        float z = b2[j];
        for (int k = 0; k < MLP_H; ++k) z = fmaf(sm.h1[s][k], sm.w2[k][j], z);
        sm.z2[s][j] = z;
        sm.h2[s][j] = rnd(silu(z), bf16);
    }
    __syncthreads();
    // layer 3, residual, loss, dL/dy = 2 (y - tn) / (nb * 5)
    float lsum = 0.f;
    for (int i = tid; i < SB * MLP_OUT; i += NT) {
        const int s = i / MLP_OUT, o = i % MLP_OUT;
        float d = 0.f;
        if (s < ns) {
            float y = b3[o];
            for (int k = 0; k < MLP_H; ++k) y = fmaf(sm.h2[s][k], rnd(W3[k * MLP_OUT + o], bf16), y);
            const float tn = (t[(size_t)idx[s0 + s] * MLP_OUT + o] - prm.norm[2 * MLP_IN + o]) /
                             prm.norm[2 * MLP_IN + MLP_OUT + o];
            const float r = y - tn;
            lsum = fmaf(r, r, lsum);
            d = 2.f * r / (float)(nb * MLP_OUT);
        }
        sm.dy[s][o] = d;
    }
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if ((tid & 31) == 0) sm.red[tid >> 5] = lsum;
    __syncthreads();
    if (tid == 0) {
        double s = 0.0;
        for (int w = 0; w < NT / 32; ++w) s += sm.red[w];
        atomicAdd(loss, s / (double)(nb * MLP_OUT));
    }
    // gW3 = h2^T dy, gb3 = sum dy
    float *gW1 = grad, *gb1 = gW1 + MLP_IN * MLP_H, *gW2 = gb1 + MLP_H, *gb2 = gW2 + MLP_H * MLP_H;
    float *gW3 = gb2 + MLP_H, *gb3 = gW3 + MLP_H * MLP_OUT;
    for (int i = tid; i < MLP_H * MLP_OUT; i += NT) {
        const int k = i / MLP_OUT, o = i % MLP_OUT;
        float a = 0.f;
        for (int s = 0; s < ns; ++s) a = fmaf(sm.h2[s][k], sm.dy[s][o], a);
        atomicAdd(&gW3[i], a);
    }
    if (tid < MLP_OUT) {
        float a = 0.f;
        for (int s = 0; s < ns; ++s) a += sm.dy[s][tid];
        atomicAdd(&gb3[tid], a);
    }
    // dz2 = (dy W3^T) * s'(z2), stored over z2
    __syncthreads();
    for (int i = tid; i < SB * MLP_H; i += NT) {
        const int s = i / MLP_H, j = i % MLP_H;
        float d = 0.f;
        for (int o = 0; o < MLP_OUT; ++o) d = fmaf(sm.dy[s][o], rnd(W3[j * MLP_OUT + o], bf16), d);
        sm.z2[s][j] = d * silu_grad(sm.z2[s][j]);
    }
    __syncthreads();
    // gW2 = h1^T dz2, gb2
    for (int i = tid; i < MLP_H * MLP_H; i += NT) {
        const int k = i / MLP_H, j = i % MLP_H;
        float a = 0.f;
        for (int s = 0; s < ns; ++s) a = fmaf(sm.h1[s][k], sm.z2[s][j], a);
        atomicAdd(&gW2[i], a);
    }
    if (tid < MLP_H) {
        float a = 0.f;
        for (int s = 0; s < ns; ++s) a += sm.z2[s][tid];
        atomicAdd(&gb2[tid], a);
    }
    // dz1 = (dz2 W2^T) * s'(z1), stored over z1
    for (int i = tid; i < SB * MLP_H; i += NT) {
        const int s = i / MLP_H, k = i % MLP_H;
        float d = 0.f;
        for (int j = 0; j < MLP_H; ++j) d = fmaf(sm.z2[s][j], sm.w2[k][j], d);
        sm.z1[s][k] = d * silu_grad(sm.z1[s][k]);
    }
    __syncthreads();
    // gW1 = xn^T dz1, gb1
    for (int i = tid; i < MLP_IN * MLP_H; i += NT) {
        const int f = i / MLP_H, k = i % MLP_H;
        float a = 0.f;
        for (int s = 0; s < ns; ++s) a = fmaf(sm.xn[s][f], sm.z1[s][k], a);
        atomicAdd(&gW1[i], a);
    }
    if (tid < MLP_H) {
        float a = 0.f;
        for (int s = 0; s < ns; ++s) a += sm.z1[s][tid];
        atomicAdd(&gb1[tid], a);
    }
}

// Adam on the FP32 master weights; clears the gradient.
__global__ void k_mlp_adam(float *w, float *m, float *v, float *grad, int n, float lr, float b1,
                           float b2, float eps, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float g = grad[i];
    const float mi = b1 * m[i] + (1.f - b1) * g;
    const float vi = b2 * v[i] + (1.f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    grad[i] = 0.f;
}

}  // namespace

size_t mlp_train_smem() { return sizeof(TrainSmem); }

cudaError_t launch_mlp_train(const MlpParams &p, const float *x, const float *t, const int *idx, int nb,
                             float *grad, double *loss, int bf16, cudaStream_t s) {
    const size_t smem = sizeof(TrainSmem);
    static SmemLimit lim;
    size_t *attr = lim.slot();
    if (!attr) return cudaErrorInvalidDevice;
    if (smem > *attr) {
        cudaError_t e = cudaFuncSetAttribute(k_mlp_train, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        *attr = smem;
    }
    k_mlp_train<<<(nb + SB - 1) / SB, NT, smem, s>>>(p, x, t, idx, nb, grad, loss, bf16);
    return cudaGetLastError();
}

__global__ void k_mlp_round(const float *w, float *w16, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) w16[i] = mlp_round(w[i], 1);
}

cudaError_t launch_mlp_round(const float *w, float *w16, int n, cudaStream_t s) {
    k_mlp_round<<<(n + 255) / 256, 256, 0, s>>>(w, w16, n);
    return cudaGetLastError();
}

cudaError_t launch_mlp_adam(float *w, float *m, float *v, float *grad, int n, float lr, float b1, float b2,
                            float eps, int step, cudaStream_t s) {
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    k_mlp_adam<<<(n + 255) / 256, 256, 0, s>>>(w, m, v, grad, n, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}
