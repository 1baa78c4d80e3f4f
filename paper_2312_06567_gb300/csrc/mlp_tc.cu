// Batched inference of the learned Q' guess network on tensor cores.
//
// The network (9 -> 64 -> 64 -> 5, SiLU; features and target as in
// bgk_mlp.cuh) applied to a batch of points is three dense contractions,
// [B x 16] [16 x 64], [B x 64] [64 x 64] and [B x 64] [64 x 16] (inputs and
// outputs padded with zeros), the shape tensor cores are built for.  One CTA
// takes tiles of 128 points:
//   * each thread owns one point (one row): it normalises its features,
//     rounds them to BF16 and writes its row of the layer's A operand into
//     shared memory in the MMA's K-major core-matrix layout;
//   * one thread issues tcgen05.mma (kind::f16, BF16 inputs, FP32
//     accumulation in tensor memory, M = 128) against the weights, which
//     every CTA rounds to BF16 and lays out once (the B operands);
//   * each thread reads its row of the accumulator back (tcgen05.ld 32x32b),
//     adds the bias, applies SiLU, rounds to BF16 and writes the next
//     layer's A row; after the third layer it de-normalises the output.
// The arithmetic is the BF16 inference the Newton kernel runs inline (BF16
// weights and layer inputs, FP32 sums, FP32 biases and SiLU), except for the
// summation order and the tensor core's truncating accumulation.
#include "bgk_internal.cuh"

namespace {

constexpr int TM = 128;                        // points per tile
constexpr int K1 = 16;                         // 9 features padded to one K-step
constexpr int N3 = 16;                         // 5 outputs padded to the smallest N for M = 128
constexpr int OFF_B1 = 0;                      // [64 rows][16 K]   SBO 256   2048 B
constexpr int OFF_B2 = OFF_B1 + 2048;          // [64 rows][64 K]   SBO 1024  8192 B
constexpr int OFF_B3 = OFF_B2 + 8192;          // [16 rows][64 K]   SBO 1024  2048 B
constexpr int OFF_A0 = OFF_B3 + 2048;          // [128 rows][16 K]  SBO 256   4096 B
constexpr int OFF_A1 = OFF_A0 + 4096;          // [128 rows][64 K]  SBO 1024  16384 B
constexpr int OFF_A2 = OFF_A1 + 16384;         // [128 rows][64 K]  SBO 1024  16384 B
constexpr int OFF_END = OFF_A2 + 16384;        // 49152 B
constexpr size_t MLP_TC_SMEM = 1024 + OFF_END + 1024;   // alignment slack, then biases and barrier
constexpr int TMEM_COLS = 128;                 // layer 1 at 0..63, layer 2 at 64..127, layer 3 at 0..15

// K-major core-matrix layout without swizzle: 8-row groups `sbo` bytes apart,
// K-chunks of 8 BF16 128 B apart, rows 16 B apart.
__device__ __forceinline__ int kmaj(int r, int k, int sbo) { return (r / 8) * sbo + (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2; }

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) |
           ((uint64_t)1 << 46);
}
// kind::f16, FP32 accumulator, BF16 A and B (K-major), M = 128
__device__ __forceinline__ uint32_t idesc_n(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(id), "r"(acc)
        : "memory");
}
__device__ __forceinline__ bool bar_try(uint32_t bar, uint32_t par) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(par)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// bounded wait (about 1 s) for the MMA commit of the given phase
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t par) {
    if (bar_try(bar, par)) return true;
    const unsigned long long t0 = now_ns();
    for (;;) {
        for (int i = 0; i < 32; ++i)
            if (bar_try(bar, par)) return true;
        if (now_ns() - t0 > 1000000000ull) return false;
    }
}
// 32 consecutive accumulator columns of this thread's row
__device__ __forceinline__ void tmem_row32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
        "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);      // a in the low half (lower address)
    return *reinterpret_cast<const uint32_t *>(&h);
}
// SiLU of 32 accumulator columns plus bias, rounded to BF16, written as four
// 16-byte chunks of this thread's row of a K = 64 operand (chunks c0 .. c0+3)
__device__ __forceinline__ void silu_row(const float (&z)[32], const float *bias, uint8_t *A, int row, int c0) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        uint32_t w[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const int j = 8 * c + 2 * h;
            const float a = z[j] + bias[j], b = z[j + 1] + bias[j + 1];
            w[h] = pack_bf16(a / (1.f + __expf(-a)), b / (1.f + __expf(-b)));
        }
        *reinterpret_cast<uint4 *>(A + kmaj(row, 8 * (c0 + c), 1024)) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

__global__ void __launch_bounds__(TM, 4) k_mlp_infer_tc(MlpParams p, const float *x, long long n, float *delta,
                                                       unsigned int *status) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *sm = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    float *sb = reinterpret_cast<float *>(sm + OFF_END);       // b1[64] b2[64] b3[5] norm[28]
    unsigned long long *bar = reinterpret_cast<unsigned long long *>(sb + 164);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + 1);
    int *abort_flag = reinterpret_cast<int *>(tslot + 1);
    const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;

    // ---- weights as BF16 B operands (row = output unit, K = input unit) and the FP32 biases
    const float *W1 = p.w, *b1 = W1 + MLP_IN * MLP_H, *W2 = b1 + MLP_H, *b2 = W2 + MLP_H * MLP_H;
    const float *W3 = b2 + MLP_H, *b3 = W3 + MLP_H * MLP_OUT;
    for (int i = tid; i < MLP_H * K1; i += TM) {
        const int n_ = i / K1, k = i % K1;
        const float v = k < MLP_IN ? W1[k * MLP_H + n_] : 0.f;
        *reinterpret_cast<__nv_bfloat16 *>(sm + OFF_B1 + kmaj(n_, k, 256)) = __float2bfloat16_rn(v);
    }
    for (int i = tid; i < MLP_H * MLP_H; i += TM) {
        const int n_ = i / MLP_H, k = i % MLP_H;
        *reinterpret_cast<__nv_bfloat16 *>(sm + OFF_B2 + kmaj(n_, k, 1024)) = __float2bfloat16_rn(W2[k * MLP_H + n_]);
    }
    for (int i = tid; i < N3 * MLP_H; i += TM) {
        const int n_ = i / MLP_H, k = i % MLP_H;
        const float v = n_ < MLP_OUT ? W3[k * MLP_OUT + n_] : 0.f;
        *reinterpret_cast<__nv_bfloat16 *>(sm + OFF_B3 + kmaj(n_, k, 1024)) = __float2bfloat16_rn(v);
    }
    if (tid < MLP_H) {
        sb[tid] = b1[tid];
        sb[64 + tid] = b2[tid];
    }
    if (tid < MLP_OUT) sb[128 + tid] = b3[tid];
    if (tid < MLP_NNORM) sb[136 + tid] = p.norm[tid];
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *abort_flag = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    const uint32_t lane_base = tmem + ((uint32_t)(32 * warp) << 16);   // this warp's 32 accumulator rows
    const float *xm = sb + 136, *xs = sb + 136 + MLP_IN, *tmean = sb + 136 + 2 * MLP_IN, *tstd = tmean + MLP_OUT;
    uint32_t phase = 0;
    // one MMA group and its commit by thread 0, then everyone waits for it
    auto run_layer = [&](int layer) -> bool {
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (layer == 0) {
                mma(tmem, sdesc(su32(sm + OFF_A0), 256), sdesc(su32(sm + OFF_B1), 256), idesc_n(MLP_H), 0u);
            } else {
                const int offA = layer == 1 ? OFF_A1 : OFF_A2, offB = layer == 1 ? OFF_B2 : OFF_B3;
                const uint32_t d = tmem + (layer == 1 ? 64u : 0u);
                const uint32_t id = idesc_n(layer == 1 ? MLP_H : N3);
                for (int ks = 0; ks < 4; ++ks)
                    mma(d, sdesc(su32(sm + offA) + ks * 256, 1024), sdesc(su32(sm + offB) + ks * 256, 1024), id,
                        ks ? 1u : 0u);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
                         : "memory");
        }
        const bool ok = bar_wait(su32(bar), phase & 1);
        phase += 1;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        return __syncthreads_and(ok ? 1 : 0) != 0;
    };

    const long long n_tiles = (n + TM - 1) / TM;
    for (long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const long long pt = tile * TM + tid;
        const bool live = pt < n;
        // ---- layer-1 input: normalised features rounded to BF16, zero padded
        {
            float xn[K1];
#pragma unroll
            for (int f = 0; f < K1; ++f) xn[f] = 0.f;
            if (live) {
#pragma unroll
                for (int f = 0; f < MLP_IN; ++f) xn[f] = (__ldg(x + pt * MLP_IN + f) - xm[f]) / xs[f];
            }
#pragma unroll
            for (int c = 0; c < 2; ++c)
                *reinterpret_cast<uint4 *>(sm + OFF_A0 + kmaj(tid, 8 * c, 256)) =
                    make_uint4(pack_bf16(xn[8 * c], xn[8 * c + 1]), pack_bf16(xn[8 * c + 2], xn[8 * c + 3]),
                               pack_bf16(xn[8 * c + 4], xn[8 * c + 5]), pack_bf16(xn[8 * c + 6], xn[8 * c + 7]));
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (!run_layer(0)) { if (tid == 0) *abort_flag = 1; break; }
        // ---- hidden layer 1 -> A1
        {
            float z[32];
            tmem_row32(lane_base + 0, z);
            silu_row(z, sb, sm + OFF_A1, tid, 0);
            tmem_row32(lane_base + 32, z);
            silu_row(z, sb + 32, sm + OFF_A1, tid, 4);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (!run_layer(1)) { if (tid == 0) *abort_flag = 1; break; }
        // ---- hidden layer 2 -> A2
        {
            float z[32];
            tmem_row32(lane_base + 64, z);
            silu_row(z, sb + 64, sm + OFF_A2, tid, 0);
            tmem_row32(lane_base + 96, z);
            silu_row(z, sb + 96, sm + OFF_A2, tid, 4);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (!run_layer(2)) { if (tid == 0) *abort_flag = 1; break; }
        // ---- output: bias, de-normalisation
        {
            float z[32];
            tmem_row32(lane_base + 0, z);
            if (live) {
#pragma unroll
                for (int o = 0; o < MLP_OUT; ++o) delta[pt * MLP_OUT + o] = (z[o] + sb[128 + o]) * tstd[o] + tmean[o];
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
    }
    if (tid == 0 && *abort_flag) atomicOr(status, BGK_DEV_TIMEOUT);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

}  // namespace

cudaError_t launch_mlp_infer_tc(const MlpParams &p, const float *x, long long n, float *delta, unsigned int *status,
                                cudaStream_t s) {
    static SmemLimit lim;
    size_t *attr = lim.slot();
    if (!attr) return cudaErrorInvalidDevice;
    if (MLP_TC_SMEM > *attr) {
        const cudaError_t e =
            cudaFuncSetAttribute(k_mlp_infer_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MLP_TC_SMEM);
        if (e != cudaSuccess) return e;
        *attr = MLP_TC_SMEM;
    }
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const long long tiles = (n + TM - 1) / TM;
    const long long grid = tiles < 4ll * sms ? tiles : 4ll * sms;    // four CTAs per SM (TMEM: 4 x 128 columns)
    k_mlp_infer_tc<<<(unsigned)grid, TM, MLP_TC_SMEM, s>>>(p, x, n, delta, status);
    return cudaGetLastError();
}
