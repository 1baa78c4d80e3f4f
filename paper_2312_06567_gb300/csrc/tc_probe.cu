// Tensor-core probe of the FR element operator (measurement, not the stage).
//
// The FR divergence of one element at one velocity applies, per reference
// direction d, the element operator Op_d[s][s'] (the 1-D derivative with the
// own-trace lift folded in, D - g' (x) l, acting along the d-lines of the
// element's (p+1)^3 nodes; section "Numerical method").  Written densely it
// is a GEMM: t_d[s][n] = sum_s' Op_d[s][s'] f[s'][n] over the columns n of a
// panel of element-velocity pairs.  This probe runs that GEMM the way a
// tensor-core stage would, at p = 3 (64 nodes):
//   * panels of 48 velocity columns x 64 nodes arrive by TMA tiled copies
//     (cp.async.bulk.tensor, a tensor map over this GPU's own memory) into a
//     ring of shared-memory stages, already split into BF16 hi and lo parts
//     and laid out in the MMA's K-major core-matrix order;
//   * one thread issues tcgen05.mma (kind::f16, BF16 inputs, FP32
//     accumulation in tensor memory, M = 64, N = 48, K = 16) for the three
//     directions and the three products of the split (hi.hi + lo.hi + hi.lo),
//     36 instructions per panel, into a double-buffered TMEM accumulator;
//   * four warps read the accumulators back with tcgen05.ld (16x128b) and
//     either reduce them (throughput) or store them (checked on the host).
// It reports the operator's throughput as it streams from HBM and its
// arithmetic against an FP64 evaluation: the largest relative error and the
// relative bias of the outputs' magnitudes (the tensor core truncates its
// FP32 accumulation toward zero, so the error has a sign).
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/bgk.h"
#include "bgk_internal.cuh"

namespace {

constexpr int PQ = 4, PNS = 64;              // p = 3
constexpr int PN = 48;                        // velocity columns per panel
constexpr int PSTAGES = 4;                    // ring depth
constexpr int PANEL_BYTES = PN * PNS * 2;     // one BF16 piece of a panel (6144 B)
constexpr int OP_BYTES = PNS * PNS * 2;       // one BF16 piece of one direction's operator (8192 B)
constexpr int PTHREADS = 160;                 // warp 0 issues copies and MMAs, warps 1-4 read TMEM back
constexpr int TMEM_COLS = 512;                // 2 buffers x 3 directions x 48 columns = 288, rounded up
constexpr size_t PROBE_SMEM = 1024 + 6 * OP_BYTES + (size_t)PSTAGES * 2 * PANEL_BYTES + 1024;
constexpr size_t PROBE_SMEM_LAUNCH = 120 * 1024;   // > half an SM's shared memory: one CTA per SM (TMEM)
static_assert(PROBE_SMEM <= PROBE_SMEM_LAUNCH, "probe shared memory");

// Offset of element (row r, k) in the K-major core-matrix layout without
// swizzle: 8-row groups 1024 B apart (8 K-chunks of 8 rows x 16 B), K-chunks
// 128 B apart, rows 16 B apart.
__host__ __device__ inline size_t kmajor_off(int r, int k) {
    return (size_t)(r / 8) * 1024 + (size_t)(k / 8) * 128 + (size_t)(r % 8) * 16 + (size_t)(k % 8) * 2;
}

__device__ __forceinline__ uint32_t s_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ unsigned long long p_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ bool p_try(uint32_t bar, uint32_t par) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(par)
        : "memory");
    return ok != 0;
}
// bounded wait (about 1 s) on a barrier phase; false if it gave up
__device__ __forceinline__ bool p_wait(uint32_t bar, uint32_t par) {
    if (p_try(bar, par)) return true;
    const unsigned long long t0 = p_ns();
    for (;;) {
        for (int i = 0; i < 32; ++i)
            if (p_try(bar, par)) return true;
        if (p_ns() - t0 > 1000000000ull) return false;
    }
}
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    // start >> 4, leading (K-chunk) offset 128 B, stride (8-row group) offset
    // 1024 B, the fixed 0b001 of bits 46-48, no base offset, no swizzle
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46);
}
// kind::f16 instruction descriptor: FP32 accumulator, BF16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(PN >> 3) << 17) | ((uint32_t)(64 >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(IDESC), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tma_panel(uint32_t dst, const CUtensorMap *map, int piece, int panel, uint32_t bar) {
    // box (64 elements of one core matrix, 48 core matrices, 1 panel) at (0, 0, 2 panel + piece)
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
            "r"(dst), "l"(map), "r"(0), "r"(0), "r"(2 * panel + piece), "r"(bar)
        : "memory");
}
// 16 lanes x 128 bits, repeated 4 times along the columns: thread t holds
// rows t/4 and t/4 + 8 of its warp's 16 lanes at columns t%4 + 4 j, j < 4
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[8]) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.16x128b.x4.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// ops: [3 directions][2 pieces][OP_BYTES] (K-major layout); panels via the
// tensor map (2 pieces per panel); out (check mode): [n_check][3][64][48].
__global__ void __launch_bounds__(PTHREADS, 1)
    k_probe_fr_tc(const __grid_constant__ CUtensorMap map, const uint8_t *ops, int n_panels, int n_check,
                  float *out, double *checksum, unsigned int *status) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *sm = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *sA = sm;                                           // 6 x OP_BYTES
    uint8_t *sB = sA + 6 * OP_BYTES;                            // PSTAGES x 2 x PANEL_BYTES
    unsigned long long *bars = (unsigned long long *)(sB + (size_t)PSTAGES * 2 * PANEL_BYTES);
    unsigned long long *full = bars, *empty = bars + PSTAGES, *acc_full = bars + 2 * PSTAGES,
                       *acc_empty = bars + 2 * PSTAGES + 2;
    uint32_t *tslot = (uint32_t *)(bars + 2 * PSTAGES + 4);
    volatile int *abort_flag = (volatile int *)(tslot + 1);
    const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;

    for (int i = tid; i < 6 * OP_BYTES / 16; i += PTHREADS)
        reinterpret_cast<uint4 *>(sA)[i] = reinterpret_cast<const uint4 *>(ops)[i];
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (tid == 0) {
        for (int s = 0; s < PSTAGES; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(s_u32(full + s)), "r"(1) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(s_u32(empty + s)), "r"(1) : "memory");
        }
        for (int b = 0; b < 2; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(s_u32(acc_full + b)), "r"(1) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(s_u32(acc_empty + b)), "r"(4) : "memory");
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s_u32(tslot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;

    // this CTA's panels: blockIdx.x, blockIdx.x + gridDim.x, ...
    const int n_my = n_panels > (int)blockIdx.x ? (n_panels - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    auto panel_of = [&](int i) { return (int)blockIdx.x + i * (int)gridDim.x; };

    int issued = 0;                 // panels whose copies were issued (thread 0)
    int mma_done = 0;               // panels whose MMAs were issued (thread 0)
    if (tid == 0) {
        bool ok = true;
        auto issue = [&](int j) {
            const int s = j % PSTAGES;
            if (j >= PSTAGES && !p_wait(s_u32(empty + s), ((j / PSTAGES) & 1) ^ 1)) return false;
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(s_u32(full + s)),
                         "r"(2 * PANEL_BYTES)
                         : "memory");
            const uint32_t dst = s_u32(sB + (size_t)s * 2 * PANEL_BYTES);
            tma_panel(dst, &map, 0, panel_of(j), s_u32(full + s));
            tma_panel(dst + PANEL_BYTES, &map, 1, panel_of(j), s_u32(full + s));
            return true;
        };
        for (int j = 0; j < PSTAGES - 1 && j < n_my && ok; ++j) ok = issue(j), issued += ok ? 1 : 0;
        for (int i = 0; i < n_my && ok; ++i) {
            const int j = i + PSTAGES - 1;
            if (j < n_my) {
                ok = issue(j);
                if (!ok) break;
                ++issued;
            }
            const int s = i % PSTAGES, b = i & 1;
            if (!p_wait(s_u32(full + s), (i / PSTAGES) & 1)) { ok = false; break; }
            if (i >= 2 && !p_wait(s_u32(acc_empty + b), ((i / 2) & 1) ^ 1)) { ok = false; break; }
            if (*abort_flag) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t aB = s_u32(sB + (size_t)s * 2 * PANEL_BYTES);
            for (int d = 0; d < 3; ++d) {
                const uint32_t dcol = tmem + (uint32_t)(b * 3 * PN + d * PN);
                const uint32_t aH = s_u32(sA + (size_t)(2 * d) * OP_BYTES), aL = aH + OP_BYTES;
                // hi.hi, lo.hi, hi.lo, each over four K-steps of 16 nodes (256 B apart)
                const uint32_t pa[3] = {aH, aL, aH}, pb[3] = {aB, aB, aB + PANEL_BYTES};
                for (int pass = 0; pass < 3; ++pass)
                    for (int ks = 0; ks < 4; ++ks)
                        mma_bf16(dcol, smem_desc(pa[pass] + ks * 256), smem_desc(pb[pass] + ks * 256),
                                 (pass | ks) ? 1u : 0u);
            }
            mma_commit(s_u32(empty + s));
            mma_commit(s_u32(acc_full + b));
            ++mma_done;
        }
        if (!ok) {
            *abort_flag = 1;
            atomicOr(status, BGK_DEV_TIMEOUT);
        }
    } else if (warp >= 1) {
        // ---- TMEM readback (whole warps 1-4; lanes 1-31 of warp 0 stay out:
        // tcgen05.ld and __all_sync are collective over the full warp, and its
        // lane 0 is the issuing thread): warp w reads lanes 32 (w % 4) .. + 15,
        // the M = 64 layout ----
        const int q = warp % 4;
        const int r0 = 16 * q + lane / 4, r1 = r0 + 8;      // this thread's two output rows
        double sum = 0.0;
        for (int i = 0; i < n_my; ++i) {
            const int b = i & 1;
            bool ok = false;
            // wait for the accumulator, unless the issuing thread gave up
            const unsigned long long t0 = p_ns();
            while (!(ok = p_try(s_u32(acc_full + b), (i / 2) & 1))) {
                if (*abort_flag || p_ns() - t0 > 1000000000ull) break;
            }
            ok = __all_sync(0xffffffffu, ok);              // the warp's TMEM loads are collective
            if (!ok) {
                if (lane == 0) { *abort_flag = 1; atomicOr(status, BGK_DEV_TIMEOUT); }
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int panel = panel_of(i);
            float acc = 0.f;
            for (int d = 0; d < 3; ++d) {
#pragma unroll
                for (int c0 = 0; c0 < PN; c0 += 16) {
                    float v[8];
                    tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * 3 * PN + d * PN + c0), v);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    if (panel < n_check) {
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const int col = c0 + lane % 4 + 4 * j;
                            out[(((size_t)panel * 3 + d) * PNS + r0) * PN + col] = v[2 * j];
                            out[(((size_t)panel * 3 + d) * PNS + r1) * PN + col] = v[2 * j + 1];
                        }
                    }
#pragma unroll
                    for (int j = 0; j < 8; ++j) acc += v[j];
                }
            }
            sum += acc;
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0)
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(s_u32(acc_empty + b)) : "memory");
        }
        atomicAdd(checksum, sum);
    }
    // no copy or MMA may still be in flight when TMEM is released and the CTA exits
    if (tid == 0) {
        for (int j = mma_done; j < issued; ++j) p_wait(s_u32(full + j % PSTAGES), (j / PSTAGES) & 1);
        if (mma_done > 0) {
            const int last = mma_done - 1;
            p_wait(s_u32(acc_full + (last & 1)), (last / 2) & 1);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

// Fill n panels (both pieces) with BF16 values in [0.5, 2) from a hash: the
// bulk of the streamed data, never checked.
__global__ void k_probe_fill(uint16_t *p, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        uint32_t h = (uint32_t)i * 2654435761u;
        h ^= h >> 15;
        p[i] = (uint16_t)(0x3F00u + (h & 0xFFu));
    }
}

uint16_t bf16_rn(float x) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}
float bf16_val(uint16_t h) {
    uint32_t u = (uint32_t)h << 16;
    float x;
    std::memcpy(&x, &u, 4);
    return x;
}

}  // namespace

extern "C" BGK_API bgk_status bgk_probe_tc(long long n_panels, double out[6]) {
    if (!out || n_panels < 16 || n_panels > (1ll << 22)) return BGK_EINVAL;
    int dev = 0, sms = 0, cc_major = 0, cc_minor = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return BGK_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return BGK_ECUDA;
    cudaDeviceGetAttribute(&cc_major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&cc_minor, cudaDevAttrComputeCapabilityMinor, dev);
    if (cc_major != 10 || cc_minor != 3) return BGK_ENOTSUP;    // built for sm_103a only

    // ---- the p = 3 element operators of the first octant (u_d > 0 on every
    // axis: the inflow trace is the left face's, folded in as D - g_L' (x) l(-1)),
    // FP32-rounded, split into BF16 hi + lo, in the K-major layout
    FROps fr{};
    fr_build_host(3, fr);
    float Dt[PQ][PQ];
    for (int i = 0; i < PQ; ++i)
        for (int j = 0; j < PQ; ++j) Dt[i][j] = (float)(fr.D[i][j] - fr.dgL[i] * fr.lm[j]);
    std::vector<uint8_t> ops(6 * OP_BYTES, 0);
    std::vector<double> opf(3 * PNS * PNS, 0.0);          // the operators as the split represents them
    for (int d = 0; d < 3; ++d)
        for (int r = 0; r < PNS; ++r)
            for (int k = 0; k < PNS; ++k) {
                const int ir[3] = {r % PQ, (r / PQ) % PQ, r / (PQ * PQ)}, ik[3] = {k % PQ, (k / PQ) % PQ, k / (PQ * PQ)};
                bool line = true;
                for (int e = 0; e < 3; ++e)
                    if (e != d && ir[e] != ik[e]) line = false;
                const float v = line ? Dt[ir[d]][ik[d]] : 0.f;
                const uint16_t hi = bf16_rn(v), lo = bf16_rn(v - bf16_val(hi));
                std::memcpy(&ops[(size_t)(2 * d) * OP_BYTES + kmajor_off(r, k)], &hi, 2);
                std::memcpy(&ops[(size_t)(2 * d + 1) * OP_BYTES + kmajor_off(r, k)], &lo, 2);
                opf[((size_t)d * PNS + r) * PNS + k] = (double)bf16_val(hi) + (double)bf16_val(lo);
            }

    // ---- panels: the first n_check carry seeded values that are checked
    const int n_check = 8;
    std::vector<uint16_t> chk((size_t)n_check * 2 * PANEL_BYTES / 2, 0);
    std::vector<double> dat((size_t)n_check * PN * PNS);
    uint64_t state = 0x9E3779B97F4A7C15ull;
    for (int pnl = 0; pnl < n_check; ++pnl)
        for (int n = 0; n < PN; ++n)
            for (int k = 0; k < PNS; ++k) {
                state = state * 6364136223846793005ull + 1442695040888963407ull;
                const double u01 = (double)(state >> 11) * (1.0 / 9007199254740992.0);
                const float v = (float)(0.5 + u01);                 // FP32 data in [0.5, 1.5)
                const uint16_t hi = bf16_rn(v), lo = bf16_rn(v - bf16_val(hi));
                uint16_t *base = chk.data() + (size_t)pnl * PANEL_BYTES;      // 2 pieces x PANEL_BYTES / 2
                base[kmajor_off(n, k) / 2] = hi;
                base[PANEL_BYTES / 2 + kmajor_off(n, k) / 2] = lo;
                dat[((size_t)pnl * PN + n) * PNS + k] = (double)v;
            }
    const size_t total = (size_t)n_panels * 2 * PANEL_BYTES;
    uint8_t *dpan = nullptr, *dops = nullptr;
    float *dout = nullptr;
    double *dsum = nullptr;
    unsigned int *dstat = nullptr;
    bgk_status st = BGK_OK;
    auto cu = [&](cudaError_t e) {
        if (e != cudaSuccess && st == BGK_OK) st = (e == cudaErrorMemoryAllocation) ? BGK_ENOMEM : BGK_ECUDA;
        return st == BGK_OK;
    };
    cu(cudaMalloc(&dpan, total));
    cu(cudaMalloc(&dops, ops.size()));
    cu(cudaMalloc(&dout, (size_t)n_check * 3 * PNS * PN * sizeof(float)));
    cu(cudaMalloc(&dsum, sizeof(double)));
    cu(cudaMalloc(&dstat, sizeof(unsigned int)));
    if (st == BGK_OK) {
        k_probe_fill<<<sms * 4, 256>>>((uint16_t *)dpan, total / 2);
        cu(cudaGetLastError());
        cu(cudaMemcpy(dpan, chk.data(), chk.size() * 2, cudaMemcpyHostToDevice));
        cu(cudaMemcpy(dops, ops.data(), ops.size(), cudaMemcpyHostToDevice));
        cu(cudaMemset(dout, 0, (size_t)n_check * 3 * PNS * PN * sizeof(float)));
        cu(cudaMemset(dsum, 0, sizeof(double)));
        cu(cudaMemset(dstat, 0, sizeof(unsigned int)));
    }
    // tensor map: 64 BF16 (one 128-B core matrix) x 48 core matrices x 2 n_panels pieces
    CUtensorMap map;
    std::memset(&map, 0, sizeof map);
    if (st == BGK_OK) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult qr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &qr) !=
                cudaSuccess ||
            qr != cudaDriverEntryPointSuccess || !fn) {
            st = BGK_ENOTSUP;
        } else {
            const cuuint64_t dims[3] = {64, 48, (cuuint64_t)(2 * n_panels)};
            const cuuint64_t strides[2] = {128, (cuuint64_t)PANEL_BYTES};
            const cuuint32_t box[3] = {64, 48, 1}, estr[3] = {1, 1, 1};
            const CUresult r = ((PFN_cuTensorMapEncodeTiled_v12000)fn)(
                &map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, dpan, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) st = BGK_ECUDA;
        }
    }
    float ms = 0.f;
    if (st == BGK_OK) cu(cudaFuncSetAttribute(k_probe_fr_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PROBE_SMEM_LAUNCH));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (st == BGK_OK) {
        cu(cudaEventCreate(&e0));
        cu(cudaEventCreate(&e1));
    }
    if (st == BGK_OK) {
        // one warm-up pass, then the timed pass
        for (int pass = 0; pass < 2 && st == BGK_OK; ++pass) {
            cu(cudaMemset(dsum, 0, sizeof(double)));
            cu(cudaEventRecord(e0));
            k_probe_fr_tc<<<sms, PTHREADS, PROBE_SMEM_LAUNCH>>>(map, dops, (int)n_panels, n_check, dout, dsum, dstat);
            cu(cudaGetLastError());
            cu(cudaEventRecord(e1));
            cu(cudaEventSynchronize(e1));
        }
        cu(cudaEventElapsedTime(&ms, e0, e1));
    }
    unsigned int hstat = 0;
    std::vector<float> hout((size_t)n_check * 3 * PNS * PN);
    if (st == BGK_OK) {
        cu(cudaMemcpy(&hstat, dstat, sizeof hstat, cudaMemcpyDeviceToHost));
        cu(cudaMemcpy(hout.data(), dout, hout.size() * sizeof(float), cudaMemcpyDeviceToHost));
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(dpan); cudaFree(dops); cudaFree(dout); cudaFree(dsum); cudaFree(dstat);
    if (st != BGK_OK) return st;
    if (hstat) return BGK_ETIMEOUT;

    // ---- the checked panels against FP64: the operator of the split applied
    // to the FP32 data (what the split would compute exactly, up to the
    // neglected lo.lo term), its largest relative error per output column,
    // and the relative bias of the sum of all outputs
    double max_rel = 0.0, bias_num = 0.0, bias_den = 0.0;
    for (int pnl = 0; pnl < n_check; ++pnl)
        for (int d = 0; d < 3; ++d)
            for (int n = 0; n < PN; ++n) {
                double colmax = 0.0, errmax = 0.0;
                for (int r = 0; r < PNS; ++r) {
                    double ref = 0.0, mag = 0.0;
                    for (int k = 0; k < PNS; ++k) {
                        const double a = opf[((size_t)d * PNS + r) * PNS + k], x = dat[((size_t)pnl * PN + n) * PNS + k];
                        ref += a * x;
                        mag += std::fabs(a * x);
                    }
                    const double got = hout[(((size_t)pnl * 3 + d) * PNS + r) * PN + n];
                    colmax = std::fmax(colmax, mag);
                    errmax = std::fmax(errmax, std::fabs(got - ref));
                    bias_num += ref > 0.0 ? got - ref : (ref < 0.0 ? ref - got : 0.0);
                    bias_den += std::fabs(ref);
                }
                max_rel = std::fmax(max_rel, errmax / colmax);
            }
    const double flops = (double)n_panels * 3.0 * 3.0 * 2.0 * 64.0 * PN * PNS;
    out[0] = flops / (ms * 1e-3);                       // useful MMA flop/s (three split products)
    out[1] = (double)n_panels * PN * PNS / (ms * 1e-3); // operator applications (DOF) per second, 3 directions
    out[2] = (double)total / (ms * 1e-3);               // operand bytes streamed per second
    out[3] = max_rel;                                   // vs sum |a x| of the output's terms
    out[4] = bias_num / bias_den;                       // sum (got - ref) sign(ref) / sum |ref|: < 0 = shrunk toward zero
    out[5] = ms;
    return BGK_OK;
}
