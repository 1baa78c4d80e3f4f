// bgk_moments_noalloc: the raw-moment reduction for callers that cannot
// allocate device memory.
//
// Who needs this: code that runs where cudaMalloc is not available or not
// allowed -- inside a memory pool that a host framework has already claimed
// in full, in a real-time loop that must not pay allocation latency or risk
// allocation failure, or in a plugin whose host forbids its own allocations.
// Such a caller owns its input and output buffers but cannot give this
// library a context (bgk_create allocates).  This entry point therefore
// keeps its scratch -- the per-velocity-block partial sums -- in one
// file-scope device array of fixed size, and allocates nothing.
//
// Scratch rules:
//  * The array below is BGK_NOALLOC_SCRATCH_DOUBLES doubles (16 MiB); every
//    GPU that loads libbgk holds it until the process exits.
//  * Every call shares it and leaves the last call's partial sums in it.
//    Each call writes every partial it later reads, so nothing needs to
//    start at zero.  Calls that overlap on the GPU (on different streams, or
//    from different host threads without ordering) race on it.
//  * Host code may not pass the array's name to a kernel: on the host that
//    name is only a stand-in, not a device address.  The device address is
//    looked up with cudaGetSymbolAddress for the context current on the
//    calling thread.  The set-up happens on the first call made with a
//    device current; later calls whose stream is not being captured look the
//    address up again (cheap), so a call from another context on the same
//    device (a plugin host's own driver-API context, or after
//    cudaDeviceReset) gets that context's address.  A call whose stream is
//    being captured uses the address the last uncaptured call on that
//    device found: make at least one call on the device, from the context
//    that will capture, before any stream capture begins.
#include <mutex>

#include "../../include/bgk.h"
#include "bgk_internal.cuh"

#define BGK_NOALLOC_SCRATCH_DOUBLES (1 << 21)
#define BGK_NOALLOC_MAX_DEVICES 64

static __device__ __align__(256) double g_moment_scratch[BGK_NOALLOC_SCRATCH_DOUBLES];

namespace {

std::mutex g_setup_mutex;
double *g_scratch_ptr[BGK_NOALLOC_MAX_DEVICES];

struct GridConsts {
    int n[3];
    double lo[3], h[3];
};

// Velocity node and trapezoid weight of index k (k1 fastest), from the grid
// descriptor itself, so no table needs to be allocated.
__device__ __forceinline__ void node(const GridConsts &g, int k, double u[3], double &w) {
    const int j[3] = {k % g.n[0], (k / g.n[0]) % g.n[1], k / (g.n[0] * g.n[1])};
    w = 1.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        u[d] = g.lo[d] + j[d] * g.h[d];
        w *= (j[d] == 0 || j[d] == g.n[d] - 1) ? 0.5 * g.h[d] : g.h[d];
    }
}

__global__ void __launch_bounds__(256) k_moments_partial_noalloc(const double *f, int C, int Nu, int P,
                                                                 int Kblk, GridConsts g, double *scr) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const int vb = blockIdx.y;
    const int k0 = vb * Kblk, k1 = min(Nu, k0 + Kblk);
    double m[BGK_NMOM];
#pragma unroll
    for (int j = 0; j < BGK_NMOM; ++j) m[j] = 0.0;
    for (int k = k0; k < k1; ++k) {
        double u[3], w;
        node(g, k, u, w);
        const double wF = w * f[(size_t)k * P + p];
        m[0] += wF;
        m[1] = fma(wF, u[0], m[1]);
        m[2] = fma(wF, u[1], m[2]);
        m[3] = fma(wF, u[2], m[3]);
        m[4] = fma(wF * u[0], u[0], m[4]);
        m[5] = fma(wF * u[1], u[1], m[5]);
        m[6] = fma(wF * u[2], u[2], m[6]);
        m[7] = fma(wF * u[0], u[1], m[7]);
        m[8] = fma(wF * u[0], u[2], m[8]);
        m[9] = fma(wF * u[1], u[2], m[9]);
        if (C == 2) m[10] = fma(w, f[((size_t)Nu + k) * P + p], m[10]);
    }
#pragma unroll
    for (int j = 0; j < BGK_NMOM; ++j) scr[((size_t)vb * BGK_NMOM + j) * P + p] = m[j];
}

__global__ void k_moments_finish_noalloc(const double *scr, int n_vblk, int P, double *m_out) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    for (int j = 0; j < BGK_NMOM; ++j) {
        double s = 0.0;
        for (int vb = 0; vb < n_vblk; ++vb) s += scr[((size_t)vb * BGK_NMOM + j) * P + p];
        m_out[(size_t)p * BGK_NMOM + j] = s;
    }
}

// Device address of the scratch array in the calling thread's current
// context: looked up whenever the stream is not being captured (and kept per
// device); during a capture the kept address is used (no lookup may run
// then).
cudaError_t scratch_for_current_device(cudaStream_t s, double **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= BGK_NOALLOC_MAX_DEVICES) return cudaErrorInvalidDevice;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (cs == cudaStreamCaptureStatusNone) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_moment_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = (double *)ptr;
    } else if (!g_scratch_ptr[dev]) {
        return cudaErrorStreamCaptureUnsupported;    // no uncaptured call on this device yet
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" BGK_API bgk_status bgk_moments_noalloc(const bgk_vgrid_desc *vgrid, const double *f,
                                                  int n_comp, int n_points, double *m, void *stream) {
    if (!vgrid || !f || !m || n_points <= 0 || (n_comp != 1 && n_comp != 2)) return BGK_EINVAL;
    GridConsts g;
    long long Nu = 1;
    for (int d = 0; d < 3; ++d) {
        if (vgrid->n[d] < 2 || !(vgrid->hi[d] > vgrid->lo[d])) return BGK_EINVAL;
        g.n[d] = vgrid->n[d];
        g.lo[d] = vgrid->lo[d];
        g.h[d] = (vgrid->hi[d] - vgrid->lo[d]) / (vgrid->n[d] - 1);
        Nu *= vgrid->n[d];
    }
    if (Nu > (1ll << 30)) return BGK_EINVAL;
    // Velocity blocks: enough CTAs to occupy the GPU, within the fixed scratch.
    const long long per_block = (long long)BGK_NMOM * n_points;
    if (per_block > BGK_NOALLOC_SCRATCH_DOUBLES) return BGK_EINVAL;   // n_points > 190650
    const int n_pb = (n_points + 255) / 256;
    long long n_vblk = (2432 + n_pb - 1) / n_pb;
    if (n_vblk > 64) n_vblk = 64;
    if (n_vblk > Nu) n_vblk = Nu;
    if (n_vblk > BGK_NOALLOC_SCRATCH_DOUBLES / per_block) n_vblk = BGK_NOALLOC_SCRATCH_DOUBLES / per_block;
    if (n_vblk < 1) n_vblk = 1;
    const int Kblk = (int)((Nu + n_vblk - 1) / n_vblk);
    n_vblk = (Nu + Kblk - 1) / Kblk;

    double *scr = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    if (scratch_for_current_device(s, &scr) != cudaSuccess) return BGK_ECUDA;
    dim3 grid(n_pb, (unsigned)n_vblk);
    k_moments_partial_noalloc<<<grid, 256, 0, s>>>(f, n_comp, (int)Nu, n_points, Kblk, g, scr);
    if (cudaGetLastError() != cudaSuccess) return BGK_ECUDA;
    k_moments_finish_noalloc<<<n_pb, 256, 0, s>>>(scr, (int)n_vblk, n_points, m);
    if (cudaGetLastError() != cudaSuccess) return BGK_ECUDA;
    return BGK_OK;
}
