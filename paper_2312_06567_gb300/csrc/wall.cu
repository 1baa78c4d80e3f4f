// Diffuse-wall densities (section "Implementation & problem setup": the wall
// is a weak boundary whose exterior state enters through the upwind flux).
// At every flux node of a diffuse face the particles entering the gas
// (u_n < 0, n the outward normal of the gas) are drawn from the wall
// Maxwellian rho_w M(u; U_w, theta_w); rho_w makes the node's net discrete
// mass flux vanish:
//     rho_w = - sum_{u_n > 0} w u_n F^- / sum_{u_n < 0} w u_n M(u; U_w, theta_w)
// with F^- the element's interior trace.  One block per (wall element, face),
// threads striding over the velocities, FP64 sums reduced across the block.
#include "bgk_internal.cuh"

namespace {

constexpr int WT = 256;

template <typename T, int Q>
__global__ void __launch_bounds__(WT) k_wall_density(const T *f, const T *fvec, const double *bcval,
                                                    const double *vtab, const int *wall_ef, int Ne, int Nu,
                                                    int C, FROps fr, double *rho_w) {
    constexpr int NS = Q * Q * Q, NF = Q * Q;
    __shared__ double red[WT / 32][2 * NF];
    __shared__ double nv[NF][3];
    __shared__ double lwr[Q];
    const int e = wall_ef[2 * blockIdx.x], face = wall_ef[2 * blockIdx.x + 1];
    const int d = face / 2, side = face % 2;
    if (threadIdx.x < NF * 3) {
        const int i = threadIdx.x / 3, c = threadIdx.x % 3;
        nv[i][c] = (side ? 1.0 : -1.0) * (double)fvec[(((size_t)e * 6 + face) * NF + i) * 3 + c];
    }
    if (threadIdx.x < Q) lwr[threadIdx.x] = side ? fr.lp[threadIdx.x] : fr.lm[threadIdx.x];
    __syncthreads();
    double num[NF], den[NF];
#pragma unroll
    for (int i = 0; i < NF; ++i) { num[i] = 0.0; den[i] = 0.0; }
    const size_t P = (size_t)Ne * NS;
    const int sd = d == 0 ? 1 : (d == 1 ? Q : Q * Q);           // node stride along the face normal
    const int sa = d == 0 ? Q : 1, sb = d == 2 ? Q : Q * Q;       // strides of the face point indices
    for (int k = threadIdx.x; k < Nu; k += WT) {
        const double *vt = vtab + (size_t)k * BGK_VTAB;
        const double u1 = vt[0], u2 = vt[1], u3 = vt[2], w = vt[3];
        const double M = bcval[((size_t)face * C + 0) * Nu + k];
        const T *fe = f + (size_t)k * P + (size_t)e * NS;
#pragma unroll
        for (int b = 0; b < Q; ++b)
#pragma unroll
            for (int a = 0; a < Q; ++a) {
                const int i = a + Q * b;
                const double un = u1 * nv[i][0] + u2 * nv[i][1] + u3 * nv[i][2];
                // the line of nodes through face point (a, b) along axis d
                const T *ln = fe + a * sa + b * sb;
                double tr = 0.0;
#pragma unroll
                for (int j = 0; j < Q; ++j) tr = fma(lwr[j], (double)ln[j * sd], tr);
                if (un > 0.0) num[i] = fma(w * un, tr, num[i]);
                else if (un < 0.0) den[i] = fma(w * un, M, den[i]);
            }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < NF; ++i) {
        double a = num[i], b = den[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            b += __shfl_xor_sync(0xffffffffu, b, o);
        }
        if (lane == 0) { red[warp][i] = a; red[warp][NF + i] = b; }
    }
    __syncthreads();
    if (threadIdx.x < NF) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < WT / 32; ++w) { a += red[w][threadIdx.x]; b += red[w][NF + threadIdx.x]; }
        rho_w[((size_t)e * 6 + face) * NF + threadIdx.x] = b < 0.0 ? -a / b : 0.0;
    }
}

template <typename T, int Q>
cudaError_t launch_q(const T *f, const T *fvec, const double *bcval, const double *vtab, const int *wall_ef,
                     int n_wall, int Ne, int Nu, int C, const FROps &fr, double *rho_w, cudaStream_t s) {
    k_wall_density<T, Q><<<n_wall, WT, 0, s>>>(f, fvec, bcval, vtab, wall_ef, Ne, Nu, C, fr, rho_w);
    return cudaGetLastError();
}

}  // namespace

template <typename T>
cudaError_t launch_wall_density(const T *f, const T *fvec, const double *bcval, const double *vtab,
                                const int *wall_ef, int n_wall, int q, int Ne, int Nu, int C, FROps fr,
                                double *rho_w, cudaStream_t s) {
    if (n_wall == 0) return cudaSuccess;
    switch (q) {
        case 2: return launch_q<T, 2>(f, fvec, bcval, vtab, wall_ef, n_wall, Ne, Nu, C, fr, rho_w, s);
        case 3: return launch_q<T, 3>(f, fvec, bcval, vtab, wall_ef, n_wall, Ne, Nu, C, fr, rho_w, s);
        case 4: return launch_q<T, 4>(f, fvec, bcval, vtab, wall_ef, n_wall, Ne, Nu, C, fr, rho_w, s);
        case 5: return launch_q<T, 5>(f, fvec, bcval, vtab, wall_ef, n_wall, Ne, Nu, C, fr, rho_w, s);
        default: return cudaErrorInvalidValue;
    }
}

template cudaError_t launch_wall_density<double>(const double *, const double *, const double *, const double *,
                                                 const int *, int, int, int, int, int, FROps, double *, cudaStream_t);
template cudaError_t launch_wall_density<float>(const float *, const float *, const double *, const double *,
                                                const int *, int, int, int, int, int, FROps, double *, cudaStream_t);
