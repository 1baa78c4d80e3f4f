// Internal declarations shared by the libbgk translation units.
// Kernel argument structs are passed by value (constant bank), so every
// operator table a kernel needs travels with its launch.
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

#include "bgk_mlp.cuh"

#define BGK_MAXQ 5          // FR order p <= 4
#define BGK_NMOM 11         // raw moment slots per point
#define BGK_NMACRO 10       // macroscopic fields per point (bgk_macro)
#define BGK_NEQ 20          // equilibrium record per point (12 used by the FP64 form)
// FP32 equilibrium record per point (mixed form), the FP32 values the stage
// kernels derive from the FP64 record, in the order they are used:
//   0 E0  1 V1  2 A11  3 1/tau  4 gamma1  5 gamma4/2  6 U0_1  7 gfac
//   8 V2  9 V3  10 A12  11 A13  12 A22  13 A23  14 A33  15 gamma0
//   16 gamma2  17 gamma3  18 U0_2  19 U0_3  20 gamma4  21..23 unused
#define BGK_NEQ32 24
// Curvilinear node record: S^1 (3), S^2 (3), S^3 (3) (S^d = J grad xi_d),
// 1/J, the quadrature weight W_s J_s, unused.
#define BGK_NGEO 12
// FP32 node record of the mixed form: S^1..S^3 (9), 1/J, then for the six
// faces 2d + side the difference S_face - S^d_node at the flux node on the
// node's line (18; formed in FP64), the node's geometric remainder H (3, see
// CurvOps32), unused.
#define BGK_NGEO32 32
// Non-periodic face kinds (face 2d + side).
#define BGK_FK_DIRICHLET 0
#define BGK_FK_SPECULAR 1
#define BGK_FK_DIFFUSE 2
#define BGK_FK_CLOSED 3
#define BGK_VTAB 8          // velocity table record: u1 u2 u3 w e=|u|^2/2 w*u1 w*u1^2 (2/h1)*u1
#define BGK_MAXV 128        // nodes per velocity axis at most

// Dynamic shared-memory limits a launcher has raised with cudaFuncSetAttribute,
// which acts on the calling thread's current device: one entry per device, so
// each device of a process gets its own call.
#define BGK_MAX_DEVICES 64
struct SmemLimit {
    size_t set[BGK_MAX_DEVICES] = {};
    // the current device's entry, or nullptr if the device cannot be queried
    size_t *slot() {
        int d = 0;
        if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= BGK_MAX_DEVICES) return nullptr;
        return &set[d];
    }
};

// Device status bits (OR-ed by kernels, read by the host after a stage).
#define BGK_DEV_NOCONV 1u
#define BGK_DEV_NONFINITE 2u
#define BGK_DEV_TIMEOUT 4u     // a bounded wait inside a kernel gave up

// FP32 stage kernel variants (bgk_set_stage_kernel) and the deepest copy ring.
#define BGK_STAGE_AUTO 0
#define BGK_STAGE_PLAIN 1
#define BGK_STAGE_ASYNC 2
#define BGK_STAGE_LINE 3        // asynchronous copies, one thread per node line, short runs
#define BGK_STAGE_LINE_WIDE 4   // the same with runs twice as long
#define BGK_STAGE_HALF 5        // asynchronous copies, one thread per half node line, short runs
#define BGK_STAGE_HALF_WIDE 6   // the same with runs twice as long
#define BGK_MAX_DEPTH 16

// 1-D FR operators on Gauss--Legendre nodes (section "Numerical method").
struct FROps {
    int q;                              // p + 1
    double D[BGK_MAXQ][BGK_MAXQ];       // D[i][j] = l_j'(xi_i)
    double lm[BGK_MAXQ], lp[BGK_MAXQ];  // l_j(-1), l_j(+1)
    double dgL[BGK_MAXQ], dgR[BGK_MAXQ];// correction-function derivatives at the nodes
    double wq[BGK_MAXQ];                // Gauss weights
    double xi[BGK_MAXQ];                // nodes
};

struct MeshInfo {
    int n[3];
    int periodic[3];
    int specular[6];                    // face 2d + side reflects specularly
    int face_kind[6];                   // BGK_FK_* of each non-periodic face
    double two_over_h[3];
    int Ne, Ns;
};

// Uniform velocity grid: node j on axis d is lo[d] + j h[d].  A context that
// holds a slab of the third axis (a velocity shard) sees the slab as its grid;
// w3lo / w3hi say whether the slab's first / last third-axis plane is an end of
// the whole grid (trapezoid half weight) or an interior plane (full weight).
struct VelGrid {
    int n[3];
    double lo[3], h[3];
    int w3lo, w3hi;
};

// Trapezoid factor of third-axis plane j3 of a (possibly sharded) grid.
__host__ __device__ __forceinline__ float trap3(int j3, const VelGrid &vg) {
    return ((j3 == 0 && vg.w3lo) || (j3 == vg.n[2] - 1 && vg.w3hi)) ? 0.5f : 1.0f;
}

struct GasInfo {
    double delta, Pr, mu_ref, theta_ref, theta_S, gamma;
};

// Velocity node k with its index on axis d mirrored (j_d -> n_d - 1 - j_d):
// the reflection u_d -> -u_d on a grid symmetric in axis d.
__device__ __forceinline__ int mirror_velocity(int k, int d, const int n[3]) {
    const int j1 = k % n[0], j2 = (k / n[0]) % n[1], j3 = k / (n[0] * n[1]);
    const int m1 = d == 0 ? n[0] - 1 - j1 : j1, m2 = d == 1 ? n[1] - 1 - j2 : j2, m3 = d == 2 ? n[2] - 1 - j3 : j3;
    return m1 + n[0] * (m2 + n[1] * m3);
}

// FP32 equilibrium exactly as the mixed-form stage evaluates it:
// g32(u) = E0 * exp2(L), L = -log2(e)/2 c^T A c, c = u - V, all in FP32 with
// every product rounded explicitly (no contraction), so the Q' kernel can
// reproduce the stage's values bit for bit when it measures their moments.
struct Eq32 {
    float E0, V1, V2, V3, A11, A22, A33, A12, A13, A23;   // A pre-scaled by -log2(e)/2 (x2 off-diagonal)
    __device__ __forceinline__ void load(const double *q) {
        const float s2 = -0.72134752044448170f;            // -log2(e)/2
        E0 = (float)exp(q[0]);
        V1 = (float)q[1]; V2 = (float)q[2]; V3 = (float)q[3];
        A11 = __fmul_rn((float)q[4], s2); A22 = __fmul_rn((float)q[5], s2);
        A33 = __fmul_rn((float)q[6], s2);
        A12 = __fmul_rn((float)q[7], 2.f * s2); A13 = __fmul_rn((float)q[8], 2.f * s2);
        A23 = __fmul_rn((float)q[9], 2.f * s2);
    }
    // the ten parameters in the order load() sets them (E0, V1..V3, A11..A23)
    __device__ __forceinline__ void set(const float *v) {
        E0 = v[0]; V1 = v[1]; V2 = v[2]; V3 = v[3];
        A11 = v[4]; A22 = v[5]; A33 = v[6]; A12 = v[7]; A13 = v[8]; A23 = v[9];
    }
    __device__ __forceinline__ void get(float *v) const {
        v[0] = E0; v[1] = V1; v[2] = V2; v[3] = V3;
        v[4] = A11; v[5] = A22; v[6] = A33; v[7] = A12; v[8] = A13; v[9] = A23;
    }
    // per first-axis line: the coefficient of c1 and the constant part
    __device__ __forceinline__ void line(float u2, float u3, float &lin, float &cst) const {
        const float c2 = __fsub_rn(u2, V2), c3 = __fsub_rn(u3, V3);
        lin = fmaf(A12, c2, __fmul_rn(A13, c3));
        cst = fmaf(__fmul_rn(A22, c2), c2, fmaf(__fmul_rn(A23, c2), c3, __fmul_rn(__fmul_rn(A33, c3), c3)));
    }
    __device__ __forceinline__ float g(float u1, float lin, float cst) const {
        const float c1 = __fsub_rn(u1, V1);
        return __fmul_rn(E0, ex2(fmaf(c1, fmaf(A11, c1, lin), cst)));
    }
    // 2^x on the special-function unit (a few ulp; the moment correction
    // absorbs the bias, and both kernels that use Eq32 see the same values)
    static __device__ __forceinline__ float ex2(float x) {
        float y;
        asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
        return y;
    }
};

// Newton statistics accumulated on the device.
struct NewtonStats {
    unsigned long long iter_sum;
    unsigned long long solves;
    int iter_max;
    int pad;
    unsigned long long res_max_bits;    // bit pattern of a non-negative double
};

// FP32 operator tables of the curvilinear mixed-form stage.  Per direction
// and node i of a line, with Ft_j = a_j f_j (a_j = u . S^d_j), the operator is
//   t_i = sum_{j != i} D_ij (Ft_j - Ft_i) - sum_j def_j (Ft_j - Ft_i)
//       + g_R'_i (A_R f^up_R - Ft_i - sum_j l_j(+1) (Ft_j - Ft_i)) + (left face)
// (the diagonal of D and the weight sums never enter, so the traces are exact
// for constant data).  g_L' is the mirror image of g_R' and l(-1) that of
// l(+1), so the two faces' lift weights sum_i W_i g'_i cancel exactly;
// def[j] is the defect, divided by sum_i W_i, of the column sums
// sum_i W_i (d t_i / d Ft_j) of the rounded operator (zero in exact
// arithmetic; its entries sum to zero): the element quadrature of the
// divergence then telescopes exactly for the stored coefficients.  The stage
// evaluates it regrouped, Ft_j - Ft_i = a_j (f_j - f_i) + (a_j - a_i) f_i: the
// sums act on deviations a_j (f_j - f_i), and every term proportional to f_i
// is geometry times u, summed over the three directions into the node's
// vector H (formed on the host in FP64 with these FP32 coefficients, about
// zero for a continuous mesh) and added as f_i u . H.
struct CurvOps32 {
    float D[BGK_MAXQ][BGK_MAXQ];
    float lp[BGK_MAXQ], lm[BGK_MAXQ];
    float dgL[BGK_MAXQ], dgR[BGK_MAXQ];
    float def[BGK_MAXQ];
};

// Arguments of the fused stage kernel:  f_out = a f_n + b f_s + c R(f_s).
template <typename T>
struct StageArgs {
    const T *f_n;            // may be null when a == 0
    const T *f_s;
    T *f_out;
    const double *eq;        // [P][BGK_NEQ]
    const double *vtab;      // [Nu][BGK_VTAB]
    const float4 *vtab32;    // [Nu] (u1, u2, u3, 0) rounded to FP32
    const double *bcval;     // [6][C][Nu] exterior Maxwellian values of Dirichlet faces
    double *part;            // [n_vblk][BGK_NMOM][P] moment partials of f_out (or null)
    const float *eq32;       // [P][BGK_NEQ32] (mixed form)
    // curvilinear meshes (all null on the uniform box)
    const T *geo;            // [P][BGK_NGEO]
    const T *fvec;           // [Ne][6][Q*Q][3] face vectors, oriented +xi_d
    const double *rho_w;     // [Ne][6][Q*Q] diffuse-wall densities of this stage's input
    CurvOps32 cops;          // FP32 operator tables (mixed form)
    unsigned int *status;    // device status word (BGK_DEV_* bits)
    double a, b, c;
    // FP32 copies made on the host: a, a + b, c, and the metric terms 2/h_d
    // (converting them in the kernel costs an FP64-pipe instruction each time
    // the compiler rematerialises them inside the velocity loop)
    float a32, ab32, c32, toh32[3];
    int Nu, P, Kblk;
    // bounded waits of the copy-ring kernels: limit (0: about 2 s), and the
    // number of velocities a block's ring delivers before it stops (0: all;
    // set only by the test entry bgk_test_ring_stall)
    unsigned long long wait_ns;
    int ring_limit;
    VelGrid vg;
    FROps fr;
    MeshInfo mesh;
};

struct QPrimeArgs {
    const double *part;      // [n_vblk][BGK_NMOM][P]
    int n_vblk;
    const double *vtab;
    const float4 *vtab32;
    const double *guess;     // [P][5] or null
    double *eq;              // [P][BGK_NEQ] or null
    float *eq32;             // [P][BGK_NEQ32] or null (written with eq)
    double *qp;              // [P][5] or null
    int *iters;              // [P] or null
    unsigned int *status;
    NewtonStats *stats;
    int P, Nu;
    double tol;              // stopping tolerance of the FP64 engine
    double tol32;            // stopping tolerance of the FP32-sum engine
    int max_iter;
    GasInfo gas;
    VelGrid vg;
    int mixed;               // also fit the FP32-equilibrium moment correction
    // learned initial guess and the training log
    MlpParams mlp;
    int guess_mode;          // 0: start from q, 1: start from the network's guess
    int mlp_bf16;
    float *log;              // [log_max][MLP_LOG_STRIDE] (features, Delta) of converged solves
    unsigned long long *log_count;
    long long log_max;
    unsigned long long *fallbacks;   // guesses rejected (restart from q)
};

struct MomentArgs64 {
    const double *f;
    double *part;
    const double *vtab;
    int Nu, P, Kblk, C;
};

// The 1-D FR operators of order p on Gauss--Legendre nodes (bgk_api.cu, host).
void fr_build_host(int p, FROps &fr);

// Curvilinear metric terms (geometry.cu, host): geo[P][BGK_NGEO],
// fvec[Ne][6][q*q][3]; false with err on a non-positive Jacobian.
#include <string>
#include <vector>
bool build_curved_geometry(const FROps &fr, const int n[3], const int periodic[3], const double *x,
                           std::vector<double> &geo, std::vector<double> &fvec, std::string &err);

// Diffuse-wall densities of a state (wall.cu): rho_w[e][f][fp] for the n_wall
// (element, face) pairs in wall_ef[2 * i], wall_ef[2 * i + 1].
template <typename T>
cudaError_t launch_wall_density(const T *f, const T *fvec, const double *bcval, const double *vtab,
                                const int *wall_ef, int n_wall, int q, int Ne, int Nu, int C, FROps fr,
                                double *rho_w, cudaStream_t s);

// Launchers: the Q' solve and its tensor refinement (kernels_qprime.cu); the
// FP64 moments, stage and Maxwellian (kernels_f64.cu); the FP32 moments and
// stage (kernels_f32.cu, the line kernels in kernels_f32_line.cu).
cudaError_t launch_moments_f64(const MomentArgs64 &a, int n_vblk, cudaStream_t s);
cudaError_t launch_qprime(const QPrimeArgs &a, bool fp32_sums, cudaStream_t s);
// tensor variant of the ES equilibrium: refines the eq record k_qprime wrote
cudaError_t launch_qprime_tensor(const QPrimeArgs &a, bool fp32_sums, cudaStream_t s);
cudaError_t launch_stage_f64(const StageArgs<double> &a, int C, int n_vblk, cudaStream_t s);
cudaError_t launch_maxwellian_f64(double *f, const double *q, const double *vtab, int Nu, int P,
                                  int C, double delta, cudaStream_t s);
cudaError_t launch_moments_f32(const float *f, double *part, const double *vtab, int Nu, int P,
                               int Kblk, int C, int n_vblk, cudaStream_t s);
cudaError_t launch_moments_f32_exact(const float *f, double *part, const VelGrid &vg, int Nu, int P, int Kblk,
                                     int C, int n_vblk, cudaStream_t s);
cudaError_t launch_stage_f32(const StageArgs<float> &a, int C, int n_vblk, int variant, int depth,
                             cudaStream_t s);
bool stage_f32_tma_supported(const StageArgs<float> &a, int C, int depth);
// line kernels: kind 0 line, 1 line_wide, 2 half, 3 half_wide
bool stage_f32_line_supported(const StageArgs<float> &a, int C, int kind, int depth);
cudaError_t launch_stage_f32_line(const StageArgs<float> &a, int C, int n_vblk, int kind, int depth, cudaStream_t s);
// any FP32 stage variant: is it available for these arguments
bool stage_f32_variant_supported(const StageArgs<float> &a, int C, int variant, int depth);
cudaError_t launch_maxwellian_f32(float *f, const double *q, const double *vtab, int Nu, int P, int C,
                                  double delta, cudaStream_t s);
cudaError_t launch_macro(const double *mom, double *out, int P, const MeshInfo &mesh, const FROps &fr,
                         const GasInfo &gas, const double face_rho[6], const double *geo, cudaStream_t s);
// per-point entropy sum_k w_k F ln F of the F component (kernels_f64.cu);
// part holds n_vblk * P doubles, *nonpos counts the non-positive values
template <typename T>
cudaError_t launch_entropy(const T *f, const double *vtab, int Nu, int P, int Kblk, int n_vblk, double *part,
                           double *h_out, unsigned int *nonpos, cudaStream_t s);
// out[j][p] = sum over velocity blocks of part[vb][j][p] (kernels_f64.cu):
// a shard's partial raw moments in the layout the Q' solve reads (one block)
cudaError_t launch_sum_partials(const double *part, int n_vblk, int P, double *out, cudaStream_t s);
cudaError_t launch_reduce_moments(const double *part, int n_vblk, int P, double *m_out,
                                  cudaStream_t s);
