// Mixed-precision (BGK_MIXED) kernels: the state f is FP32 and the FR
// advection, equilibrium evaluation, source and Runge--Kutta update run in
// FP32; the moments that feed the Q' solve are accumulated so that their
// error stays random (unbiased) and far below FP32 resolution, and the Q'
// solve itself runs in FP64 (the k_qprime_f64 kernel, shared with the FP64
// form).  Dzanic & Martinelli, arXiv 2312.06567, section "Methodology".
//
// Moment accumulation without systematic error: with centred velocity
// indices jt = j - jc on each axis (u = uc + jt h) and trapezoid factors
// c in {1/2, 1}, every coefficient c jt^a (|jt| < 64, a <= 2) is exact in
// FP32.  Along each first-axis line the sums L_a = sum c1 jt1^a F are FP32
// (a few tens of terms), the lines of one (j3 = const) plane are combined
// with exact coefficients c2 jt2^b in Kahan-compensated FP32, and the planes
// in FP64; the index moments J_abc = sum c F jt1^a jt2^b jt3^c are turned
// into the raw moments sum w u^alpha F in FP64 at the end.
#include <type_traits>

#include "stage_f32_common.cuh"

namespace {

// packed FP32 helpers (two IEEE operations per issue)
__device__ __forceinline__ float2 pdup(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 pneg(float2 v) { return make_float2(-v.x, -v.y); }
__device__ __forceinline__ float2 psub(float2 x, float2 y) { return __ffma2_rn(y, make_float2(-1.f, -1.f), x); }

// ---------------------------------------------------------------------------
// Fused stage, FP32 state.  Same discretisation as the FP64 stage kernel
// (all FP32 stage kernels sum each node's own-line terms in the order
// j = i+1, ..., i+Q-1 mod Q, so their results agree bit for bit):
// per direction t_d = sum_j Dt[side][i][j] f_j + dg[side][i] f^+ with the
// inflow trace folded into Dt; div = sum_d (2/h_d) u_d t_d;
// R = -div + (g' - f)/tau.  g' = exp(c0) * exp2(-log2(e)/2 c^T A c) with the
// per-point factor exp(c0) from FP64 and the exponent in FP32.
//
// Curvilinear elements (CURV): the transformed-flux form of the FP64 stage
// kernel (kernels_f64.cu) in FP32, regrouped so that every rounding acts on
// deviations (see CurvOps32).  a_d = u . S^d per node is staged beside f; per
// direction, with w_j = a_j (f_j - f_i),
//   t_i = sum_{j != i} D_ij w_j - sum_j def_j w_j
//       + g_R'_i (A_R dev_R - sum_j l_j(+1) w_j) + g_L'_i (A_L dev_L - sum_j l_j(-1) w_j),
// A = a_i + u.(S_face - S_i) the face's normal velocity, dev = (upwind trace)
// - f_i: the own trace sum_j l_j (f_j - f_i) on an outflow face, the
// neighbour's sum_j l_j (nb_j - f_i) or the exterior value minus f_i on an
// inflow face, -f_i on a closed face (F^I = 0); then
// div = (1/J) (sum_d t_d + f_i u . H).  This is the FP64 kernel's F^I - trace
// form term for term in exact arithmetic; constant data and the exact
// telescoping of the element quadrature survive the FP32 arithmetic.
template <int Q, int C, bool CURV>
// Held to 128 registers (two blocks, 16 warps per SM; the curvilinear
// instantiation keeps its geometry in shared memory): 1.7x faster on the
// sphere O-grid at p = 1 than one block of 8 warps without the cap.
#ifndef BGK_PLAIN_MINB
#define BGK_PLAIN_MINB 2
#endif
__global__ void __launch_bounds__(256, BGK_PLAIN_MINB) k_stage_f32(StageArgs<float> a) {
    constexpr int NS = Q * Q * Q;
    constexpr int EB = 256 / NS;
    constexpr int NT = EB * NS;
    __shared__ float sf[2][C][NT];
    __shared__ float sA[CURV ? 2 : 1][CURV ? 3 : 1][CURV ? NT : 1];    // a_d = u . S^d (CURV)
    // CURV: the block's node records (S^1..S^3, H, 1/J; odd stride, no bank
    // conflicts), face vectors, and per velocity the face points' u . S_face
    constexpr int NFA = CURV ? EB * 6 * Q * Q : 1;
    __shared__ float sG[CURV ? NT : 1][13];
    __shared__ float sFv[NFA][3];
    __shared__ float sAf[CURV ? 2 : 1][NFA];
    __shared__ float cD[CURV ? Q : 1][CURV ? Q : 1];     // D (CURV)
    __shared__ float cl[2][CURV ? Q : 1];                // l(+1), l(-1) (CURV)
    __shared__ float cg[2][CURV ? Q : 1];                // g_L', g_R' (CURV)
    __shared__ float cdef[CURV ? Q : 1];                 // column-sum defects of D (CURV)
    __shared__ float sD[2][Q][Q];         // Dt = D - dg (x) l, FP32
    __shared__ float sdg[2][Q];           // dg (FP32)
    __shared__ float seps[2][Q];          // eps_i = sum_j Dt_ij + dg_i  (exact defect, tiny)
    __shared__ float slam[2][Q];          // neighbour-trace weights lambda_j
    __shared__ float sdlam[2];            // sum_j lambda_j - 1 (exact defect, tiny)
    // CURV: the moment accumulators (the FP64 index moments [11][NT], then the
    // plane pairs [14][NT]) live in dynamic shared memory, leaving the
    // registers to the curvilinear operator
    extern __shared__ __align__(16) double dyn_acc[];
    const int tid = threadIdx.x;
    // Operators and the deviation form.  With f_i the thread's own value,
    //   t_i = sum_j Dt_ij (f_j - f_i) + dg_i dn + eps_i f_i,
    //   dn  = sum_j lambda_j (nb_j - f_i) + dlam f_i   (= f^+ - f_i),
    // equals sum_j Dt_ij f_j + dg_i f^+ in exact arithmetic.  Every product
    // with an O(1) coefficient acts on a deviation, so FP32 cancellation error
    // no longer repeats coherently across velocities and elements; lambda_j
    // = +-sum_i W_i Dt_ij (side L: the left neighbour's right trace, side R:
    // the right neighbour's left trace) makes sum_i W_i t_i telescope between
    // neighbours, which keeps the advection discretely conservative up to
    // second-order rounding terms.
    load_ops_f32<Q>(a.fr, tid, sD, sdg, seps, slam, sdlam);
    if constexpr (CURV) {
        if (tid < Q * Q) cD[tid / Q][tid % Q] = a.cops.D[tid / Q][tid % Q];
        if (tid < Q) {
            cl[0][tid] = a.cops.lp[tid]; cl[1][tid] = a.cops.lm[tid];
            cg[0][tid] = a.cops.dgL[tid]; cg[1][tid] = a.cops.dgR[tid];
            cdef[tid] = a.cops.def[tid];
        }
    }
    const int e0 = blockIdx.x * EB;
    const int le = tid / NS, s = tid - le * NS;
    const int e = e0 + le;
    const bool active = tid < NT && e < a.mesh.Ne;
    const int p = e * NS + s;
    const int vb = blockIdx.y;
    const int k0 = vb * a.Kblk;
    const int k1 = min(a.Nu, k0 + a.Kblk);
    const int id[3] = {s % Q, (s / Q) % Q, s / (Q * Q)};
    const int stride[3] = {1, Q, Q * Q};
    const int n1 = a.mesh.n[0], n2 = a.mesh.n[1], n3 = a.mesh.n[2];
    const int ec[3] = {e % n1, (e / n1) % n2, e / (n1 * n2)};
    const int estr[3] = {1, n1, n1 * n2};
    const int nn[3] = {n1, n2, n3};
    int en_[3][2], base[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        en_[d][0] = ec[d] > 0 ? e - estr[d] : (a.mesh.periodic[d] ? e + (nn[d] - 1) * estr[d] : -1);
        en_[d][1] = ec[d] < nn[d] - 1 ? e + estr[d] : (a.mesh.periodic[d] ? e - (nn[d] - 1) * estr[d] : -1);
        base[d] = s - id[d] * stride[d];
    }
    if constexpr (CURV) {
        if (tid < NT) {
            const float *g = a.geo + (size_t)p * BGK_NGEO32;
#pragma unroll
            for (int i = 0; i < 9; ++i) sG[tid][i] = active ? g[i] : 0.f;
            sG[tid][9] = active ? g[28] : 0.f;
            sG[tid][10] = active ? g[29] : 0.f;
            sG[tid][11] = active ? g[30] : 0.f;
            sG[tid][12] = active ? g[9] : 0.f;
        }
        for (int r = tid; r < NFA * 3; r += blockDim.x) {
            const int el = r / (6 * Q * Q * 3);
            sFv[r / 3][r % 3] = e0 + el < a.mesh.Ne ? a.fvec[(size_t)e0 * 6 * Q * Q * 3 + r] : 0.f;
        }
    }
    Eq32 e32;
    float itau = 0.f, gfac = 0.f;
    float gm[5] = {0.f, 0.f, 0.f, 0.f, 0.f}, U0f[3] = {0.f, 0.f, 0.f};
    {
        const double qz[10] = {0.0, 0.0, 0.0, 0.0, 1.0, 1.0, 1.0, 0.0, 0.0, 0.0};
        const double *q = active ? a.eq + (size_t)p * BGK_NEQ : qz;
        e32.load(q);
        if (active) {
            itau = (float)q[10]; gfac = (float)q[11];
#pragma unroll
            for (int i = 0; i < 5; ++i) gm[i] = (float)q[12 + i];
            U0f[0] = (float)q[17]; U0f[1] = (float)q[18]; U0f[2] = (float)q[19];
        }
    }
    const VelGrid &vg = a.vg;
    const int vn1 = vg.n[0], vn2 = vg.n[1], vn3 = vg.n[2];
    const int jc[3] = {(vn1 - 1) / 2, (vn2 - 1) / 2, (vn3 - 1) / 2};
    const double uc[3] = {vg.lo[0] + jc[0] * vg.h[0], vg.lo[1] + jc[1] * vg.h[1], vg.lo[2] + jc[2] * vg.h[2]};
    const float toh[3] = {a.toh32[0], a.toh32[1], a.toh32[2]};
    // f_out = a f^n + b f + c R written as (a + b) f + a (f^n - f) + c R: for
    // SSP-RK3 a + b = 1 exactly, which FP32 roundings of a and b would not keep
    // (1/3 and 2/3 both round up in FP32, a 3e-8 mass gain per step).
    const float fa = a.a32, fab = a.ab32, fc = a.c32;
    typename std::conditional<CURV, IndexMomentsS, IndexMoments>::type acc;
    if constexpr (CURV) acc.init(reinterpret_cast<float *>(dyn_acc + 11 * NT), dyn_acc, NT, tid);
    else acc.init();
    const size_t slab = (size_t)a.P;
    __syncthreads();

    int buf = 0;
    for (int kl = k0; kl < k1; kl += vn1) {
        const int line = kl / vn1;
        const int j2 = line % vn2, j3 = line / vn2;
        if (j3 != acc.j3cur) {
            if (acc.j3cur >= 0) acc.flush_plane(trap3(acc.j3cur, vg), (float)(acc.j3cur - jc[2]));
            acc.j3cur = j3;
        }
        const float4 vl = __ldg(a.vtab32 + kl);
        const float u2 = vl.y, u3 = vl.z;
        float lin, cst;
        e32.line(u2, u3, lin, cst);
        // moment correction gamma . phi(ut): the part that is constant on the line
        const float t2 = u2 - U0f[1], t3 = u3 - U0f[2];
        const float corr_line = fmaf(gm[2], t2, fmaf(gm[3], t3, fmaf(0.5f * gm[4], fmaf(t2, t2, t3 * t3), gm[0])));
        float jt1 = (float)(-jc[0]);                  // centred index as a float counter
        for (int j1 = 0; j1 < vn1; ++j1, jt1 += 1.f) {
            const int k = kl + j1;
            float fself[C];
            float ad[3] = {0.f, 0.f, 0.f};
            if constexpr (CURV) {
                const float uu1 = __ldg(a.vtab32 + k).x;
                for (int r = tid; r < NFA; r += blockDim.x)
                    sAf[buf][r] = fmaf(uu1, sFv[r][0], fmaf(u2, sFv[r][1], u3 * sFv[r][2]));
            }
            if (active) {
                if constexpr (CURV) {
                    const float uu[3] = {__ldg(a.vtab32 + k).x, u2, u3};
#pragma unroll
                    for (int d = 0; d < 3; ++d)
                        ad[d] = fmaf(uu[0], sG[tid][3 * d], fmaf(uu[1], sG[tid][3 * d + 1], uu[2] * sG[tid][3 * d + 2]));
                }
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    fself[c] = __ldg(a.f_s + ((size_t)c * a.Nu + k) * slab + p);
                    sf[buf][c][tid] = fself[c];
                }
                if constexpr (CURV) {
#pragma unroll
                    for (int d = 0; d < 3; ++d) sA[buf][d][tid] = ad[d];
                }
            }
            __syncthreads();
            if (active) {
                const float u1 = __ldg(a.vtab32 + k).x;
                const float u[3] = {u1, u2, u3};
                const float g32 = e32.g(u1, lin, cst);
                const float t1 = u1 - U0f[0];
                const float corr = fmaf(t1, fmaf(0.5f * gm[4], t1, gm[1]), corr_line);
                // The correction g32 * corr is a fraction of an ulp of g32; it is
                // added to the residual (whose exact value has random low bits,
                // so the rounding stays unbiased), never rounded into g itself.
                const float gc = __fmul_rn(g32, corr);
                float outv[C];
                if constexpr (CURV && C == 2) {
                    // curvilinear, F and G: the per-component body below on the pair
                    // (F, G) -- the two components share the geometry, the face
                    // normal velocities, the upwind decisions and the equilibrium
                    const float2 fi2 = make_float2(fself[0], fself[1]), nfi2 = pneg(fi2);
                    const float *fs0 = a.f_s + (size_t)k * slab, *fs1 = a.f_s + ((size_t)a.Nu + k) * slab;
                    float2 div = pdup(0.f);
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        const float *own0 = sf[buf][0] + le * NS + base[d], *own1 = sf[buf][1] + le * NS + base[d];
                        const float *ownA = sA[buf][d] + le * NS + base[d];
                        float2 dF = pdup(0.f), E = dF, trL = dF, trR = dF, fmL = dF, fmR = dF;
#pragma unroll
                        for (int m = 1; m < Q; ++m) {
                            const int j = (id[d] + m) % Q;
                            const float2 dfj = __fadd2_rn(make_float2(own0[j * stride[d]], own1[j * stride[d]]), nfi2);
                            const float2 wj = __fmul2_rn(pdup(ownA[j * stride[d]]), dfj);
                            dF = __ffma2_rn(pdup(cD[id[d]][j]), wj, dF);
                            E = __ffma2_rn(pdup(cdef[j]), wj, E);
                            trL = __ffma2_rn(pdup(cl[1][j]), wj, trL);
                            trR = __ffma2_rn(pdup(cl[0][j]), wj, trR);
                            fmL = __ffma2_rn(pdup(cl[1][j]), dfj, fmL);
                            fmR = __ffma2_rn(pdup(cl[0][j]), dfj, fmR);
                        }
                        float2 X[2];
#pragma unroll
                        for (int side = 0; side < 2; ++side) {
                            const int fpi = d == 0 ? id[1] + Q * id[2] : (d == 1 ? id[0] + Q * id[2] : id[0] + Q * id[1]);
                            const float A = sAf[buf][(le * 6 + 2 * d + side) * Q * Q + fpi];
                            const float un = side ? A : -A;               // outward
                            const int en = en_[d][side];
                            const int kind = a.mesh.face_kind[2 * d + side];
                            float2 dev;
                            if (en < 0 && kind == BGK_FK_CLOSED) {
                                dev = nfi2;                               // F^I = 0
                            } else if (un > 0.f) {
                                dev = side ? fmR : fmL;
                            } else if (en >= e0 && en < e0 + EB) {
                                const float *nb0 = sf[buf][0] + (en - e0) * NS + base[d];
                                const float *nb1 = sf[buf][1] + (en - e0) * NS + base[d];
                                dev = pdup(0.f);
#pragma unroll
                                for (int j = 0; j < Q; ++j)
                                    dev = __ffma2_rn(pdup(cl[side][j]),
                                                     __fadd2_rn(make_float2(nb0[j * stride[d]], nb1[j * stride[d]]), nfi2), dev);
                            } else if (en >= 0) {
                                const float *nb0 = fs0 + (size_t)en * NS + base[d], *nb1 = fs1 + (size_t)en * NS + base[d];
                                dev = pdup(0.f);
#pragma unroll
                                for (int j = 0; j < Q; ++j)
                                    dev = __ffma2_rn(pdup(cl[side][j]),
                                                     __fadd2_rn(make_float2(__ldg(nb0 + j * stride[d]), __ldg(nb1 + j * stride[d])), nfi2),
                                                     dev);
                            } else {
                                double fp0 = __ldg(a.bcval + ((size_t)(2 * d + side) * C + 0) * a.Nu + k);
                                double fp1 = __ldg(a.bcval + ((size_t)(2 * d + side) * C + 1) * a.Nu + k);
                                if (kind == BGK_FK_DIFFUSE) {
                                    const double rw = __ldg(a.rho_w + ((size_t)e * 6 + 2 * d + side) * Q * Q + fpi);
                                    fp0 *= rw;
                                    fp1 *= rw;
                                }
                                dev = __fadd2_rn(make_float2((float)fp0, (float)fp1), nfi2);
                            }
                            X[side] = __ffma2_rn(pdup(A), dev, pneg(side ? trR : trL));
                        }
                        div = __fadd2_rn(div, __ffma2_rn(X[1], pdup(cg[1][id[d]]),
                                                         __ffma2_rn(X[0], pdup(cg[0][id[d]]), psub(dF, E))));
                    }
                    const float uH = fmaf(u[0], sG[tid][9], fmaf(u[1], sG[tid][10], u[2] * sG[tid][11]));
                    div = __fmul2_rn(__ffma2_rn(fi2, pdup(uH), div), pdup(sG[tid][12]));
                    const float2 eqv = make_float2(g32, __fmul_rn(gfac, g32));
                    const float2 eqc = make_float2(gc, __fmul_rn(gfac, gc));
                    const float2 it2 = pdup(itau);
                    const float2 R = __ffma2_rn(psub(eqv, fi2), it2, __ffma2_rn(eqc, it2, pneg(div)));
                    const float2 fn2 = fa != 0.f ? make_float2(__ldg(a.f_n + (size_t)k * slab + p),
                                                               __ldg(a.f_n + ((size_t)a.Nu + k) * slab + p))
                                                 : pdup(0.f);
                    const float2 out = rk_update2(fi2, fn2, R, fa, fab, fc, fa != 0.f);
                    a.f_out[(size_t)k * slab + p] = out.x;
                    a.f_out[((size_t)a.Nu + k) * slab + p] = out.y;
                    outv[0] = out.x;
                    outv[C - 1] = out.y;
                } else if constexpr (!CURV && C == 2) {
                    // box, F and G: each component's operations exactly as in the
                    // scalar body below, on the pair (F, G)
                    const float2 fi2 = make_float2(fself[0], fself[1]), nfi2 = pneg(fi2);
                    const float *fs0 = a.f_s + (size_t)k * slab, *fs1 = a.f_s + ((size_t)a.Nu + k) * slab;
                    float2 div = pdup(0.f);
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        const int side = u[d] > 0.f ? 0 : 1;
                        const float *own0 = sf[buf][0] + le * NS + base[d], *own1 = sf[buf][1] + le * NS + base[d];
                        float2 t = pdup(0.f);
#pragma unroll
                        for (int m = 1; m < Q; ++m) {
                            const int j = (id[d] + m) % Q;
                            t = __ffma2_rn(pdup(sD[side][id[d]][j]),
                                           __fadd2_rn(make_float2(own0[j * stride[d]], own1[j * stride[d]]), nfi2), t);
                        }
                        const int en = side ? en_[d][1] : en_[d][0];
                        float2 dn;
                        if (en >= e0 && en < e0 + EB) {
                            const float *nb0 = sf[buf][0] + (en - e0) * NS + base[d];
                            const float *nb1 = sf[buf][1] + (en - e0) * NS + base[d];
                            dn = __fmul2_rn(pdup(sdlam[side]), fi2);
#pragma unroll
                            for (int j = 0; j < Q; ++j)
                                dn = __ffma2_rn(pdup(slam[side][j]),
                                                __fadd2_rn(make_float2(nb0[j * stride[d]], nb1[j * stride[d]]), nfi2), dn);
                        } else if (en >= 0) {
                            const float *nb0 = fs0 + (size_t)en * NS + base[d], *nb1 = fs1 + (size_t)en * NS + base[d];
                            dn = __fmul2_rn(pdup(sdlam[side]), fi2);
#pragma unroll
                            for (int j = 0; j < Q; ++j)
                                dn = __ffma2_rn(pdup(slam[side][j]),
                                                __fadd2_rn(make_float2(__ldg(nb0 + j * stride[d]), __ldg(nb1 + j * stride[d])), nfi2),
                                                dn);
                        } else if (a.mesh.specular[2 * d + side]) {
                            const int km = mirror_velocity(k, d, a.vg.n);
                            const float *mr0 = a.f_s + (size_t)km * slab + (size_t)e * NS + base[d];
                            const float *mr1 = a.f_s + ((size_t)a.Nu + km) * slab + (size_t)e * NS + base[d];
                            dn = __fmul2_rn(pdup(sdlam[1 - side]), fi2);
#pragma unroll
                            for (int j = 0; j < Q; ++j)
                                dn = __ffma2_rn(pdup(slam[1 - side][j]),
                                                __fadd2_rn(make_float2(__ldg(mr0 + j * stride[d]), __ldg(mr1 + j * stride[d])), nfi2),
                                                dn);
                        } else {
                            dn = __fadd2_rn(make_float2((float)__ldg(a.bcval + ((size_t)(2 * d + side) * C + 0) * a.Nu + k),
                                                        (float)__ldg(a.bcval + ((size_t)(2 * d + side) * C + 1) * a.Nu + k)),
                                            nfi2);
                        }
                        t = __ffma2_rn(pdup(sdg[side][id[d]]), dn, __ffma2_rn(pdup(seps[side][id[d]]), fi2, t));
                        div = __ffma2_rn(pdup(toh[d] * u[d]), t, div);
                    }
                    const float2 eqv = make_float2(g32, __fmul_rn(gfac, g32));
                    const float2 eqc = make_float2(gc, __fmul_rn(gfac, gc));
                    const float2 it2 = pdup(itau);
                    const float2 R = __ffma2_rn(psub(eqv, fi2), it2, __ffma2_rn(eqc, it2, pneg(div)));
                    const float2 fn2 = fa != 0.f ? make_float2(__ldg(a.f_n + (size_t)k * slab + p),
                                                               __ldg(a.f_n + ((size_t)a.Nu + k) * slab + p))
                                                 : pdup(0.f);
                    const float2 out = rk_update2(fi2, fn2, R, fa, fab, fc, fa != 0.f);
                    a.f_out[(size_t)k * slab + p] = out.x;
                    a.f_out[((size_t)a.Nu + k) * slab + p] = out.y;
                    outv[0] = out.x;
                    outv[C - 1] = out.y;
                } else {
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    const float *fs = a.f_s + ((size_t)c * a.Nu + k) * slab;
                    const float *sfc = sf[buf][c];
                    const float fi = fself[c];
                    float div = 0.f;
                    if constexpr (CURV) {
#pragma unroll
                        for (int d = 0; d < 3; ++d) {
                            const float *own = sfc + le * NS + base[d];
                            const float *ownA = sA[buf][d] + le * NS + base[d];
                            float dF = 0.f, E = 0.f, trL = 0.f, trR = 0.f, fmL = 0.f, fmR = 0.f;
#pragma unroll
                            for (int m = 1; m < Q; ++m) {
                                const int j = (id[d] + m) % Q;
                                const float dfj = own[j * stride[d]] - fi;
                                const float wj = ownA[j * stride[d]] * dfj;
                                dF = fmaf(cD[id[d]][j], wj, dF);
                                E = fmaf(cdef[j], wj, E);
                                trL = fmaf(cl[1][j], wj, trL);
                                trR = fmaf(cl[0][j], wj, trR);
                                fmL = fmaf(cl[1][j], dfj, fmL);
                                fmR = fmaf(cl[0][j], dfj, fmR);
                            }
                            float X[2];
#pragma unroll
                            for (int side = 0; side < 2; ++side) {
                                const int fpi = d == 0 ? id[1] + Q * id[2] : (d == 1 ? id[0] + Q * id[2] : id[0] + Q * id[1]);
                                const float A = sAf[buf][(le * 6 + 2 * d + side) * Q * Q + fpi];
                                const float un = side ? A : -A;           // outward
                                const int en = en_[d][side];
                                const int kind = a.mesh.face_kind[2 * d + side];
                                float dev;
                                if (en < 0 && kind == BGK_FK_CLOSED) {
                                    dev = -fi;                            // F^I = 0
                                } else if (un > 0.f) {
                                    dev = side ? fmR : fmL;
                                } else if (en >= e0 && en < e0 + EB) {
                                    const float *nb = sfc + (en - e0) * NS + base[d];
                                    dev = 0.f;
#pragma unroll
                                    for (int j = 0; j < Q; ++j) dev = fmaf(cl[side][j], nb[j * stride[d]] - fi, dev);
                                } else if (en >= 0) {
                                    const float *nb = fs + (size_t)en * NS + base[d];
                                    dev = 0.f;
#pragma unroll
                                    for (int j = 0; j < Q; ++j) dev = fmaf(cl[side][j], __ldg(nb + j * stride[d]) - fi, dev);
                                } else {
                                    double fpd = __ldg(a.bcval + ((size_t)(2 * d + side) * C + c) * a.Nu + k);
                                    if (kind == BGK_FK_DIFFUSE)
                                        fpd *= __ldg(a.rho_w + ((size_t)e * 6 + 2 * d + side) * Q * Q + fpi);
                                    dev = (float)fpd - fi;
                                }
                                X[side] = fmaf(A, dev, -(side ? trR : trL));
                            }
                            div += fmaf(X[1], cg[1][id[d]], fmaf(X[0], cg[0][id[d]], dF - E));
                        }
                        div = fmaf(fi, fmaf(u[0], sG[tid][9], fmaf(u[1], sG[tid][10], u[2] * sG[tid][11])), div);
                        div *= sG[tid][12];
                    } else {
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        const int side = u[d] > 0.f ? 0 : 1;
                        const float *own = sfc + le * NS + base[d];
                        float t = 0.f;
#pragma unroll
                        // own-line sum in the canonical order j = i+1, ..., i+Q-1 (mod Q);
                        // the j = i term is zero
#pragma unroll
                        for (int m = 1; m < Q; ++m) {
                            const int j = (id[d] + m) % Q;
                            t = fmaf(sD[side][id[d]][j], own[j * stride[d]] - fi, t);
                        }
                        const int en = side ? en_[d][1] : en_[d][0];
                        float dn;
                        if (en >= e0 && en < e0 + EB) {
                            const float *nb = sfc + (en - e0) * NS + base[d];
                            dn = sdlam[side] * fi;
#pragma unroll
                            for (int j = 0; j < Q; ++j) dn = fmaf(slam[side][j], nb[j * stride[d]] - fi, dn);
                        } else if (en >= 0) {
                            const float *nb = fs + (size_t)en * NS + base[d];
                            dn = sdlam[side] * fi;
#pragma unroll
                            for (int j = 0; j < Q; ++j) dn = fmaf(slam[side][j], __ldg(nb + j * stride[d]) - fi, dn);
                        } else if (a.mesh.specular[2 * d + side]) {
                            // the element's own outflow trace through this face at the
                            // mirrored velocity, with the weights of that outflow, so the
                            // reflected inflow telescopes against it exactly
                            const float *mr = a.f_s + ((size_t)c * a.Nu + mirror_velocity(k, d, a.vg.n)) * slab +
                                              (size_t)e * NS + base[d];
                            dn = sdlam[1 - side] * fi;
#pragma unroll
                            for (int j = 0; j < Q; ++j) dn = fmaf(slam[1 - side][j], __ldg(mr + j * stride[d]) - fi, dn);
                        } else {
                            dn = (float)__ldg(a.bcval + ((size_t)(2 * d + side) * C + c) * a.Nu + k) - fi;
                        }
                        t = fmaf(sdg[side][id[d]], dn, fmaf(seps[side][id[d]], fi, t));
                        div = fmaf(toh[d] * u[d], t, div);
                    }
                    }
                    const float eqv = (c == 0) ? g32 : __fmul_rn(gfac, g32);
                    const float eqc = (c == 0) ? gc : __fmul_rn(gfac, gc);
                    const float R = fmaf(eqv - fself[c], itau, fmaf(eqc, itau, -div));
                    const float fn = fa != 0.f ? __ldg(a.f_n + ((size_t)c * a.Nu + k) * slab + p) : 0.f;
                    const float out = rk_update(fself[c], fn, R, fa, fab, fc, fa != 0.f);
                    a.f_out[((size_t)c * a.Nu + k) * slab + p] = out;
                    outv[c] = out;
                }
                }
                acc.add(trap(j1, vn1), jt1, outv[0], C == 2 ? outv[C - 1] : 0.f);
            }
            buf ^= 1;
        }
        acc.end_line(trap(j2, vn2), (float)(j2 - jc[1]));
    }
    if (acc.j3cur >= 0) acc.flush_plane(trap3(acc.j3cur, vg), (float)(acc.j3cur - jc[2]));
    if (a.part && active) {
        double m[BGK_NMOM], Jv[11];
        if constexpr (CURV) acc.get(Jv);
        else
#pragma unroll
            for (int q = 0; q < 11; ++q) Jv[q] = acc.J[q];
        index_to_raw(Jv, vg, uc, m);
#pragma unroll
        for (int j = 0; j < BGK_NMOM; ++j) a.part[((size_t)vb * BGK_NMOM + j) * a.P + p] = m[j];
    }
}

// ---------------------------------------------------------------------------
// Fused FP32 stage with asynchronous staging.  The arithmetic is that of
// k_stage_f32, term for term; only the source of the operands differs.  A
// block owns a run of EB consecutive elements of one mesh row (first axis).
// For each velocity it needs its own values, the upwind neighbour element
// along the first axis (outside the run only at its two ends), the upwind
// neighbour runs along the second and third axes (each contiguous in the
// [k][e][s] layout) and f^n.  One producer thread copies these with bulk
// asynchronous copies (cp.async.bulk, completion counted in bytes on an
// mbarrier) into a ring of S stage buffers, up to S velocities ahead of the
// consumer warps, which wait on the stage's "full" barrier, compute from
// shared memory and release the stage on its "empty" barrier.  Every wait
// is bounded (about 2 s): a wait that gives up sets BGK_DEV_TIMEOUT, and the
// producer then waits, again bounded, for its copies still in flight before
// the block exits.
template <int Q, int C>
struct TmaGeom {
    static constexpr int NS = Q * Q * Q;
    static constexpr int EB = 256 / NS;                  // elements per block
    static constexpr int NCT = (EB * NS + 31) / 32 * 32;  // consumer threads
    static constexpr int NTHR = NCT + 32;                 // + one producer warp
    static constexpr int SLOTS = StageGeom<Q, C, EB>::SLOTS;
    static constexpr int PER_C = StageGeom<Q, C, EB>::PER_C;
    static constexpr int STAGE = StageGeom<Q, C, EB>::STAGE;
};


template <int Q, int C>
__global__ void __launch_bounds__(TmaGeom<Q, C>::NTHR, 2) k_stage_f32_tma(StageArgs<float> a, int S) {
    using G = TmaGeom<Q, C>;
    constexpr int NS = G::NS, EB = G::EB, NCT = G::NCT, SLOTS = G::SLOTS, PER_C = G::PER_C, STAGE = G::STAGE;
    extern __shared__ __align__(128) float sbuf[];
    // [S][STAGE] copy ring | [11][NCT] FP64 index moments | [14][NCT] plane pairs | 2S mbarriers
    double *Jsm = reinterpret_cast<double *>(sbuf + (size_t)S * STAGE);
    float *Psm = reinterpret_cast<float *>(Jsm + 11 * NCT);
    unsigned long long *bars = reinterpret_cast<unsigned long long *>(Psm + 14 * NCT);
    __shared__ float sD[2][Q][Q];
    __shared__ float sdg[2][Q], seps[2][Q], slam[2][Q], sdlam[2];
    __shared__ int s_abort;
    const int tid = threadIdx.x;
    RunGeom g;
    g.init(a.mesh, EB, blockIdx.x);
    const int nel = g.nel, e0 = g.e0;
    const int xn0 = g.xn0, xn1 = g.xn1, yn0 = g.yn0, yn1 = g.yn1, zn0 = g.zn0, zn1 = g.zn1;
    const int vb = blockIdx.y;
    const int k0 = vb * a.Kblk, k1 = min(a.Nu, k0 + a.Kblk);
    const size_t slab = (size_t)a.P;
    if (tid == 0) {
        ring_init(bars, S, NCT / 32);
        s_abort = 0;
    }
    load_ops_f32<Q>(a.fr, tid, sD, sdg, seps, slam, sdlam);
    __syncthreads();

    if (tid >= NCT) {
        if (tid == NCT) ring_producer<Q, C, EB>(a, g, sbuf, bars, S, k0, k1, &s_abort);
        return;
    }

    // ---- consumers ----
    const int lane = tid & 31;
    const int l = tid / NS, s = tid - l * NS;
    const bool active = l < nel;
    const int p = (e0 + l) * NS + s;
    const int id[3] = {s % Q, (s / Q) % Q, s / (Q * Q)};
    const int stride[3] = {1, Q, Q * Q};
    int base[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) base[d] = s - id[d] * stride[d];
    // Dirichlet faces of this element: bit 2d + side
    const int bcm = (l == 0 && xn0 < 0 ? 1 : 0) | (l == nel - 1 && xn1 < 0 ? 2 : 0) | (yn0 < 0 ? 4 : 0) |
                    (yn1 < 0 ? 8 : 0) | (zn0 < 0 ? 16 : 0) | (zn1 < 0 ? 32 : 0);
    // offsets (floats, within a component's stage region) of the own line and
    // of the upwind neighbour line; along x the neighbour sits one slot left
    // (side 0) or right (side 1) of the own element
    const int own_off = (l + 1) * NS;
    const int nby_off = (SLOTS + l) * NS + base[1], nbz_off = (SLOTS + EB + l) * NS + base[2];
    const int fn_off = (SLOTS + 2 * EB + l) * NS + s;
    Eq32 e32;
    float itau = 0.f, gfac = 0.f;
    float gm[5] = {0.f, 0.f, 0.f, 0.f, 0.f}, U0f[3] = {0.f, 0.f, 0.f};
    {
        const double qz[10] = {0.0, 0.0, 0.0, 0.0, 1.0, 1.0, 1.0, 0.0, 0.0, 0.0};
        const double *q = active ? a.eq + (size_t)p * BGK_NEQ : qz;
        e32.load(q);
        if (active) {
            itau = (float)q[10]; gfac = (float)q[11];
#pragma unroll
            for (int i = 0; i < 5; ++i) gm[i] = (float)q[12 + i];
            U0f[0] = (float)q[17]; U0f[1] = (float)q[18]; U0f[2] = (float)q[19];
        }
    }
    const VelGrid &vg = a.vg;
    const int vn1 = vg.n[0], vn2 = vg.n[1], vn3 = vg.n[2];
    const int jc[3] = {(vn1 - 1) / 2, (vn2 - 1) / 2, (vn3 - 1) / 2};
    const double uc[3] = {vg.lo[0] + jc[0] * vg.h[0], vg.lo[1] + jc[1] * vg.h[1], vg.lo[2] + jc[2] * vg.h[2]};
    const float toh[3] = {a.toh32[0], a.toh32[1], a.toh32[2]};
    const float fa = a.a32, fab = a.ab32, fc = a.c32;
    IndexMomentsS acc;
    acc.init(Psm, Jsm, NCT, tid);
    int slot = 0;
    uint32_t par = 0;
    bool ok = true;
    for (int kl = k0; kl < k1; kl += vn1) {
        const int line = kl / vn1;
        const int j2 = line % vn2, j3 = line / vn2;
        if (j3 != acc.j3cur) {
            if (acc.j3cur >= 0) acc.flush_plane(trap3(acc.j3cur, vg), (float)(acc.j3cur - jc[2]));
            acc.j3cur = j3;
        }
        const float4 vl = __ldg(a.vtab32 + kl);
        const float u2 = vl.y, u3 = vl.z;
        float lin, cst;
        e32.line(u2, u3, lin, cst);
        const float t2 = u2 - U0f[1], t3 = u3 - U0f[2];
        const float corr_line = fmaf(gm[2], t2, fmaf(gm[3], t3, fmaf(0.5f * gm[4], fmaf(t2, t2, t3 * t3), gm[0])));
        float jt1 = (float)(-jc[0]);
        for (int j1 = 0; j1 < vn1; ++j1, jt1 += 1.f) {
            const int k = kl + j1;
            ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(bars + slot), par, a.wait_ns));
            if (!ok) break;
            if (active) {
                const float *st = sbuf + (size_t)slot * STAGE;
                const float u1 = __ldg(a.vtab32 + k).x;
                const float u[3] = {u1, u2, u3};
                const float g32 = e32.g(u1, lin, cst);
                const float t1 = u1 - U0f[0];
                const float corr = fmaf(t1, fmaf(0.5f * gm[4], t1, gm[1]), corr_line);
                const float gc = __fmul_rn(g32, corr);
                float outv[C];
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    const float *sc = st + c * PER_C;
                    const float fi = sc[own_off + s];
                    float div = 0.f;
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        const int side = u[d] > 0.f ? 0 : 1;
                        const float *own = sc + own_off + base[d];
                        float t = 0.f;
#pragma unroll
                        // own-line sum in the canonical order j = i+1, ..., i+Q-1 (mod Q);
                        // the j = i term is zero
#pragma unroll
                        for (int m = 1; m < Q; ++m) {
                            const int j = (id[d] + m) % Q;
                            t = fmaf(sD[side][id[d]][j], own[j * stride[d]] - fi, t);
                        }
                        float dn;
                        if (!((bcm >> (2 * d + side)) & 1)) {
                            const float *nb = sc + (d == 0 ? own_off + base[0] + (side ? NS : -NS)
                                                           : (d == 1 ? nby_off : nbz_off));
                            dn = sdlam[side] * fi;
#pragma unroll
                            for (int j = 0; j < Q; ++j) dn = fmaf(slam[side][j], nb[j * stride[d]] - fi, dn);
                        } else {
                            dn = (float)__ldg(a.bcval + ((size_t)(2 * d + side) * C + c) * a.Nu + k) - fi;
                        }
                        t = fmaf(sdg[side][id[d]], dn, fmaf(seps[side][id[d]], fi, t));
                        div = fmaf(toh[d] * u[d], t, div);
                    }
                    const float eqv = (c == 0) ? g32 : __fmul_rn(gfac, g32);
                    const float eqc = (c == 0) ? gc : __fmul_rn(gfac, gc);
                    const float R = fmaf(eqv - fi, itau, fmaf(eqc, itau, -div));
                    const float out = rk_update(fi, fa != 0.f ? sc[fn_off] : 0.f, R, fa, fab, fc, fa != 0.f);
                    a.f_out[((size_t)c * a.Nu + k) * slab + p] = out;
                    outv[c] = out;
                }
                acc.add(trap(j1, vn1), jt1, outv[0], C == 2 ? outv[C - 1] : 0.f);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(bars + S + slot));
            if (++slot == S) { slot = 0; par ^= 1u; }
        }
        if (!ok) break;
        acc.end_line(trap(j2, vn2), (float)(j2 - jc[1]));
    }
    if (!ok) {
        *(volatile int *)&s_abort = 1;
        if (lane == 0) atomicOr(a.status, BGK_DEV_TIMEOUT);
        return;
    }
    if (acc.j3cur >= 0) acc.flush_plane(trap3(acc.j3cur, vg), (float)(acc.j3cur - jc[2]));
    if (a.part && active) {
        double J[11], m[BGK_NMOM];
        acc.get(J);
        index_to_raw(J, vg, uc, m);
#pragma unroll
        for (int j = 0; j < BGK_NMOM; ++j) a.part[((size_t)vb * BGK_NMOM + j) * a.P + p] = m[j];
    }
}

// Raw moments of an FP32 state with the stage epilogue's error-free
// accumulation (IndexMoments, velocities in the same order), for the stepping
// path when the state was set from outside: memory-bound, with no FP64 work
// per DOF, and equal to what a stage's epilogue yields for the same values.
__global__ void __launch_bounds__(256) k_moments_f32_exact(const float *f, double *part, VelGrid vg, int Nu, int P,
                                                            int Kblk, int C) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const int vb = blockIdx.y;
    const int k0 = vb * Kblk, k1 = min(Nu, k0 + Kblk);
    const int vn1 = vg.n[0], vn2 = vg.n[1], vn3 = vg.n[2];
    const int jc[3] = {(vn1 - 1) / 2, (vn2 - 1) / 2, (vn3 - 1) / 2};
    IndexMoments acc;
    acc.init();
    for (int kl = k0; kl < k1; kl += vn1) {
        const int line = kl / vn1;
        const int j2 = line % vn2, j3 = line / vn2;
        if (j3 != acc.j3cur) {
            if (acc.j3cur >= 0) acc.flush_plane(trap3(acc.j3cur, vg), (float)(acc.j3cur - jc[2]));
            acc.j3cur = j3;
        }
        float jt1 = (float)(-jc[0]);
#pragma unroll 8
        for (int j1 = 0; j1 < vn1; ++j1, jt1 += 1.f) {
            const size_t k = (size_t)(kl + j1);
            const float F = __ldcs(f + k * P + p);
            const float G = C == 2 ? __ldcs(f + ((size_t)Nu + k) * P + p) : 0.f;
            acc.add(trap(j1, vn1), jt1, F, G);
        }
        acc.end_line(trap(j2, vn2), (float)(j2 - jc[1]));
    }
    if (acc.j3cur >= 0) acc.flush_plane(trap3(acc.j3cur, vg), (float)(acc.j3cur - jc[2]));
    const double uc[3] = {vg.lo[0] + jc[0] * vg.h[0], vg.lo[1] + jc[1] * vg.h[1], vg.lo[2] + jc[2] * vg.h[2]};
    double m[BGK_NMOM];
    index_to_raw(acc.J, vg, uc, m);
#pragma unroll
    for (int j = 0; j < BGK_NMOM; ++j) part[((size_t)vb * BGK_NMOM + j) * P + p] = m[j];
}

// Raw moments of an FP32 state with FP64 accumulation (initialisation and
// test entry points; the stepping loop takes its moments from the stage).
__global__ void __launch_bounds__(256) k_moments_f32(const float *f, double *part, const double *vtab,
                                                     int Nu, int P, int Kblk, int C) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const int vb = blockIdx.y;
    const int k0 = vb * Kblk, k1 = min(Nu, k0 + Kblk);
    double m[BGK_NMOM];
#pragma unroll
    for (int j = 0; j < BGK_NMOM; ++j) m[j] = 0.0;
    for (int k = k0; k < k1; ++k) {
        const double *v = vtab + (size_t)k * BGK_VTAB;
        const double u1 = __ldg(v + 0), u2 = __ldg(v + 1), u3 = __ldg(v + 2), w = __ldg(v + 3);
        const double wF = w * (double)__ldg(f + (size_t)k * P + p);
        m[0] += wF;
        m[1] = fma(wF, u1, m[1]);
        m[2] = fma(wF, u2, m[2]);
        m[3] = fma(wF, u3, m[3]);
        m[4] = fma(wF * u1, u1, m[4]);
        m[5] = fma(wF * u2, u2, m[5]);
        m[6] = fma(wF * u3, u3, m[6]);
        m[7] = fma(wF * u1, u2, m[7]);
        m[8] = fma(wF * u1, u3, m[8]);
        m[9] = fma(wF * u2, u3, m[9]);
        if (C == 2) m[10] = fma(w, (double)__ldg(f + ((size_t)Nu + k) * P + p), m[10]);
    }
#pragma unroll
    for (int j = 0; j < BGK_NMOM; ++j) part[((size_t)vb * BGK_NMOM + j) * P + p] = m[j];
}

__global__ void k_maxwellian_f32(float *f, const double *qin, const double *vtab, int Nu, int P,
                                 int C, double delta) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)Nu * P) return;
    const int k = (int)(i / P), p = (int)(i - (size_t)k * P);
    const double *q = qin + (size_t)p * 5;
    const double rho = q[0], th = q[4];
    const double *vt = vtab + (size_t)k * BGK_VTAB;
    const double c1 = vt[0] - q[1], c2 = vt[1] - q[2], c3 = vt[2] - q[3];
    const double twopi_th = 6.283185307179586476925286766559 * th;
    const double F = rho / (twopi_th * sqrt(twopi_th)) * exp(-(c1 * c1 + c2 * c2 + c3 * c3) / (2.0 * th));
    f[(size_t)k * P + p] = (float)F;
    if (C == 2) f[((size_t)Nu + k) * P + p] = (float)(0.5 * delta * th * F);
}

}  // namespace

cudaError_t launch_moments_f32_exact(const float *f, double *part, const VelGrid &vg, int Nu, int P, int Kblk,
                                     int C, int n_vblk, cudaStream_t s) {
    dim3 grid((P + 255) / 256, n_vblk);
    k_moments_f32_exact<<<grid, 256, 0, s>>>(f, part, vg, Nu, P, Kblk, C);
    return cudaGetLastError();
}

cudaError_t launch_moments_f32(const float *f, double *part, const double *vtab, int Nu, int P,
                               int Kblk, int C, int n_vblk, cudaStream_t s) {
    dim3 grid((P + 255) / 256, n_vblk);
    k_moments_f32<<<grid, 256, 0, s>>>(f, part, vtab, Nu, P, Kblk, C);
    return cudaGetLastError();
}

template <int Q>
static cudaError_t stage32_q(const StageArgs<float> &a, int C, int n_vblk, cudaStream_t s) {
    constexpr int NS = Q * Q * Q, EB = 256 / NS;
    dim3 grid((a.mesh.Ne + EB - 1) / EB, n_vblk);
    if (a.geo) {
        // the curvilinear instantiations' moment accumulators (dynamic shared memory)
        const size_t dyn = (size_t)EB * NS * (11 * sizeof(double) + 14 * sizeof(float));
        static SmemLimit lim;
        size_t *attr = lim.slot();
        if (!attr) return cudaErrorInvalidDevice;
        if (dyn > *attr) {
            cudaError_t e = cudaFuncSetAttribute(k_stage_f32<Q, 1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(k_stage_f32<Q, 2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
            if (e != cudaSuccess) return e;
            *attr = dyn;
        }
        if (C == 1) k_stage_f32<Q, 1, true><<<grid, EB * NS, dyn, s>>>(a);
        else k_stage_f32<Q, 2, true><<<grid, EB * NS, dyn, s>>>(a);
    } else {
        if (C == 1) k_stage_f32<Q, 1, false><<<grid, EB * NS, 0, s>>>(a);
        else k_stage_f32<Q, 2, false><<<grid, EB * NS, 0, s>>>(a);
    }
    return cudaGetLastError();
}

template <int Q, int C>
static size_t tma_smem(int depth) {
    using G = TmaGeom<Q, C>;
    return (size_t)depth * G::STAGE * sizeof(float) + (11 * sizeof(double) + 14 * sizeof(float)) * G::NCT +
           2 * (size_t)depth * sizeof(unsigned long long);
}

template <int Q, int C>
static cudaError_t stage32_tma(const StageArgs<float> &a, int n_vblk, int depth, cudaStream_t s) {
    using G = TmaGeom<Q, C>;
    const size_t smem = tma_smem<Q, C>(depth);
    static SmemLimit lim;                 // dynamic shared memory limit set so far, per device
    size_t *attr = lim.slot();
    if (!attr) return cudaErrorInvalidDevice;
    if (smem > *attr) {
        cudaError_t e = cudaFuncSetAttribute(k_stage_f32_tma<Q, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        *attr = smem;
    }
    const int cpr = (a.mesh.n[0] + G::EB - 1) / G::EB;
    dim3 grid(cpr * a.mesh.n[1] * a.mesh.n[2], n_vblk);
    k_stage_f32_tma<Q, C><<<grid, G::NTHR, smem, s>>>(a, depth);
    return cudaGetLastError();
}

static bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

static bool any_specular(const MeshInfo &m) {
    for (int f = 0; f < 6; ++f)
        if (m.specular[f]) return true;
    return false;
}

bool stage_f32_tma_supported(const StageArgs<float> &a, int C, int depth) {
    if (a.fr.q != 2 && a.fr.q != 4) return false;          // element slabs of whole 16-byte units
    if (any_specular(a.mesh)) return false;                 // reflected traces are not staged
    if (a.geo) return false;                                // curvilinear: the plain kernel only
    if (depth < 2 || depth > BGK_MAX_DEPTH) return false;
    if (!aligned16(a.f_s) || (a.a32 != 0.f && !aligned16(a.f_n))) return false;
    const size_t smem = a.fr.q == 2 ? (C == 1 ? tma_smem<2, 1>(depth) : tma_smem<2, 2>(depth))
                                    : (C == 1 ? tma_smem<4, 1>(depth) : tma_smem<4, 2>(depth));
    return smem <= 200 * 1024;
}

bool stage_f32_variant_supported(const StageArgs<float> &a, int C, int variant, int depth) {
    switch (variant) {
        case BGK_STAGE_AUTO:
        case BGK_STAGE_PLAIN: return a.fr.q >= 2 && a.fr.q <= BGK_MAXQ;
        case BGK_STAGE_ASYNC: return stage_f32_tma_supported(a, C, depth);
        case BGK_STAGE_LINE:
        case BGK_STAGE_LINE_WIDE:
        case BGK_STAGE_HALF:
        case BGK_STAGE_HALF_WIDE: return stage_f32_line_supported(a, C, variant - BGK_STAGE_LINE, depth);
        default: return false;
    }
}

cudaError_t launch_stage_f32(const StageArgs<float> &a, int C, int n_vblk, int variant, int depth, cudaStream_t s) {
    if (variant >= BGK_STAGE_LINE && variant <= BGK_STAGE_HALF_WIDE)
        return launch_stage_f32_line(a, C, n_vblk, variant - BGK_STAGE_LINE, depth, s);
    if ((variant == BGK_STAGE_AUTO || variant == BGK_STAGE_ASYNC) && stage_f32_tma_supported(a, C, depth)) {
        if (a.fr.q == 2) return C == 1 ? stage32_tma<2, 1>(a, n_vblk, depth, s) : stage32_tma<2, 2>(a, n_vblk, depth, s);
        return C == 1 ? stage32_tma<4, 1>(a, n_vblk, depth, s) : stage32_tma<4, 2>(a, n_vblk, depth, s);
    }
    if (variant == BGK_STAGE_ASYNC) return cudaErrorInvalidValue;
    switch (a.fr.q) {
        case 2: return stage32_q<2>(a, C, n_vblk, s);
        case 3: return stage32_q<3>(a, C, n_vblk, s);
        case 4: return stage32_q<4>(a, C, n_vblk, s);
        case 5: return stage32_q<5>(a, C, n_vblk, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_maxwellian_f32(float *f, const double *q, const double *vtab, int Nu, int P, int C,
                                  double delta, cudaStream_t s) {
    const size_t n = (size_t)Nu * P;
    k_maxwellian_f32<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(f, q, vtab, Nu, P, C, delta);
    return cudaGetLastError();
}
