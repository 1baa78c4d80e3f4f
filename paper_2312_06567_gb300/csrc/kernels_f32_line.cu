// Mixed-form fused stage, one thread per first-axis node line.
//
// Same FR advection (deviation form with telescoping trace weights), FP32
// equilibrium with its moment correction, Runge--Kutta update and
// error-free moment epilogue as k_stage_f32, evaluated term for term in the
// same order for every point, so the results are bit-identical; what
// changes is the work mapping.  Each consumer thread owns the Q nodes
// (i, j, k), i = 0..Q-1, of one line along the first element axis, i.e. Q
// points:
//   - its own line and every line it needs (the other lines of its element
//     in the second and third directions, the upwind neighbours' lines)
//     arrive as one vector load each from the shared-memory stage;
//   - own-line sums run in the canonical order j = i+1, ..., i+Q-1 (mod Q)
//     of all FP32 stage kernels, Q-1 terms with no masked iteration;
//   - the coefficients of the second- and third-direction sums are the same
//     for the thread's Q points (one load serves Q products), and the
//     first-direction deviations f_j - f_i are formed once per pair (the
//     negated difference is exact);
//   - the barrier wait, the velocity bookkeeping and the loop control are
//     paid once per Q points.
// The operands arrive through the copy ring of the node-per-thread pipelined
// kernel, fed here without a producer warp: the consumer warp that releases
// a slot last (a shared-memory count, ordered by block-scope fences before
// and after it) refills the slot for the velocity S ahead (ring_issue_u), as
// a whole warp with one elected lane issuing the copies, so every register
// of the block works on the stage.  The velocity grid's axis values sit in
// shared memory (a tensor grid), so neither the consumers nor the refill
// wait on a load of the velocity table.  Every thread runs the velocity body
// (an idle one past the end of a short run only skips its stores), so the
// body does not diverge.  The FP32 equilibrium
// parameters come from the record the Q' solve writes beside its FP64 one
// (BGK_NEQ32), the plane-level moment pairs live in shared memory and the
// FP64 index moments accumulate in the moment-partials buffer, which this
// block owns for its points and velocity block, converted to raw moments at
// the end.  Dzanic & Martinelli, arXiv 2312.06567, section "Methodology".
#include <type_traits>

#include "stage_f32_common.cuh"

namespace {

template <int Q, int C, int EB, int NPT>
struct LineGeom {
    static constexpr int NH = Q / NPT;                  // threads per node line
    // consumer threads: the run's lines, rounded up to whole warps (at Q = 3
    // the last warp's extra threads map past the run and stay idle)
    static constexpr int NCT = (EB * Q * Q * NH + 31) / 32 * 32;
    static constexpr int NTHR = NCT;                    // no producer warp: the ring feeds itself
    static constexpr int NW = NCT / 32;
    static constexpr int NQ = C == 2 ? 7 : 6;           // plane quantities per point
    // resident blocks asked of the register allocator: a budget of about 96
    // registers per thread (128 with a whole line per thread)
    // (Q = 3: 16-element runs, 144 threads in 160: three blocks per SM of up
    // to 136 registers, which the packed F/G body fits without spills -- 28.3
    // ms of stage per step on the normal shock against 35.7 with two blocks;
    // the per-component body needed 167 registers)
    static constexpr int MINB = Q == 3 ? 3
                                       : (65536 / (NTHR * (NPT == Q ? 128 : 96)) > 0 ? 65536 / (NTHR * (NPT == Q ? 128 : 96))
                                                                                      : 1);
    static_assert(Q % NPT == 0, "a thread takes a whole fraction of a line");
};

template <int N>
__device__ __forceinline__ void ld_vec(const float *p, float (&v)[N]);
template <>
__device__ __forceinline__ void ld_vec<4>(const float *p, float (&v)[4]) {
    const float4 t = *reinterpret_cast<const float4 *>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
template <>
__device__ __forceinline__ void ld_vec<2>(const float *p, float (&v)[2]) {
    const float2 t = *reinterpret_cast<const float2 *>(p);
    v[0] = t.x; v[1] = t.y;
}
template <>
__device__ __forceinline__ void ld_vec<3>(const float *p, float (&v)[3]) {
    v[0] = p[0]; v[1] = p[1]; v[2] = p[2];               // 4-byte aligned only
}
template <>
__device__ __forceinline__ void ld_vec<1>(const float *p, float (&v)[1]) {
    v[0] = *p;
}
template <int N>
__device__ __forceinline__ void st_vec(float *p, const float (&v)[N]);
template <>
__device__ __forceinline__ void st_vec<4>(float *p, const float (&v)[4]) {
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
template <>
__device__ __forceinline__ void st_vec<2>(float *p, const float (&v)[2]) {
    *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]);
}
template <>
__device__ __forceinline__ void st_vec<3>(float *p, const float (&v)[3]) {
    p[0] = v[0]; p[1] = v[1]; p[2] = v[2];
}
template <>
__device__ __forceinline__ void st_vec<1>(float *p, const float (&v)[1]) {
    *p = v[0];
}

// Element-wise FR updates over a thread's NPT points.  With NPT even they run
// on pairs of points with the packed FP32 instructions (two IEEE operations
// per issue, each rounded exactly as its scalar form), so the results are
// bit-identical to the scalar sequence of the other FP32 stage kernels
// (x - y as sub2, the pair helpers of stage_f32_common.cuh).

// t[i] = fmaf(D, G[i] - F[i], t[i]), D common to the points
template <int N>
__device__ __forceinline__ void acc_dev(float (&t)[N], float D, const float (&G)[N], const float (&F)[N]) {
    if constexpr (N % 2 == 0) {
        const float2 d2 = make_float2(D, D);
#pragma unroll
        for (int i = 0; i < N; i += 2) {
            const float2 dv = sub2(make_float2(G[i], G[i + 1]), make_float2(F[i], F[i + 1]));
            const float2 r = __ffma2_rn(d2, dv, make_float2(t[i], t[i + 1]));
            t[i] = r.x; t[i + 1] = r.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < N; ++i) t[i] = fmaf(D, __fsub_rn(G[i], F[i]), t[i]);
    }
}
// y[i] = c * F[i]
template <int N>
__device__ __forceinline__ void scale_vec(float (&y)[N], float c, const float (&F)[N]) {
    if constexpr (N % 2 == 0) {
        const float2 c2 = make_float2(c, c);
#pragma unroll
        for (int i = 0; i < N; i += 2) {
            const float2 r = __fmul2_rn(c2, make_float2(F[i], F[i + 1]));
            y[i] = r.x; y[i + 1] = r.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < N; ++i) y[i] = __fmul_rn(c, F[i]);
    }
}
// t[i] = fmaf(a[i], dn[i], fmaf(b[i], F[i], t[i])); div[i] = fmaf(cu, t[i], div[i])
template <int N>
__device__ __forceinline__ void lift_vec(float (&t)[N], const float *a, const float *b, const float (&dn)[N],
                                         const float (&F)[N], float cu, float (&div)[N], bool first) {
    if constexpr (N % 2 == 0) {
        const float2 cu2 = make_float2(cu, cu), z2 = make_float2(0.f, 0.f);
#pragma unroll
        for (int i = 0; i < N; i += 2) {
            const float2 a2 = make_float2(a[i], a[i + 1]), b2 = make_float2(b[i], b[i + 1]);
            float2 tt = __ffma2_rn(b2, make_float2(F[i], F[i + 1]), make_float2(t[i], t[i + 1]));
            tt = __ffma2_rn(a2, make_float2(dn[i], dn[i + 1]), tt);
            const float2 dv = __ffma2_rn(cu2, tt, first ? z2 : make_float2(div[i], div[i + 1]));
            t[i] = tt.x; t[i + 1] = tt.y;
            div[i] = dv.x; div[i + 1] = dv.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < N; ++i) {
            t[i] = fmaf(a[i], dn[i], fmaf(b[i], F[i], t[i]));
            div[i] = fmaf(cu, t[i], first ? 0.f : div[i]);
        }
    }
}

// shared-memory fetch-and-add by one thread, as one PTX atomic (no
// warp-aggregation sequence around it)
__device__ __forceinline__ unsigned int atom_add_shared(unsigned int *p, unsigned int v) {
    unsigned int old;
    asm volatile("atom.shared.add.u32 %0, [%1], %2;" : "=r"(old) : "r"(smem_u32(p)), "r"(v) : "memory");
    return old;
}


// Line sums of one point (the first level of IndexMoments): F, F jt, F jt^2
// and, with two components, G; error-free pairs.
template <int C>
struct LineAcc {
    float L[C == 2 ? 4 : 3], Lc[C == 2 ? 4 : 3];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int q = 0; q < (C == 2 ? 4 : 3); ++q) L[q] = Lc[q] = 0.f;
    }
    __device__ __forceinline__ void add(float cj1, float jt1, float F, float G) {
        const float cF = __fmul_rn(cj1, F);
        sum2(L[0], Lc[0], cF);
        const float p1 = __fmul_rn(cF, jt1);
        sum2(L[1], Lc[1], p1);
        Lc[1] = __fadd_rn(Lc[1], fmaf(cF, jt1, -p1));
        const float jj = __fmul_rn(jt1, jt1);
        const float p2 = __fmul_rn(cF, jj);
        sum2(L[2], Lc[2], p2);
        Lc[2] = __fadd_rn(Lc[2], fmaf(cF, jj, -p2));
        if (C == 2) sum2(L[C == 2 ? 3 : 0], Lc[C == 2 ? 3 : 0], __fmul_rn(cj1, G));
    }
    __device__ __forceinline__ float Ls(int q) const { return L[q]; }
    __device__ __forceinline__ float Lcs(int q) const { return Lc[q]; }
};

// LineAcc<2>::add of one point on packed FP32, lane for lane the same
// operations: the (sum, error) pairs (L0, L3) of c F and c G side by side,
// and (L1, L2) of c F jt and c F jt^2 (their product errors taken negated,
// fma(x, -y, p) = -(x y - p) exactly, and subtracted)
struct LineAccFG {
    float2 A, Ae, B, Be;
    __device__ __forceinline__ void zero() { A = Ae = B = Be = make_float2(0.f, 0.f); }
    __device__ __forceinline__ void add(float cj1, float jt1, float F, float G) {
        const float2 cFG = __fmul2_rn(dup2(cj1), make_float2(F, G));
        sum2x2(A, Ae, cFG);
        const float jj = __fmul_rn(jt1, jt1), njt1 = -jt1, njj = __fmul_rn(njt1, jt1);      // exact
        const float2 cF = dup2(cFG.x);
        const float2 p = __fmul2_rn(cF, make_float2(jt1, jj));
        sum2x2(B, Be, p);
        Be = sub2(Be, __ffma2_rn(cF, make_float2(njt1, njj), p));
    }
    __device__ __forceinline__ float Ls(int q) const { return q == 0 ? A.x : q == 1 ? B.x : q == 2 ? B.y : A.y; }
    __device__ __forceinline__ float Lcs(int q) const { return q == 0 ? Ae.x : q == 1 ? Be.x : q == 2 ? Be.y : Ae.y; }
};

// LineAcc::add of two points at once, operation for operation; the product
// errors are taken negated, -(x y - p) = fma(x, -y, p) exactly, and
// subtracted, so no value is negated per point
template <int C>
__device__ __forceinline__ void add_pair(LineAcc<C> &A, LineAcc<C> &B, float cj1, float jt1, float2 F, float2 G) {
    const float2 cF = __fmul2_rn(dup2(cj1), F);
    float2 s = make_float2(A.L[0], B.L[0]), e = make_float2(A.Lc[0], B.Lc[0]);
    sum2x2(s, e, cF);
    A.L[0] = s.x; B.L[0] = s.y; A.Lc[0] = e.x; B.Lc[0] = e.y;
    const float njt1 = -jt1;
    const float2 p1 = __fmul2_rn(cF, dup2(jt1));
    s = make_float2(A.L[1], B.L[1]); e = make_float2(A.Lc[1], B.Lc[1]);
    sum2x2(s, e, p1);
    e = sub2(e, __ffma2_rn(cF, dup2(njt1), p1));
    A.L[1] = s.x; B.L[1] = s.y; A.Lc[1] = e.x; B.Lc[1] = e.y;
    const float jj = __fmul_rn(jt1, jt1), njj = __fmul_rn(njt1, jt1);       // exact
    const float2 p2 = __fmul2_rn(cF, dup2(jj));
    s = make_float2(A.L[2], B.L[2]); e = make_float2(A.Lc[2], B.Lc[2]);
    sum2x2(s, e, p2);
    e = sub2(e, __ffma2_rn(cF, dup2(njj), p2));
    A.L[2] = s.x; B.L[2] = s.y; A.Lc[2] = e.x; B.Lc[2] = e.y;
    if constexpr (C == 2) {
        s = make_float2(A.L[3], B.L[3]); e = make_float2(A.Lc[3], B.Lc[3]);
        sum2x2(s, e, __fmul2_rn(dup2(cj1), G));
        A.L[3] = s.x; B.L[3] = s.y; A.Lc[3] = e.x; B.Lc[3] = e.y;
    }
}

// Plane pairs of one point in shared memory: P[q] at P[q * n], errors at
// P[(NQ + q) * n]; the same operations as IndexMoments::plane_add/end_line.
template <int NQ>
__device__ __forceinline__ void plane_add_s(float *P, int n, int q, float c, float sum, float err) {
    float ps = P[q * n], pc = P[(NQ + q) * n];
    const float pr = __fmul_rn(c, sum);
    sum2(ps, pc, pr);
    pc = __fadd_rn(pc, fmaf(c, sum, -pr));
    pc = fmaf(c, err, pc);
    P[q * n] = ps;
    P[(NQ + q) * n] = pc;
}

// BC = false: the mesh is periodic in every direction, so no face is a
// Dirichlet face and the per-direction tests drop out.
template <int Q, int C, int EB, int NPT, bool BC>
__global__ void __launch_bounds__(LineGeom<Q, C, EB, NPT>::NTHR, LineGeom<Q, C, EB, NPT>::MINB) k_stage_f32_line(StageArgs<float> a, int S) {
    using SG = StageGeom<Q, C, EB>;
    using LG = LineGeom<Q, C, EB, NPT>;
    constexpr int NS = SG::NS, SLOTS = SG::SLOTS, PER_C = SG::PER_C, STAGE = SG::STAGE;
    constexpr int NCT = LG::NCT, NQ = LG::NQ, NH = LG::NH, NTT = Q * Q * NH;
    extern __shared__ __align__(128) float sbuf[];
    // [S][STAGE] copy ring | [NPT][2 NQ][NCT] plane pairs | 2S mbarriers | [S] release counts | [S] fills
    float *Psm = sbuf + (size_t)S * STAGE;
    unsigned long long *bars = reinterpret_cast<unsigned long long *>(Psm + NPT * 2 * NQ * NCT);
    unsigned int *rel = reinterpret_cast<unsigned int *>(bars + 2 * S);
    unsigned int *fills = rel + S;
    __shared__ __align__(16) float sD[2][Q][Q];
    __shared__ __align__(16) float sdg[2][Q];
    __shared__ __align__(16) float seps[2][Q];
    __shared__ __align__(16) float slam[2][Q];
    __shared__ float sdlam[2];
    // the same entries arranged for whole-row vector loads: sDr[side][n][m] =
    // sD[side][n][(n + m) mod Q] (row n in the canonical order from n), and
    // sCf[side][n] = (dlam, dg_n, eps_n, 0)
    __shared__ __align__(16) float sDr[2][Q][Q];
    __shared__ float4 sCf[2][Q];
    // the velocity grid's axis values (a tensor grid: u_d of a velocity
    // depends on its index on axis d only) with the first axis's trapezoid
    // factors, so neither the consumers nor the ring refill read the velocity
    // table from global memory
    __shared__ float2 su1c[BGK_MAXV];                    // (u1, trapezoid factor) of the first-axis nodes
    __shared__ float su2[BGK_MAXV], su3[BGK_MAXV];
    __shared__ unsigned int s_exited;
    __shared__ unsigned long long s_wait_ns;
    __shared__ int s_nfill;                              // velocities the ring delivers
    constexpr int NW = LG::NW;
    const int tid = threadIdx.x;
    RunGeom g;
    g.init(a.mesh, EB, blockIdx.x);
    const int vb = blockIdx.y;
    const int k0 = vb * a.Kblk, k1 = min(a.Nu, k0 + a.Kblk);
    const int nk = k1 - k0;
    const size_t slab = (size_t)a.P;
    const VelGrid &vg = a.vg;
    const int vn1 = vg.n[0], vn2 = vg.n[1], vn3 = vg.n[2];
    if (tid == 0) {
        ring_init(bars, S, NW);
        s_exited = 0;
        s_wait_ns = a.wait_ns;
        for (int i = 0; i < S; ++i) {
            rel[i] = 0;
            fills[i] = 0;
        }
        // the first S velocities
        const int nring = a.ring_limit > 0 ? min(nk, a.ring_limit) : nk;
        s_nfill = nring;
        for (int i = 0; i < S && i < nring; ++i) {
            ring_issue<Q, C, EB>(a, g, sbuf, bars, i, k0 + i);
            fills[i] = 1;
        }
    }
    for (int j = tid; j < vn1; j += blockDim.x) su1c[j] = make_float2(__ldg(a.vtab32 + j).x, trap(j, vn1));
    for (int j = tid; j < vn2; j += blockDim.x) su2[j] = __ldg(a.vtab32 + (size_t)j * vn1).y;
    for (int j = tid; j < vn3; j += blockDim.x) su3[j] = __ldg(a.vtab32 + (size_t)j * vn1 * vn2).z;
    load_ops_f32<Q>(a.fr, tid, sD, sdg, seps, slam, sdlam);
    __syncthreads();
    if (tid < 2 * Q * Q) {
        const int side = tid / (Q * Q), n = (tid / Q) % Q, m = tid % Q;
        sDr[side][n][m] = sD[side][n][(n + m) % Q];
    }
    if (tid < 2 * Q) {
        const int side = tid / Q, n = tid % Q;
        sCf[side][n] = make_float4(sdlam[side], sdg[side][n], seps[side][n], 0.f);
    }
    __syncthreads();

    // ---- consumers: thread = (element l of the run, node line r = jy + Q kz, part h of the line) ----
    const int lane = tid & 31;
    const int l = tid / NTT, rem = tid - l * NTT;
    const int r = rem / NH, h = rem - r * NH;
    const int jy = r % Q, kz = r / Q;
    const int i0 = NPT * h;                              // first node of this thread on its line
    const bool active = l < g.nel;
    const int pb = (g.e0 + l) * NS + Q * r + i0;         // point of local node i: pb + i
    const int bcm = !BC ? 0
                        : (l == 0 && g.xn0 < 0 ? 1 : 0) | (l == g.nel - 1 && g.xn1 < 0 ? 2 : 0) | (g.yn0 < 0 ? 4 : 0) |
                              (g.yn1 < 0 ? 8 : 0) | (g.zn0 < 0 ? 16 : 0) | (g.zn1 < 0 ? 32 : 0);
    const int own_off = (l + SG::PAD) * NS;              // own element within a component's stage region
    const int ln = Q * r;                                // own line within an element
    const bool mom = a.part != nullptr;
    // per-point FP32 parameters used every velocity
    float E0[NPT], V1[NPT], A11[NPT], itau[NPT], gm1[NPT], gm4h[NPT], U0x[NPT], gfac[NPT];
#pragma unroll
    for (int i = 0; i < NPT; ++i) {
        E0[i] = V1[i] = A11[i] = itau[i] = gm1[i] = gm4h[i] = U0x[i] = gfac[i] = 0.f;
        if (active) {
            const float4 *rec = reinterpret_cast<const float4 *>(a.eq32 + (size_t)(pb + i) * BGK_NEQ32);
            const float4 r0 = __ldg(rec), r1 = __ldg(rec + 1);
            E0[i] = r0.x; V1[i] = r0.y; A11[i] = r0.z; itau[i] = r0.w;
            gm1[i] = r1.x; gm4h[i] = r1.y; U0x[i] = r1.z; gfac[i] = r1.w;
        }
    }
    const int jc[3] = {(vn1 - 1) / 2, (vn2 - 1) / 2, (vn3 - 1) / 2};
    const float toh0 = a.toh32[0], toh1 = a.toh32[1], toh2 = a.toh32[2];
    const float fa = a.a32, fab = a.ab32, fc = a.c32;
    float *Pme = Psm + tid;                              // this thread's plane pairs: point i at Pme + i 2NQ NCT
    if (mom) {
#pragma unroll
        for (int i = 0; i < NPT; ++i)
#pragma unroll
            for (int q = 0; q < 2 * NQ; ++q) Pme[(i * 2 * NQ + q) * NCT] = 0.f;
    }
    // FP64 index moments of the finished planes, kept in the partials buffer
    int j3cur = -1;
    bool first_plane = true;
    auto flush_plane = [&](int j3) {
        const double c = trap3(j3, vg), t = (float)(j3 - jc[2]);
#pragma unroll
        for (int i = 0; i < NPT; ++i) {
            float *P = Pme + i * 2 * NQ * NCT;
            double Pd[7];
#pragma unroll
            for (int q = 0; q < 7; ++q) {
                Pd[q] = 0.0;
                if (q < NQ) {
                    Pd[q] = (double)P[q * NCT] + (double)P[(NQ + q) * NCT];
                    P[q * NCT] = 0.f;
                    P[(NQ + q) * NCT] = 0.f;
                }
            }
            double *J = a.part + (size_t)vb * BGK_NMOM * a.P + pb + i;
            double Jo[11];
#pragma unroll
            for (int q = 0; q < 11; ++q) Jo[q] = first_plane ? 0.0 : J[(size_t)q * a.P];
            Jo[0] = fma(c, Pd[0], Jo[0]);
            Jo[1] = fma(c, Pd[1], Jo[1]);
            Jo[2] = fma(c, Pd[2], Jo[2]);
            Jo[3] = fma(c, Pd[3], Jo[3]);
            Jo[4] = fma(c, Pd[4], Jo[4]);
            Jo[5] = fma(c, Pd[5], Jo[5]);
            Jo[6] = fma(c * t, Pd[0], Jo[6]);
            Jo[7] = fma(c * t, Pd[1], Jo[7]);
            Jo[8] = fma(c * t, Pd[3], Jo[8]);
            Jo[9] = fma(c * t * t, Pd[0], Jo[9]);
            Jo[10] = fma(c, Pd[6], Jo[10]);
#pragma unroll
            for (int q = 0; q < 11; ++q) J[(size_t)q * a.P] = Jo[q];
        }
        first_plane = false;
    };

    int slot = 0;
    uint32_t par = 0;
    bool ok = true;
    for (int kl = k0; kl < k1; kl += vn1) {
        const int line = kl / vn1;
        const int j2 = line % vn2, j3 = line / vn2;
        if (mom && active && j3 != j3cur) {
            if (j3cur >= 0) flush_plane(j3cur);
            j3cur = j3;
        }
        const float u2 = su2[j2], u3 = su3[j3];
        const int sy = u2 > 0.f ? 0 : 1, sz = u3 > 0.f ? 0 : 1;
        // per-point line constants of the equilibrium exponent and the correction
        float lin[NPT], cst[NPT], cl[NPT];
#pragma unroll
        for (int i = 0; i < NPT; ++i) {
            lin[i] = cst[i] = cl[i] = 0.f;
            if (active) {
                const float4 *rec = reinterpret_cast<const float4 *>(a.eq32 + (size_t)(pb + i) * BGK_NEQ32);
                const float4 r2 = __ldg(rec + 2), r3 = __ldg(rec + 3), r4 = __ldg(rec + 4), r5 = __ldg(rec + 5);
                Eq32 e;
                e.V2 = r2.x; e.V3 = r2.y; e.A12 = r2.z; e.A13 = r2.w;
                e.A22 = r3.x; e.A23 = r3.y; e.A33 = r3.z;
                e.line(u2, u3, lin[i], cst[i]);
                const float t2 = u2 - r4.z, t3 = u3 - r4.w;
                cl[i] = fmaf(r4.x, t2, fmaf(r4.y, t3, fmaf(0.5f * r5.x, fmaf(t2, t2, t3 * t3), r3.w)));
            }
        }
        // F and G with an odd number of points: each point's sums as pairs
        using Acc = typename std::conditional<C == 2 && NPT % 2 == 1, LineAccFG, LineAcc<C>>::type;
        Acc acc[NPT];
#pragma unroll
        for (int i = 0; i < NPT; ++i) acc[i].zero();
        float jt1 = (float)(-jc[0]);
        for (int j1 = 0; j1 < vn1; ++j1, jt1 += 1.f) {
            const int k = kl + j1;
            ok = __all_sync(0xffffffffu, mbar_wait_s(smem_u32(bars + slot), par, &s_wait_ns));
            if (!ok) break;
            // every thread computes (an idle one, past the end of a short run,
            // on stage slots that hold no element of its own: finite or not,
            // its values are never stored), so the loop body does not diverge;
            // only the stores depend on `active`
            {
                const float *st = sbuf + (size_t)slot * STAGE;
                const float u1 = su1c[j1].x;
                const int sx = u1 > 0.f ? 0 : 1;
                float outv[C][NPT];
                if constexpr (C == 2 && NPT == Q && NPT % 2 == 1) {
                    // F and G of each point as one packed FP32 pair: every
                    // component's operations exactly those of the per-component
                    // body below (x - y as fma(y, -1, x), the same rounding), so
                    // the results are the same bit for bit; the equilibrium is
                    // evaluated once for both
                    const float *s0 = st, *s1 = st + PER_C;
                    auto ld2 = [&](int off, int n, float2 *v) {
                        for (int i = 0; i < n; ++i) v[i] = make_float2(s0[off + i], s1[off + i]);
                    };
                    float2 F2[NPT], div2[NPT];
                    ld2(own_off + ln + i0, NPT, F2);
                    // ---- first direction
                    {
                        float2 F[Q], t[NPT];
                        ld2(own_off + ln, Q, F);
                        float2 dv[Q][Q];
#pragma unroll
                        for (int i = 0; i < Q; ++i)
#pragma unroll
                            for (int j = i + 1; j < Q; ++j) dv[i][j] = sub2(F[j], F[i]);
#pragma unroll
                        for (int i = 0; i < NPT; ++i) {
                            float Dr[Q];
                            ld_vec<Q>(&sD[sx][i][0], Dr);
                            t[i] = dup2(0.f);
#pragma unroll
                            for (int m = 1; m < Q; ++m) {
                                const int j = (i + m) % Q;
                                t[i] = __ffma2_rn(dup2(Dr[j]), j > i ? dv[i][j] : neg2(dv[j][i]), t[i]);
                            }
                        }
                        float2 dn[NPT];
                        if (!BC || !((bcm >> sx) & 1)) {
                            float2 NB[Q];
                            ld2(own_off + (sx ? NS : -NS) + ln, Q, NB);
                            float Lr[Q];
                            ld_vec<Q>(&slam[sx][0], Lr);
#pragma unroll
                            for (int i = 0; i < NPT; ++i) dn[i] = __fmul2_rn(dup2(sdlam[sx]), F2[i]);
#pragma unroll
                            for (int j = 0; j < Q; ++j)
#pragma unroll
                                for (int i = 0; i < NPT; ++i)
                                    dn[i] = __ffma2_rn(dup2(Lr[j]), sub2(NB[j], F2[i]), dn[i]);
                        } else {
                            const float2 bv = make_float2((float)__ldg(a.bcval + ((size_t)(0 + sx) * C + 0) * a.Nu + k),
                                                          (float)__ldg(a.bcval + ((size_t)(0 + sx) * C + 1) * a.Nu + k));
#pragma unroll
                            for (int i = 0; i < NPT; ++i) dn[i] = sub2(bv, F2[i]);
                        }
                        float Gr[NPT], Er[NPT];
                        ld_vec<NPT>(&sdg[sx][i0], Gr);
                        ld_vec<NPT>(&seps[sx][i0], Er);
                        const float2 cu = dup2(toh0 * u1);
#pragma unroll
                        for (int i = 0; i < NPT; ++i) {
                            t[i] = __ffma2_rn(dup2(Gr[i]), dn[i], __ffma2_rn(dup2(Er[i]), F2[i], t[i]));
                            div2[i] = __ffma2_rn(cu, t[i], dup2(0.f));
                        }
                    }
                    // ---- second and third directions
#pragma unroll
                    for (int dd = 1; dd < 3; ++dd) {
                        const int sd = dd == 1 ? sy : sz, nd = dd == 1 ? jy : kz;
                        float2 t[NPT], dn[NPT];
#pragma unroll
                        for (int i = 0; i < NPT; ++i) t[i] = dup2(0.f);
                        float Dr[Q];
                        ld_vec<Q>(&sDr[sd][nd][0], Dr);
                        const float4 cf = sCf[sd][nd];
#pragma unroll
                        for (int m = 1; m < Q; ++m) {
                            const int jq = (nd + m) % Q;
                            float2 Gv[NPT];
                            ld2(own_off + (dd == 1 ? Q * (jq + Q * kz) : Q * (jy + Q * jq)) + i0, NPT, Gv);
#pragma unroll
                            for (int i = 0; i < NPT; ++i) t[i] = __ffma2_rn(dup2(Dr[m]), sub2(Gv[i], F2[i]), t[i]);
                        }
                        if (!BC || !((bcm >> (2 * dd + sd)) & 1)) {
                            float Lr[Q];
                            ld_vec<Q>(&slam[sd][0], Lr);
#pragma unroll
                            for (int i = 0; i < NPT; ++i) dn[i] = __fmul2_rn(dup2(cf.x), F2[i]);
#pragma unroll
                            for (int jq = 0; jq < Q; ++jq) {
                                float2 H[NPT];
                                ld2((dd == 1 ? (SLOTS + l) * NS + Q * (jq + Q * kz) : (SLOTS + EB + l) * NS + Q * (jy + Q * jq)) + i0,
                                    NPT, H);
#pragma unroll
                                for (int i = 0; i < NPT; ++i) dn[i] = __ffma2_rn(dup2(Lr[jq]), sub2(H[i], F2[i]), dn[i]);
                            }
                        } else {
                            const float2 bv = make_float2((float)__ldg(a.bcval + ((size_t)(2 * dd + sd) * C + 0) * a.Nu + k),
                                                          (float)__ldg(a.bcval + ((size_t)(2 * dd + sd) * C + 1) * a.Nu + k));
#pragma unroll
                            for (int i = 0; i < NPT; ++i) dn[i] = sub2(bv, F2[i]);
                        }
                        const float2 cu = dup2(dd == 1 ? toh1 * u2 : toh2 * u3);
#pragma unroll
                        for (int i = 0; i < NPT; ++i) {
                            t[i] = __ffma2_rn(dup2(cf.y), dn[i], __ffma2_rn(dup2(cf.z), F2[i], t[i]));
                            div2[i] = __ffma2_rn(cu, t[i], div2[i]);
                        }
                    }
                    // ---- equilibrium (once for both), source and Runge--Kutta update
                    float2 FN[NPT];
                    if (fa != 0.f) ld2((SLOTS + 2 * EB + l) * NS + ln + i0, NPT, FN);
#pragma unroll
                    for (int i = 0; i < NPT; ++i) {
                        const float c1 = __fsub_rn(u1, V1[i]);
                        const float g32 = __fmul_rn(E0[i], Eq32::ex2(fmaf(c1, fmaf(A11[i], c1, lin[i]), cst[i])));
                        const float t1 = u1 - U0x[i];
                        const float corr = fmaf(t1, fmaf(gm4h[i], t1, gm1[i]), cl[i]);
                        const float gc = __fmul_rn(g32, corr);
                        const float2 eqv = make_float2(g32, __fmul_rn(gfac[i], g32));
                        const float2 eqc = make_float2(gc, __fmul_rn(gfac[i], gc));
                        const float2 it2 = dup2(itau[i]);
                        const float2 R = __ffma2_rn(sub2(eqv, F2[i]), it2, __ffma2_rn(eqc, it2, neg2(div2[i])));
                        const float2 o = rk_update2(F2[i], fa != 0.f ? FN[i] : dup2(0.f), R, fa, fab, fc, fa != 0.f);
                        outv[0][i] = o.x;
                        outv[C - 1][i] = o.y;
                    }
                    if (active) {
                        st_vec<NPT>(a.f_out + (size_t)k * slab + pb, outv[0]);
                        st_vec<NPT>(a.f_out + ((size_t)a.Nu + k) * slab + pb, outv[C - 1]);
                    }
                } else {
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    const float *sc = st + c * PER_C;
                    float Fi[NPT];                       // this thread's nodes
                    ld_vec<NPT>(sc + own_off + ln + i0, Fi);
                    float div[NPT];
                    // ---- first direction: the line itself and the upwind neighbour's line
                    {
                        float F[Q];
                        ld_vec<Q>(sc + own_off + ln, F);
                        float t[NPT];
                        if (NPT == Q) {
                            // deviations formed once per pair: f_i - f_j = -(f_j - f_i) exactly
                            float dv[Q][Q];
#pragma unroll
                            for (int i = 0; i < Q; ++i)
#pragma unroll
                                for (int j = i + 1; j < Q; ++j) dv[i][j] = F[j] - F[i];
#pragma unroll
                            for (int i = 0; i < NPT; ++i) {
                                float Dr[Q];
                                ld_vec<Q>(&sD[sx][i][0], Dr);
                                t[i] = 0.f;
#pragma unroll
                                for (int m = 1; m < Q; ++m) {
                                    const int j = (i + m) % Q;      // the canonical order
                                    t[i] = fmaf(Dr[j], j > i ? dv[i][j] : -dv[j][i], t[i]);
                                }
                            }
                        } else {
#pragma unroll
                            for (int i = 0; i < NPT; ++i) {
                                t[i] = 0.f;
#pragma unroll
                                for (int m = 1; m < Q; ++m) {
                                    // node j = (i0 + i + m) mod Q of the line, picked from F
                                    // without indexing a register array at run time
                                    const int j = (i0 + i + m) % Q;
                                    float Fj = F[0];
#pragma unroll
                                    for (int jj = 1; jj < Q; ++jj) Fj = j == jj ? F[jj] : Fj;
                                    t[i] = fmaf(sD[sx][i0 + i][j], Fj - Fi[i], t[i]);
                                }
                            }
                        }
                        float dn[NPT];
                        if (!BC || !((bcm >> sx) & 1)) {
                            float NB[Q];
                            ld_vec<Q>(sc + own_off + (sx ? NS : -NS) + ln, NB);
                            float Lr[Q];
                            ld_vec<Q>(&slam[sx][0], Lr);
                            scale_vec<NPT>(dn, sdlam[sx], Fi);
#pragma unroll
                            for (int j = 0; j < Q; ++j) {
                                float NBj[NPT];
#pragma unroll
                                for (int i = 0; i < NPT; ++i) NBj[i] = NB[j];
                                acc_dev<NPT>(dn, Lr[j], NBj, Fi);
                            }
                        } else {
                            const float bv = (float)__ldg(a.bcval + ((size_t)(0 + sx) * C + c) * a.Nu + k);
#pragma unroll
                            for (int i = 0; i < NPT; ++i) dn[i] = bv - Fi[i];
                        }
                        float Gr[NPT], Er[NPT];
                        ld_vec<NPT>(&sdg[sx][i0], Gr);
                        ld_vec<NPT>(&seps[sx][i0], Er);
                        lift_vec<NPT>(t, Gr, Er, dn, Fi, toh0 * u1, div, true);
                    }
                    // ---- second direction: lines (j', kz) of the element and of the upwind y element
                    {
                        float t[NPT], dn[NPT];
#pragma unroll
                        for (int i = 0; i < NPT; ++i) t[i] = 0.f;
                        float Dr[Q];
                        ld_vec<Q>(&sDr[sy][jy][0], Dr);
                        const float4 cf = sCf[sy][jy];
#pragma unroll
                        for (int m = 1; m < Q; ++m) {
                            const int jp = (jy + m) % Q;             // the canonical order
                            float Gv[NPT];
                            ld_vec<NPT>(sc + own_off + Q * (jp + Q * kz) + i0, Gv);
                            acc_dev<NPT>(t, Dr[m], Gv, Fi);
                        }
                        if (!BC || !((bcm >> (2 + sy)) & 1)) {
                            float Lr[Q];
                            ld_vec<Q>(&slam[sy][0], Lr);
                            scale_vec<NPT>(dn, cf.x, Fi);
#pragma unroll
                            for (int jp = 0; jp < Q; ++jp) {
                                float H[NPT];
                                ld_vec<NPT>(sc + (SLOTS + l) * NS + Q * (jp + Q * kz) + i0, H);
                                acc_dev<NPT>(dn, Lr[jp], H, Fi);
                            }
                        } else {
                            const float bv = (float)__ldg(a.bcval + ((size_t)(2 + sy) * C + c) * a.Nu + k);
#pragma unroll
                            for (int i = 0; i < NPT; ++i) dn[i] = bv - Fi[i];
                        }
                        float dgv[NPT], epv[NPT];
#pragma unroll
                        for (int i = 0; i < NPT; ++i) { dgv[i] = cf.y; epv[i] = cf.z; }
                        lift_vec<NPT>(t, dgv, epv, dn, Fi, toh1 * u2, div, false);
                    }
                    // ---- third direction: lines (jy, k') of the element and of the upwind z element
                    {
                        float t[NPT], dn[NPT];
#pragma unroll
                        for (int i = 0; i < NPT; ++i) t[i] = 0.f;
                        float Dr[Q];
                        ld_vec<Q>(&sDr[sz][kz][0], Dr);
                        const float4 cf = sCf[sz][kz];
#pragma unroll
                        for (int m = 1; m < Q; ++m) {
                            const int kp = (kz + m) % Q;             // the canonical order
                            float Gv[NPT];
                            ld_vec<NPT>(sc + own_off + Q * (jy + Q * kp) + i0, Gv);
                            acc_dev<NPT>(t, Dr[m], Gv, Fi);
                        }
                        if (!BC || !((bcm >> (4 + sz)) & 1)) {
                            float Lr[Q];
                            ld_vec<Q>(&slam[sz][0], Lr);
                            scale_vec<NPT>(dn, cf.x, Fi);
#pragma unroll
                            for (int kp = 0; kp < Q; ++kp) {
                                float H[NPT];
                                ld_vec<NPT>(sc + (SLOTS + EB + l) * NS + Q * (jy + Q * kp) + i0, H);
                                acc_dev<NPT>(dn, Lr[kp], H, Fi);
                            }
                        } else {
                            const float bv = (float)__ldg(a.bcval + ((size_t)(4 + sz) * C + c) * a.Nu + k);
#pragma unroll
                            for (int i = 0; i < NPT; ++i) dn[i] = bv - Fi[i];
                        }
                        float dgv[NPT], epv[NPT];
#pragma unroll
                        for (int i = 0; i < NPT; ++i) { dgv[i] = cf.y; epv[i] = cf.z; }
                        lift_vec<NPT>(t, dgv, epv, dn, Fi, toh2 * u3, div, false);
                    }
                    // ---- equilibrium, source and Runge--Kutta update
                    float FN[NPT];
                    if (fa != 0.f) ld_vec<NPT>(sc + (SLOTS + 2 * EB + l) * NS + ln + i0, FN);
                    if constexpr (NPT % 2 == 0) {
                        // the same operations on pairs of points
                        const float2 u12 = dup2(u1);
#pragma unroll
                        for (int i = 0; i < NPT; i += 2) {
                            const float2 c1 = sub2(u12, make_float2(V1[i], V1[i + 1]));
                            const float2 ex = __ffma2_rn(c1, __ffma2_rn(make_float2(A11[i], A11[i + 1]), c1,
                                                                         make_float2(lin[i], lin[i + 1])),
                                                         make_float2(cst[i], cst[i + 1]));
                            const float2 g32 = __fmul2_rn(make_float2(E0[i], E0[i + 1]),
                                                          make_float2(Eq32::ex2(ex.x), Eq32::ex2(ex.y)));
                            const float2 t1 = sub2(u12, make_float2(U0x[i], U0x[i + 1]));
                            const float2 corr = __ffma2_rn(t1, __ffma2_rn(make_float2(gm4h[i], gm4h[i + 1]), t1,
                                                                           make_float2(gm1[i], gm1[i + 1])),
                                                           make_float2(cl[i], cl[i + 1]));
                            const float2 gc = __fmul2_rn(g32, corr);
                            const float2 gf = make_float2(gfac[i], gfac[i + 1]);
                            const float2 eqv = (c == 0) ? g32 : __fmul2_rn(gf, g32);
                            const float2 eqc = (c == 0) ? gc : __fmul2_rn(gf, gc);
                            const float2 F2 = make_float2(Fi[i], Fi[i + 1]), it2 = make_float2(itau[i], itau[i + 1]);
                            const float2 R = __ffma2_rn(sub2(eqv, F2), it2,
                                                        __ffma2_rn(eqc, it2, make_float2(-div[i], -div[i + 1])));
                            const float2 o = rk_update2(F2, fa != 0.f ? make_float2(FN[i], FN[i + 1]) : dup2(0.f), R, fa,
                                                        fab, fc, fa != 0.f);
                            outv[c][i] = o.x; outv[c][i + 1] = o.y;
                        }
                    } else {
#pragma unroll
                    for (int i = 0; i < NPT; ++i) {
                        const float c1 = __fsub_rn(u1, V1[i]);
                        const float g32 = __fmul_rn(E0[i], Eq32::ex2(fmaf(c1, fmaf(A11[i], c1, lin[i]), cst[i])));
                        const float t1 = u1 - U0x[i];
                        const float corr = fmaf(t1, fmaf(gm4h[i], t1, gm1[i]), cl[i]);
                        const float gc = __fmul_rn(g32, corr);
                        const float eqv = (c == 0) ? g32 : __fmul_rn(gfac[i], g32);
                        const float eqc = (c == 0) ? gc : __fmul_rn(gfac[i], gc);
                        const float R = fmaf(eqv - Fi[i], itau[i], fmaf(eqc, itau[i], -div[i]));
                        outv[c][i] = rk_update(Fi[i], fa != 0.f ? FN[i] : 0.f, R, fa, fab, fc, fa != 0.f);
                    }
                    }
                    if (active) st_vec<NPT>(a.f_out + ((size_t)c * a.Nu + k) * slab + pb, outv[c]);
                }
                }
                if (mom) {
                    const float cj = su1c[j1].y;
                    if constexpr (NPT % 2 == 0) {
#pragma unroll
                        for (int i = 0; i < NPT; i += 2)
                            add_pair<C>(acc[i], acc[i + 1], cj, jt1, make_float2(outv[0][i], outv[0][i + 1]),
                                        C == 2 ? make_float2(outv[C - 1][i], outv[C - 1][i + 1]) : make_float2(0.f, 0.f));
                    } else {
#pragma unroll
                        for (int i = 0; i < NPT; ++i) acc[i].add(cj, jt1, outv[0][i], C == 2 ? outv[C - 1][i] : 0.f);
                    }
                }
            }
            // release the slot; the warp that releases it last refills it with
            // the velocity S ahead
            __syncwarp();
            int go = 0;
            if (lane == 0) {
                __threadfence_block();
                if (atom_add_shared(&rel[slot], 1u) == NW - 1) {
                    rel[slot] = 0;
                    __threadfence_block();
                    go = (k - k0) + S < *(volatile int *)&s_nfill ? 2 : 1;
                }
            }
            // the whole warp refills the slot (warp-uniform operands; one
            // elected lane issues the copies)
            if (__shfl_sync(0xffffffffu, go, 0) == 2) {
                // velocity k + S by its axis indices (velocity blocks are whole lines)
                int i1 = j1 + S, i2 = j2, i3 = j3;
                while (i1 >= vn1) {
                    i1 -= vn1;
                    if (++i2 == vn2) { i2 = 0; ++i3; }
                }
                ring_issue_u<Q, C, EB, true, true>(a, g, sbuf, bars, slot, k + S, make_float3(su1c[i1].x, su2[i2], su3[i3]));
                if (lane == 0) fills[slot] += 1;
            }
            if (++slot == S) { slot = 0; par ^= 1u; }
        }
        if (!ok) break;
        if (mom && active) {
            // end of the line: c2 jt2^b (line pair) into the plane pairs
            const float c2 = trap(j2, vn2), jt2 = (float)(j2 - jc[1]);
            const float bq = __fmul_rn(c2, jt2), bbq = __fmul_rn(__fmul_rn(c2, jt2), jt2);
#pragma unroll
            for (int i = 0; i < NPT; ++i) {
                float *P = Pme + i * 2 * NQ * NCT;
                plane_add_s<NQ>(P, NCT, 0, c2, acc[i].Ls(0), acc[i].Lcs(0));
                plane_add_s<NQ>(P, NCT, 1, c2, acc[i].Ls(1), acc[i].Lcs(1));
                plane_add_s<NQ>(P, NCT, 2, c2, acc[i].Ls(2), acc[i].Lcs(2));
                plane_add_s<NQ>(P, NCT, 3, bq, acc[i].Ls(0), acc[i].Lcs(0));
                plane_add_s<NQ>(P, NCT, 4, bq, acc[i].Ls(1), acc[i].Lcs(1));
                plane_add_s<NQ>(P, NCT, 5, bbq, acc[i].Ls(0), acc[i].Lcs(0));
                if (C == 2) plane_add_s<NQ>(P, NCT, NQ - 1, c2, acc[i].Ls(3), acc[i].Lcs(3));
            }
        }
    }
    if (!ok) {
        // a wait gave up: report it; the last warp to leave waits (bounded)
        // for the latest fill of every slot, so no copy is in flight at exit
        if (lane == 0) {
            atomicOr(a.status, BGK_DEV_TIMEOUT);
            __threadfence_block();
            if (atomicAdd(&s_exited, 1u) == NW - 1) {
                __threadfence_block();
                for (int i = 0; i < S; ++i)
                    if (fills[i] > 0) mbar_wait(smem_u32(bars + i), (fills[i] - 1) & 1, a.wait_ns);
            }
        }
        return;
    }
    if (mom && active) {
        if (j3cur >= 0) flush_plane(j3cur);
        const double uc[3] = {vg.lo[0] + jc[0] * vg.h[0], vg.lo[1] + jc[1] * vg.h[1], vg.lo[2] + jc[2] * vg.h[2]};
#pragma unroll
        for (int i = 0; i < NPT; ++i) {
            double *J = a.part + (size_t)vb * BGK_NMOM * a.P + pb + i;
            double Jv[11], m[BGK_NMOM];
#pragma unroll
            for (int q = 0; q < 11; ++q) Jv[q] = first_plane ? 0.0 : J[(size_t)q * a.P];
            index_to_raw(Jv, vg, uc, m);
#pragma unroll
            for (int q = 0; q < BGK_NMOM; ++q) J[(size_t)q * a.P] = m[q];
        }
    }
}

// Launch configurations: (nodes per thread, run length) per variant and order.
//   line:      NPT = Q,   runs of 4 (Q = 4) / 16 (Q = 2) elements
//   line_wide: NPT = Q,   runs of 8 / 32
//   half:      NPT = Q/2, runs of 4 / 16
//   half_wide: NPT = Q/2, runs of 8 / 32
template <int Q, int C, int EB, int NPT>
size_t line_smem(int depth) {
    using LG = LineGeom<Q, C, EB, NPT>;
    return (size_t)depth * StageGeom<Q, C, EB>::STAGE * sizeof(float) +
           (size_t)NPT * 2 * LG::NQ * LG::NCT * sizeof(float) + 2 * (size_t)depth * sizeof(unsigned long long) +
           2 * (size_t)depth * sizeof(unsigned int);
}

template <int Q, int C, int EB, int NPT>
cudaError_t line_launch(const StageArgs<float> &a, int n_vblk, int depth, cudaStream_t s) {
    const size_t smem = line_smem<Q, C, EB, NPT>(depth);
    static SmemLimit lim;
    size_t *attr = lim.slot();
    if (!attr) return cudaErrorInvalidDevice;
    if (smem > *attr) {
        cudaError_t e = cudaFuncSetAttribute(k_stage_f32_line<Q, C, EB, NPT, false>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_stage_f32_line<Q, C, EB, NPT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem);
        if (e != cudaSuccess) return e;
        *attr = smem;
    }
    const int cpr = (a.mesh.n[0] + EB - 1) / EB;
    dim3 grid(cpr * a.mesh.n[1] * a.mesh.n[2], n_vblk);
    if (a.mesh.periodic[0] && a.mesh.periodic[1] && a.mesh.periodic[2])
        k_stage_f32_line<Q, C, EB, NPT, false><<<grid, LineGeom<Q, C, EB, NPT>::NTHR, smem, s>>>(a, depth);
    else
        k_stage_f32_line<Q, C, EB, NPT, true><<<grid, LineGeom<Q, C, EB, NPT>::NTHR, smem, s>>>(a, depth);
    return cudaGetLastError();
}

// kind: 0 line, 1 line_wide, 2 half, 3 half_wide.  With launch == false only
// the shared-memory size is returned (through *smem).
template <int Q, int C>
cudaError_t line_dispatch(int kind, bool launch, const StageArgs<float> &a, int n_vblk, int depth, cudaStream_t s,
                          size_t *smem) {
    constexpr int EBS = Q == 4 ? 4 : 16, EBW = 2 * EBS, NH = Q / 2;
    switch (kind) {
        case 0: *smem = line_smem<Q, C, EBS, Q>(depth); return launch ? line_launch<Q, C, EBS, Q>(a, n_vblk, depth, s) : cudaSuccess;
        case 1: *smem = line_smem<Q, C, EBW, Q>(depth); return launch ? line_launch<Q, C, EBW, Q>(a, n_vblk, depth, s) : cudaSuccess;
        case 2: *smem = line_smem<Q, C, EBS, NH>(depth); return launch ? line_launch<Q, C, EBS, NH>(a, n_vblk, depth, s) : cudaSuccess;
        case 3: *smem = line_smem<Q, C, EBW, NH>(depth); return launch ? line_launch<Q, C, EBW, NH>(a, n_vblk, depth, s) : cudaSuccess;
        default: return cudaErrorInvalidValue;
    }
}

// p = 2: runs of 16 elements (144 lines of 3 points, in five warps), the
// line mapping only
template <int C>
cudaError_t line_dispatch3(int kind, bool launch, const StageArgs<float> &a, int n_vblk, int depth, cudaStream_t s,
                           size_t *smem) {
    if (kind != 0) return cudaErrorInvalidValue;
    *smem = line_smem<3, C, 16, 3>(depth);
    return launch ? line_launch<3, C, 16, 3>(a, n_vblk, depth, s) : cudaSuccess;
}

cudaError_t line_any(int kind, bool launch, const StageArgs<float> &a, int C, int n_vblk, int depth, cudaStream_t s,
                     size_t *smem) {
    if (a.fr.q == 4) return C == 1 ? line_dispatch<4, 1>(kind, launch, a, n_vblk, depth, s, smem)
                                   : line_dispatch<4, 2>(kind, launch, a, n_vblk, depth, s, smem);
    if (a.fr.q == 3) return C == 1 ? line_dispatch3<1>(kind, launch, a, n_vblk, depth, s, smem)
                                   : line_dispatch3<2>(kind, launch, a, n_vblk, depth, s, smem);
    return C == 1 ? line_dispatch<2, 1>(kind, launch, a, n_vblk, depth, s, smem)
                  : line_dispatch<2, 2>(kind, launch, a, n_vblk, depth, s, smem);
}

bool aligned_to(const void *p, uintptr_t n) { return ((uintptr_t)p & (n - 1)) == 0; }

}  // namespace

bool stage_f32_line_supported(const StageArgs<float> &a, int C, int kind, int depth) {
    const int Q = a.fr.q;
    if (Q != 2 && Q != 3 && Q != 4) return false;
    if (kind < 0 || kind > 3 || depth < 2 || depth > BGK_MAX_DEPTH || !a.eq32) return false;
    // p = 2: the line mapping, on rows of whole 4-element (16-byte) groups
    if (Q == 3 && (kind != 0 || a.mesh.n[0] % 4 != 0)) return false;
    for (int f = 0; f < 6; ++f)
        if (a.mesh.specular[f]) return false;               // reflected traces are not staged
    if (a.geo) return false;                                // curvilinear: the plain kernel only
    if (!aligned_to(a.f_s, 16) || (a.a32 != 0.f && !aligned_to(a.f_n, 16)) || !aligned_to(a.f_out, 16)) return false;
    size_t smem = 0;
    line_any(kind, false, a, C, 0, depth, nullptr, &smem);
    return smem <= 200 * 1024;
}

cudaError_t launch_stage_f32_line(const StageArgs<float> &a, int C, int n_vblk, int kind, int depth, cudaStream_t s) {
    if (!stage_f32_line_supported(a, C, kind, depth)) return cudaErrorInvalidValue;
    size_t smem = 0;
    return line_any(kind, true, a, C, n_vblk, depth, s, &smem);
}
