// Pieces shared by the mixed-form (FP32 state) stage kernels: error-free
// moment accumulation, the FP32 operator tables of the deviation-form FR
// advection, and the asynchronous copy ring (mbarriers, bulk copies, the
// producer) of the pipelined kernels.  Dzanic & Martinelli, arXiv 2312.06567,
// section "Methodology" (the stage being computed).
#pragma once

#include "bgk_internal.cuh"

namespace {

// Error-free accumulation (Ogita, Rump & Oishi 2005, "Sum2"): TwoSum keeps
// the exact rounding error of each addition in comp; the represented sum is
// s + comp, accurate to O(eps^2) of the sum of magnitudes.
__device__ __forceinline__ void sum2(float &s, float &comp, float v) {
    const float t = __fadd_rn(s, v);
    const float bp = __fsub_rn(t, s);
    const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(v, bp));
    s = t;
    comp = __fadd_rn(comp, e);
}

// Packed FP32 pairs (two IEEE operations per issue, each rounded exactly as
// its scalar form).  x - y, one rounding of the exact difference, is the
// same IEEE operation as x + (-y) and, paired, fma(y, -1, x) (y * -1 is
// exact).
__device__ __forceinline__ float2 sub2(float2 x, float2 y) { return __ffma2_rn(y, make_float2(-1.f, -1.f), x); }
__device__ __forceinline__ float2 dup2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 neg2(float2 v) { return make_float2(-v.x, -v.y); }
// sum2 on two independent (sum, error) pairs at once
__device__ __forceinline__ void sum2x2(float2 &s, float2 &c, float2 v) {
    const float2 t = __fadd2_rn(s, v);
    const float2 bp = sub2(t, s);
    const float2 e = __fadd2_rn(sub2(s, sub2(t, bp)), sub2(v, bp));
    s = t;
    c = __fadd2_rn(c, e);
}

// Index moments (J000, J100, J200, J010, J110, J020, J001, J101, J011, J002, JG)
// of one thread -> the 11 raw moment slots, W = h1 h2 h3.
__device__ __forceinline__ void index_to_raw(const double J[11], const VelGrid &vg, const double uc[3],
                                             double m[BGK_NMOM]) {
    const double W = vg.h[0] * vg.h[1] * vg.h[2];
    const double h1 = vg.h[0], h2 = vg.h[1], h3 = vg.h[2];
    const double J000 = J[0], J100 = J[1], J200 = J[2], J010 = J[3], J110 = J[4], J020 = J[5];
    const double J001 = J[6], J101 = J[7], J011 = J[8], J002 = J[9];
    m[0] = W * J000;
    m[1] = W * (uc[0] * J000 + h1 * J100);
    m[2] = W * (uc[1] * J000 + h2 * J010);
    m[3] = W * (uc[2] * J000 + h3 * J001);
    m[4] = W * (uc[0] * uc[0] * J000 + 2.0 * uc[0] * h1 * J100 + h1 * h1 * J200);
    m[5] = W * (uc[1] * uc[1] * J000 + 2.0 * uc[1] * h2 * J010 + h2 * h2 * J020);
    m[6] = W * (uc[2] * uc[2] * J000 + 2.0 * uc[2] * h3 * J001 + h3 * h3 * J002);
    m[7] = W * (uc[0] * uc[1] * J000 + uc[0] * h2 * J010 + h1 * uc[1] * J100 + h1 * h2 * J110);
    m[8] = W * (uc[0] * uc[2] * J000 + uc[0] * h3 * J001 + h1 * uc[2] * J100 + h1 * h3 * J101);
    m[9] = W * (uc[1] * uc[2] * J000 + uc[1] * h3 * J001 + h2 * uc[2] * J010 + h2 * h3 * J011);
    m[10] = W * J[10];
}

// The Runge--Kutta update (a + b) f + a (f^n - f) + c R of the mixed form,
// with one rounding at the level of f: the two small terms are summed first
// (their roundings are relative to themselves) and added to f last.  Adding
// a (f^n - f) to f first, on its own, rounds a value with few low bits
// (f^n - f is a whole number of ulps of f, and a = 3/4 leaves two fraction
// bits): on states that repeat across points those roundings do not cancel
// (2e-8 of the mass per step on a 512-point box holding 8 distinct states).
// has_n: a != 0 (FN is read only then).  x - y is one rounding, as x + (-y).
__device__ __forceinline__ float rk_update(float F, float FN, float R, float fa, float fab, float fc, bool has_n) {
    const float base = fab == 1.f ? F : __fmul_rn(fab, F);
    if (!has_n) return fmaf(fc, R, base);
    return __fadd_rn(base, fmaf(fa, __fsub_rn(FN, F), __fmul_rn(fc, R)));
}
// the same on two values at once, lane for lane
__device__ __forceinline__ float2 rk_update2(float2 F, float2 FN, float2 R, float fa, float fab, float fc, bool has_n) {
    const float2 base = fab == 1.f ? F : __fmul2_rn(make_float2(fab, fab), F);
    if (!has_n) return __ffma2_rn(make_float2(fc, fc), R, base);
    const float2 dN = __ffma2_rn(F, make_float2(-1.f, -1.f), FN);
    return __fadd2_rn(base, __ffma2_rn(make_float2(fa, fa), dN, __fmul2_rn(make_float2(fc, fc), R)));
}

// The same accumulation with the plane pairs and the FP64 index moments kept
// in shared memory (column `t` of [field][n] arrays, so a warp's accesses hit
// distinct banks): they change once per line and once per plane, and holding
// them in registers would cost the pipelined stage kernel a third of its
// occupancy.
struct IndexMomentsS {
    // the current line's (sum, error) pairs as packed pairs: A = (L0, LG) of
    // c F and c G, B = (L1, L2) of c F jt and c F jt^2
    float2 A, Ae, B, Be;
    float *P;                 // [14][n]: P[0..6] then Pc[0..6]
    double *J;                // [11][n]
    int n;
    int j3cur;
    __device__ void init(float *Ps, double *Js, int ncol, int t) {
        P = Ps + t;
        J = Js + t;
        n = ncol;
        A = Ae = B = Be = make_float2(0.f, 0.f);
#pragma unroll
        for (int i = 0; i < 14; ++i) P[i * n] = 0.f;
#pragma unroll
        for (int i = 0; i < 11; ++i) J[i * n] = 0.0;
        j3cur = -1;
    }
    // IndexMoments::add, lane for lane the same operations on the pairs (the
    // product errors taken negated, fma(x, -y, p) = -(x y - p) exactly, and
    // subtracted)
    __device__ __forceinline__ void add(float cj1, float jt1, float F, float G) {
        const float2 cFG = __fmul2_rn(dup2(cj1), make_float2(F, G));
        sum2x2(A, Ae, cFG);
        const float jj = __fmul_rn(jt1, jt1), njt1 = -jt1, njj = __fmul_rn(njt1, jt1);      // exact
        const float2 cF = dup2(cFG.x);
        const float2 p = __fmul2_rn(cF, make_float2(jt1, jj));
        sum2x2(B, Be, p);
        Be = sub2(Be, __ffma2_rn(cF, make_float2(njt1, njj), p));
    }
    __device__ __forceinline__ void plane_add(int i, float c, float sum, float err) {
        float ps = P[i * n], pc = P[(7 + i) * n];
        const float pr = __fmul_rn(c, sum);
        sum2(ps, pc, pr);
        pc = __fadd_rn(pc, fmaf(c, sum, -pr));
        pc = fmaf(c, err, pc);
        P[i * n] = ps;
        P[(7 + i) * n] = pc;
    }
    __device__ __forceinline__ void end_line(float c2, float jt2) {
        const float a = c2, b = __fmul_rn(c2, jt2), bb = __fmul_rn(__fmul_rn(c2, jt2), jt2);
        plane_add(0, a, A.x, Ae.x);
        plane_add(1, a, B.x, Be.x);
        plane_add(2, a, B.y, Be.y);
        plane_add(3, b, A.x, Ae.x);
        plane_add(4, b, B.x, Be.x);
        plane_add(5, bb, A.x, Ae.x);
        plane_add(6, a, A.y, Ae.y);
        A = Ae = B = Be = make_float2(0.f, 0.f);
    }
    __device__ __forceinline__ void flush_plane(float c3, float jt3) {
        const double c = c3, t = jt3;
        double Pd[7];
#pragma unroll
        for (int i = 0; i < 7; ++i) {
            Pd[i] = (double)P[i * n] + (double)P[(7 + i) * n];
            P[i * n] = 0.f;
            P[(7 + i) * n] = 0.f;
        }
        J[0] = fma(c, Pd[0], J[0]);
        J[n] = fma(c, Pd[1], J[n]);
        J[2 * n] = fma(c, Pd[2], J[2 * n]);
        J[3 * n] = fma(c, Pd[3], J[3 * n]);
        J[4 * n] = fma(c, Pd[4], J[4 * n]);
        J[5 * n] = fma(c, Pd[5], J[5 * n]);
        J[6 * n] = fma(c * t, Pd[0], J[6 * n]);
        J[7 * n] = fma(c * t, Pd[1], J[7 * n]);
        J[8 * n] = fma(c * t, Pd[3], J[8 * n]);
        J[9 * n] = fma(c * t * t, Pd[0], J[9 * n]);
        J[10 * n] = fma(c, Pd[6], J[10 * n]);
    }
    __device__ __forceinline__ void get(double out[11]) const {
#pragma unroll
        for (int i = 0; i < 11; ++i) out[i] = J[i * n];
    }
};

// Dt[side] = D - dg (x) l rounded to FP32 with explicit roundings, so every
// use (the operator itself and the conservation weights built from it) sees
// the same FP32 entries.
__device__ __forceinline__ float folded_dt(const FROps &fr, int side, int i, int j) {
    const double dg = side == 0 ? fr.dgL[i] : fr.dgR[i];
    const double l = side == 0 ? fr.lm[j] : fr.lp[j];
    return __double2float_rn(__dsub_rn(fr.D[i][j], __dmul_rn(dg, l)));
}

__device__ __forceinline__ float trap(int j, int n) { return (j == 0 || j == n - 1) ? 0.5f : 1.0f; }

// Per-thread accumulator of index moments over a run of whole first-axis lines.
// Line sums are error-free (Sum2) sums of exact products (c F exact; c F jt
// and c F jt^2 split into product + FMA-exact error); plane sums accumulate
// the lines' (sum, error) pairs the same way; planes fold in FP64.  So the
// index moments are accurate to O(2^-48) of the sums, with no bias.
struct IndexMoments {
    float L[4], Lc[4];                    // current line: 0, jt, jt^2, G (sum, error) pairs
    float P[7], Pc[7];                    // current plane: 00 10 20 01 11 02 G
    double J[11];
    int j3cur;
    __device__ void init() {
#pragma unroll
        for (int i = 0; i < 4; ++i) L[i] = Lc[i] = 0.f;
#pragma unroll
        for (int i = 0; i < 7; ++i) P[i] = Pc[i] = 0.f;
#pragma unroll
        for (int i = 0; i < 11; ++i) J[i] = 0.0;
        j3cur = -1;
    }
    __device__ __forceinline__ void add(float cj1, float jt1, float F, float G) {
        const float cF = __fmul_rn(cj1, F);                 // exact: cj1 in {1/2, 1}
        sum2(L[0], Lc[0], cF);
        const float p1 = __fmul_rn(cF, jt1);
        sum2(L[1], Lc[1], p1);
        Lc[1] = __fadd_rn(Lc[1], fmaf(cF, jt1, -p1));       // exact product error joins the error term
        const float jj = __fmul_rn(jt1, jt1);               // exact: |jt1| < 128
        const float p2 = __fmul_rn(cF, jj);
        sum2(L[2], Lc[2], p2);
        Lc[2] = __fadd_rn(Lc[2], fmaf(cF, jj, -p2));
        sum2(L[3], Lc[3], __fmul_rn(cj1, G));
    }
    __device__ __forceinline__ void flush_plane(float c3, float jt3) {
        const double c = c3, t = jt3;
        // the plane sums are P + Pc
        const double P00 = (double)P[0] + (double)Pc[0], P10 = (double)P[1] + (double)Pc[1];
        const double P20 = (double)P[2] + (double)Pc[2], P01 = (double)P[3] + (double)Pc[3];
        const double P11 = (double)P[4] + (double)Pc[4], P02 = (double)P[5] + (double)Pc[5];
        const double PG = (double)P[6] + (double)Pc[6];
        // J_abc += c3 jt3^c P_ab
        J[0] = fma(c, P00, J[0]);
        J[1] = fma(c, P10, J[1]);
        J[2] = fma(c, P20, J[2]);
        J[3] = fma(c, P01, J[3]);
        J[4] = fma(c, P11, J[4]);
        J[5] = fma(c, P02, J[5]);
        J[6] = fma(c * t, P00, J[6]);
        J[7] = fma(c * t, P10, J[7]);
        J[8] = fma(c * t, P01, J[8]);
        J[9] = fma(c * t * t, P00, J[9]);
        J[10] = fma(c, PG, J[10]);
#pragma unroll
        for (int i = 0; i < 7; ++i) P[i] = Pc[i] = 0.f;
    }
    // add c * (sum + err) of a line pair into a plane pair, error-free up to
    // O(eps^2) (c is a small integer or half-integer)
    __device__ __forceinline__ void plane_add(int i, float c, float sum, float err) {
        const float ps = __fmul_rn(c, sum);
        sum2(P[i], Pc[i], ps);
        Pc[i] = __fadd_rn(Pc[i], fmaf(c, sum, -ps));
        Pc[i] = fmaf(c, err, Pc[i]);
    }
    __device__ __forceinline__ void end_line(float c2, float jt2) {
        const float a = c2, b = __fmul_rn(c2, jt2), bb = __fmul_rn(__fmul_rn(c2, jt2), jt2);   // exact
        plane_add(0, a, L[0], Lc[0]);
        plane_add(1, a, L[1], Lc[1]);
        plane_add(2, a, L[2], Lc[2]);
        plane_add(3, b, L[0], Lc[0]);
        plane_add(4, b, L[1], Lc[1]);
        plane_add(5, bb, L[0], Lc[0]);
        plane_add(6, a, L[3], Lc[3]);
#pragma unroll
        for (int i = 0; i < 4; ++i) L[i] = Lc[i] = 0.f;
    }
};

// Shared-memory FP32 operator tables of the deviation-form advection (used by
// both FP32 stage kernels): Dt[side] (inflow trace folded in), dg[side], the
// exact defects eps_i = sum_j Dt_ij + dg_i, the telescoping neighbour-trace
// weights lambda_j = +-sum_i W_i Dt_ij and dlam = sum_j lambda_j - 1.
template <int Q>
__device__ __forceinline__ void load_ops_f32(const FROps &fr, int tid, float (*sD)[Q][Q], float (*sdg)[Q],
                                             float (*seps)[Q], float (*slam)[Q], float *sdlam) {
    if (tid < Q * Q) {
        const int i = tid / Q, j = tid % Q;
        sD[0][i][j] = folded_dt(fr, 0, i, j);
        sD[1][i][j] = folded_dt(fr, 1, i, j);
    }
    if (tid < 2 * Q) {
        const int side = tid / Q, j = tid % Q;
        double lam = 0.0, eps = side == 0 ? fr.dgL[j] : fr.dgR[j];
        for (int i = 0; i < Q; ++i) {
            lam = fma(fr.wq[i], (double)folded_dt(fr, side, i, j), lam);
            eps += (double)folded_dt(fr, side, j, i);
        }
        slam[side][j] = (float)(side == 0 ? lam : -lam);
        seps[side][j] = (float)eps;
        sdg[side][j] = (float)(side == 0 ? fr.dgL[j] : fr.dgR[j]);
        if (j == 0) {
            double tot = 0.0;
            for (int jj = 0; jj < Q; ++jj)
                for (int i = 0; i < Q; ++i) tot = fma(fr.wq[i], (double)folded_dt(fr, side, i, jj), tot);
            sdlam[side] = (float)((side == 0 ? tot : -tot) - 1.0);
        }
    }
}

// ---- asynchronous copy ring -------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Wait for the completion of the barrier phase of the given parity; false
// after limit_ns (0: about 2 s) without it.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, unsigned long long limit_ns = 0) {
    if (mbar_try(bar, parity)) return true;
    const unsigned long long lim = limit_ns ? limit_ns : 2000000000ull;
    const unsigned long long t0 = global_ns();
    for (;;) {
        // the timer is read once per 32 polls (each poll may suspend briefly)
        for (int i = 0; i < 32; ++i)
            if (mbar_try(bar, parity)) return true;
        if (global_ns() - t0 > lim) return false;
    }
}
// The same wait with its limit read from shared memory only once the first
// poll fails (keeps the limit out of the registers of a hot loop).
__device__ __forceinline__ bool mbar_wait_s(uint32_t bar, uint32_t parity, const volatile unsigned long long *limit_ns) {
    if (mbar_try(bar, parity)) return true;
    return mbar_wait(bar, parity, *limit_ns);
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const float *src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}
// The same two operations executed by a whole warp with warp-uniform
// operands: one lane, chosen by elect.sync, performs them.
__device__ __forceinline__ void mbar_expect_tx_warp(uint32_t bar, uint32_t bytes) {
    asm volatile(
        "{\n\t.reg .pred p;\n\telect.sync _|p, 0xffffffff;\n\t"
        "@p mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n\t}" ::"r"(bar),
        "r"(bytes)
        : "memory");
}
__device__ __forceinline__ void bulk_g2s_warp(uint32_t dst, const float *src, uint32_t bytes, uint32_t bar) {
    asm volatile(
        "{\n\t.reg .pred p;\n\telect.sync _|p, 0xffffffff;\n\t"
        "@p cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n\t}" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

// A block of a pipelined stage kernel owns a run of up to EB consecutive
// elements of one mesh row (first axis); its stage buffer holds, per
// component: [x-halo | the run's EB elements | x-halo] [upwind y run]
// [upwind z run] [f^n run], each element NS floats.
template <int Q, int C, int EB, bool FN = true>
struct StageGeom {
    static constexpr int NS = Q * Q * Q;
    // x-halo slots on each side of the run: one element where an element is
    // a whole number of 16-byte units (Q = 2, 4); at Q = 3 (108 bytes) the
    // halo is copied as 4 elements (432 bytes) so that every bulk copy starts
    // and ends on a 16-byte boundary, the neighbour being the one next to
    // the run
    static constexpr int PAD = Q == 3 ? 4 : 1;
    static constexpr int SLOTS = EB + 2 * PAD;
    static constexpr int PER_C = (SLOTS + (FN ? 3 : 2) * EB) * NS;   // f^n run only with FN
    static constexpr int STAGE = C * PER_C;               // floats per stage buffer
};

struct RunGeom {
    int row, x0, nel, e0;
    // first element of the upwind neighbour run on side 0 (left) / 1 (right); -1: Dirichlet face
    int xn0, xn1, yn0, yn1, zn0, zn1;
    __device__ __forceinline__ void init(const MeshInfo &m, int EB, int bx) {
        const int n1 = m.n[0], n2 = m.n[1], n3 = m.n[2];
        const int cpr = (n1 + EB - 1) / EB;
        row = bx / cpr;
        x0 = (bx - row * cpr) * EB;
        nel = min(EB, n1 - x0);
        e0 = row * n1 + x0;
        const int ey = row % n2, ez = row / n2, pl = n1 * n2;
        xn0 = x0 > 0 ? e0 - 1 : (m.periodic[0] ? row * n1 + n1 - 1 : -1);
        xn1 = x0 + nel < n1 ? e0 + nel : (m.periodic[0] ? row * n1 : -1);
        yn0 = ey > 0 ? e0 - n1 : (m.periodic[1] ? e0 + (n2 - 1) * n1 : -1);
        yn1 = ey < n2 - 1 ? e0 + n1 : (m.periodic[1] ? e0 - (n2 - 1) * n1 : -1);
        zn0 = ez > 0 ? e0 - pl : (m.periodic[2] ? e0 + (n3 - 1) * pl : -1);
        zn1 = ez < n3 - 1 ? e0 + pl : (m.periodic[2] ? e0 - (n3 - 1) * pl : -1);
    }
};

// One thread: init the S "full" (one arrival + bytes) and S "empty" (one
// arrival per consumer warp) barriers of the ring.
__device__ __forceinline__ void ring_init(unsigned long long *bars, int S, int consumer_warps) {
    for (int i = 0; i < S; ++i) {
        mbar_init(smem_u32(bars + i), 1);
        mbar_init(smem_u32(bars + S + i), consumer_warps);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Copy everything velocity k (components u) needs into ring slot `slot`: the
// run, the upwind x element (if outside the run), the upwind y and z runs and
// (with FN) f^n, with bulk copies that complete on the slot's full barrier
// (one thread).
// WARP: called by a whole warp with warp-uniform arguments (one elected lane
// issues), else by one thread.
template <int Q, int C, int EB, bool FN = true, bool WARP = false>
__device__ __forceinline__ void ring_issue_u(const StageArgs<float> &a, const RunGeom &g, float *sbuf,
                                             unsigned long long *bars, int slot, int k, float3 u) {
    using SG = StageGeom<Q, C, EB, FN>;
    constexpr int NS = SG::NS, SLOTS = SG::SLOTS, PER_C = SG::PER_C, STAGE = SG::STAGE, PAD = SG::PAD;
    const size_t slab = (size_t)a.P;
    const uint32_t runb = (uint32_t)(g.nel * NS * 4), elb = PAD * NS * 4;
    const bool with_fn = FN && a.a32 != 0.f;
    const int xe = u.x > 0.f ? g.xn0 : g.xn1, ye = u.y > 0.f ? g.yn0 : g.yn1, ze = u.z > 0.f ? g.zn0 : g.zn1;
    const uint32_t bytes =
        C * (runb + (xe >= 0 ? elb : 0u) + (ye >= 0 ? runb : 0u) + (ze >= 0 ? runb : 0u) + (with_fn ? runb : 0u));
    const uint32_t full = smem_u32(bars + slot);
    if constexpr (WARP) mbar_expect_tx_warp(full, bytes);
    else mbar_expect_tx(full, bytes);
    auto copy = [&](uint32_t dst, const float *src, uint32_t nb) {
        if constexpr (WARP) bulk_g2s_warp(dst, src, nb, full);
        else bulk_g2s(dst, src, nb, full);
    };
    float *st = sbuf + (size_t)slot * STAGE;
#pragma unroll
    for (int c = 0; c < C; ++c) {
        const float *src = a.f_s + ((size_t)c * a.Nu + k) * slab;
        float *own = st + c * PER_C;
        copy(smem_u32(own + PAD * NS), src + (size_t)g.e0 * NS, runb);
        // the upwind x neighbour: left of the run into slot PAD - 1 (with the
        // PAD - 1 elements before it), right of it into slot PAD + nel (with
        // the PAD - 1 after it)
        if (xe >= 0)
            copy(smem_u32(own + (u.x > 0.f ? 0 : (g.nel + PAD) * NS)), src + (size_t)(u.x > 0.f ? xe - (PAD - 1) : xe) * NS,
                 elb);
        if (ye >= 0) copy(smem_u32(own + SLOTS * NS), src + (size_t)ye * NS, runb);
        if (ze >= 0) copy(smem_u32(own + (SLOTS + EB) * NS), src + (size_t)ze * NS, runb);
        if (with_fn)
            copy(smem_u32(own + (SLOTS + 2 * EB) * NS), a.f_n + ((size_t)c * a.Nu + k) * slab + (size_t)g.e0 * NS, runb);
    }
}
// the same with u read from the velocity table
template <int Q, int C, int EB, bool FN = true>
__device__ __forceinline__ void ring_issue(const StageArgs<float> &a, const RunGeom &g, float *sbuf,
                                           unsigned long long *bars, int slot, int k) {
    const float4 u = __ldg(a.vtab32 + k);
    ring_issue_u<Q, C, EB, FN>(a, g, sbuf, bars, slot, k, make_float3(u.x, u.y, u.z));
}

// The producer (one thread): for every velocity of [k0, k1) wait until the
// ring slot is free, then fill it (ring_issue).  On a timeout (its own, or a
// consumer's through *abort) it stops, waits (bounded) for its copies still
// in flight and sets BGK_DEV_TIMEOUT.
template <int Q, int C, int EB>
__device__ void ring_producer(const StageArgs<float> &a, const RunGeom &g, float *sbuf, unsigned long long *bars,
                              int S, int k0, int k1, volatile int *abort) {
    int i = 0;
    bool ok = true;
    const int n = a.ring_limit > 0 ? min(k1 - k0, a.ring_limit) : k1 - k0;
    for (; i < n; ++i) {
        const int slot = i % S;
        if (i >= S && !mbar_wait(smem_u32(bars + S + slot), ((i / S) & 1) ^ 1, a.wait_ns)) { ok = false; break; }
        if (*abort) { ok = false; break; }
        ring_issue<Q, C, EB>(a, g, sbuf, bars, slot, k0 + i);
    }
    if (!ok) {
        // no copy may still be in flight when the block exits
        for (int j = max(0, i - S); j < i; ++j) mbar_wait(smem_u32(bars + j % S), (j / S) & 1, a.wait_ns);
        atomicOr(a.status, BGK_DEV_TIMEOUT);
    }
}

}  // namespace
