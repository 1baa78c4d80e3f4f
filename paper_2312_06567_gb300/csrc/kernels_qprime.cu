// The Q' solve (Dzanic & Martinelli, arXiv 2312.06567, section "Numerical
// method": the modified equilibrium whose discrete moments equal those of f,
// found by Newton's method), one warp per solution point.
//
// Unknowns x = (rho', U', theta'); T'(theta') = theta'/Pr I + B with
// B = (1 - 1/Pr) Pi/rho of f; g = rho'/sqrt(det(2 pi T')) exp(-c^T T'^-1 c/2),
// c = u - U'.  Residual R = sum_k w_k psi~_k g_k - Q with
// psi~ = (1, u, |u|^2/2 + delta theta'/2); analytic Jacobian
//   dg/drho' = g/rho',  dg/dU' = g A c,  dg/dtheta' = g (|A c|^2 - tr A)/(2 Pr).
// Velocity sums are organised by lines along the first velocity axis: lanes
// take the n2*n3 lines, each line is walked outward from the node nearest
// its own peak with the Gaussian ratio recurrence g_{j+1} = g_j r_j,
// r_{j+1} = r_j exp(-A11 h1^2) (two exps per line; the walk only ever
// decreases g, so tails underflow harmlessly), giving five line sums
// T_m = sum_j w1 g ut1^m that fold into the 35 raw moments of order <= 4 in
// coordinates ut = u - U centred on the point's macroscopic velocity; R and
// J are linear combinations of those.
//
// Velocity-sum engines (k_qprime<F32>):
//   Engine64  FP64 throughout (the FP64 form; parity with the oracle);
//   Engine32  FP32 walk and fold (GB300's FP64 pipe issues 1/64 of the FP32
//             rate), Newton algebra in FP64, converged to FP32 resolution.
//             Used by the mixed form, whose conservation does not rest on
//             this solve: see the correction pass below;
//   fused_pass  (mixed form) the exact FP32 equilibrium evaluated once per
//             velocity for both the residual (from its exact moments) and
//             the Jacobian moments: used where the evaluation is expected to
//             be the last (from the learned guess, after an update), so the
//             correction needs no pass of its own.
// The mixed form's correction pass evaluates the exact FP32 equilibrium the
// stage will use (Eq32), measures its moments with exact-product compensated
// sums, and fits gamma so that g32 (1 + gamma . phi(ut)), phi = (1, ut,
// |ut|^2/2), has exactly the moments of f: the discrete compatibility
// condition then holds for the equilibrium actually used.
#include <type_traits>

#include "bgk_internal.cuh"

namespace {

constexpr double kTwoPi = 6.283185307179586476925286766559;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
template <int N>
__device__ __forceinline__ void warp_sum_n(double (&v)[N]) {
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = warp_sum(v[i]);
}

__device__ __forceinline__ void atomic_max_nonneg_double(unsigned long long *addr, double v) {
    if (!(v >= 0.0)) v = 1.0e300;      // NaN / negative: record as "huge"
    atomicMax(addr, (unsigned long long)__double_as_longlong(v));
}

struct Sym3 {
    double t11, t22, t33, t12, t13, t23;
};

__device__ __forceinline__ bool sym3_inverse(const Sym3 &t, Sym3 &inv, double &det) {
    const double c11 = t.t22 * t.t33 - t.t23 * t.t23;
    const double c12 = t.t13 * t.t23 - t.t12 * t.t33;
    const double c13 = t.t12 * t.t23 - t.t13 * t.t22;
    const double c22 = t.t11 * t.t33 - t.t13 * t.t13;
    const double c23 = t.t12 * t.t13 - t.t11 * t.t23;
    const double c33 = t.t11 * t.t22 - t.t12 * t.t12;
    det = t.t11 * c11 + t.t12 * c12 + t.t13 * c13;
    const bool spd = (t.t11 > 0.0) && (c33 > 0.0) && (det > 0.0);
    const double r = 1.0 / det;
    inv.t11 = c11 * r; inv.t22 = c22 * r; inv.t33 = c33 * r;
    inv.t12 = c12 * r; inv.t13 = c13 * r; inv.t23 = c23 * r;
    return spd;
}

// Gaussian elimination with partial pivoting on a 5x5 system; compile-time
// indices only so everything stays in registers.  Returns false if singular.
__device__ __forceinline__ bool solve5(double J[5][5], double r[5]) {
#pragma unroll
    for (int c = 0; c < 5; ++c) {
        int piv = c;
        double best = fabs(J[c][c]);
#pragma unroll
        for (int i = c + 1; i < 5; ++i) {
            const double v = fabs(J[i][c]);
            if (v > best) { best = v; piv = i; }
        }
        if (!(best > 0.0)) return false;
#pragma unroll
        for (int i = c + 1; i < 5; ++i) {
            if (i == piv) {
#pragma unroll
                for (int j = 0; j < 5; ++j) {
                    const double t = J[c][j]; J[c][j] = J[i][j]; J[i][j] = t;
                }
                const double t = r[c]; r[c] = r[i]; r[i] = t;
            }
        }
        const double inv = 1.0 / J[c][c];
#pragma unroll
        for (int i = c + 1; i < 5; ++i) {
            const double l = J[i][c] * inv;
#pragma unroll
            for (int j = c + 1; j < 5; ++j) J[i][j] = fma(-l, J[c][j], J[i][j]);
            r[i] = fma(-l, r[c], r[i]);
        }
    }
#pragma unroll
    for (int c = 4; c >= 0; --c) {
        double s = r[c];
#pragma unroll
        for (int j = c + 1; j < 5; ++j) s = fma(-J[c][j], r[j], s);
        r[c] = s / J[c][c];
    }
    return true;
}

// Index of the centred raw moment sum w g ut1^p1 ut2^p2 ut3^p3 (p1+p2+p3 <= 4)
// in the 35-slot accumulator; the slots run over (p2, p3, p1) in that order.
__host__ __device__ constexpr int midx(int p1, int p2, int p3) {
    int idx = 0;
    for (int a = 0; a <= 4; ++a)
        for (int b = 0; b <= 4 - a; ++b)
            for (int m = 0; m <= 4 - a - b; ++m) {
                if (a == p2 && b == p3 && m == p1) return idx;
                ++idx;
            }
    return -1;
}

// ---- per-point state shared by both engines ---------------------------------
struct PointState {
    double m[BGK_NMOM];
    double rho, U0[3], E, Eth, theta, mu, tau, hU2;
    double sc_rho, sc_mom, sc_E;
    Sym3 B;
    float feat[MLP_IN];
};

// One thread: the point's moments (sum of the velocity-block partials) and
// everything derived from them.
__device__ __forceinline__ void point_prologue(const QPrimeArgs &a, int p, PointState &ps) {
#pragma unroll
    for (int j = 0; j < BGK_NMOM; ++j) ps.m[j] = 0.0;
    for (int vb = 0; vb < a.n_vblk; ++vb) {
#pragma unroll
        for (int j = 0; j < BGK_NMOM; ++j) ps.m[j] += a.part[((size_t)vb * BGK_NMOM + j) * a.P + p];
    }
    const double *m = ps.m;
    const GasInfo &gs = a.gas;
    const double rho = m[0];
    ps.rho = rho;
    ps.U0[0] = m[1] / rho; ps.U0[1] = m[2] / rho; ps.U0[2] = m[3] / rho;
    const double *U0 = ps.U0;
    ps.E = 0.5 * (m[4] + m[5] + m[6]) + m[10];
    ps.hU2 = 0.5 * (U0[0] * U0[0] + U0[1] * U0[1] + U0[2] * U0[2]);
    ps.Eth = ps.E - rho * ps.hU2;
    const double pres = (gs.gamma - 1.0) * ps.Eth;
    ps.theta = pres / rho;
    const double es = (1.0 - 1.0 / gs.Pr) / rho;
    ps.B.t11 = es * (m[4] - rho * U0[0] * U0[0]);
    ps.B.t22 = es * (m[5] - rho * U0[1] * U0[1]);
    ps.B.t33 = es * (m[6] - rho * U0[2] * U0[2]);
    ps.B.t12 = es * (m[7] - rho * U0[0] * U0[1]);
    ps.B.t13 = es * (m[8] - rho * U0[0] * U0[2]);
    ps.B.t23 = es * (m[9] - rho * U0[1] * U0[2]);
    ps.mu = gs.mu_ref;
    if (gs.theta_S >= 0.0) {
        const double r = ps.theta / gs.theta_ref;
        ps.mu = gs.mu_ref * r * sqrt(r) * (gs.theta_ref + gs.theta_S) / (ps.theta + gs.theta_S);
    }
    ps.tau = ps.mu / (gs.Pr * pres);
    ps.sc_rho = 1.0 / rho;
    ps.sc_mom = 1.0 / (rho * sqrt(ps.theta));
    ps.sc_E = 1.0 / fabs(ps.E);
    // features of the learned guess: rho, U, theta, invariants of A = Pi/(rho theta), lambda
    const double ia = 1.0 / (rho * ps.theta);
    const double a11 = (m[4] - rho * U0[0] * U0[0]) * ia, a22 = (m[5] - rho * U0[1] * U0[1]) * ia;
    const double a33 = (m[6] - rho * U0[2] * U0[2]) * ia, a12 = (m[7] - rho * U0[0] * U0[1]) * ia;
    const double a13 = (m[8] - rho * U0[0] * U0[2]) * ia, a23 = (m[9] - rho * U0[1] * U0[2]) * ia;
    const double tr = a11 + a22 + a33;
    const double tr2 = a11 * a11 + a22 * a22 + a33 * a33 + 2.0 * (a12 * a12 + a13 * a13 + a23 * a23);
    const double det = a11 * (a22 * a33 - a23 * a23) - a12 * (a12 * a33 - a23 * a13) + a13 * (a12 * a23 - a22 * a13);
    ps.feat[0] = (float)rho; ps.feat[1] = (float)U0[0]; ps.feat[2] = (float)U0[1]; ps.feat[3] = (float)U0[2];
    ps.feat[4] = (float)ps.theta; ps.feat[5] = (float)tr; ps.feat[6] = (float)(0.5 * (tr * tr - tr2));
    ps.feat[7] = (float)det;
    ps.feat[8] = (float)(ps.mu / rho * sqrt(0.5 * kTwoPi * 0.5 / ps.theta));   // sqrt(pi / (2 theta))
}

// Newton's starting point: a supplied guess, the network's, or q.  The
// network runs on the whole warp; every lane returns the same x.  `left` is
// set when the network's guess left the admissible set (rho', theta' > 0).
__device__ __forceinline__ bool initial_guess(const QPrimeArgs &a, int p, int lane, const PointState &ps, double x[5],
                                              bool &left) {
    const double xq[5] = {ps.rho, ps.U0[0], ps.U0[1], ps.U0[2], ps.theta};
    left = false;
    if (a.guess) {
#pragma unroll
        for (int j = 0; j < 5; ++j) x[j] = a.guess[(size_t)p * 5 + j];
        return false;
    }
    if (a.guess_mode == 1) {
        float dg[MLP_OUT];
        mlp_infer_warp(a.mlp, ps.feat, dg, a.mlp_bf16, lane);
        const double st = sqrt(ps.theta);
        x[0] = ps.rho * (1.0 + dg[0]);
        x[1] = ps.U0[0] + st * dg[1]; x[2] = ps.U0[1] + st * dg[2]; x[3] = ps.U0[2] + st * dg[3];
        x[4] = ps.theta * (1.0 + dg[4]);
        if (x[0] > 0.0 && x[4] > 0.0) return true;
        left = true;
    }
#pragma unroll
    for (int j = 0; j < 5; ++j) x[j] = xq[j];
    return false;
}

// A = T'^-1, c0 = ln rho' - ln sqrt(det(2 pi T')) at x.
__device__ __forceinline__ void equilibrium_params(const PointState &ps, double Pr, const double x[5], Sym3 &A,
                                                   double &c0) {
    Sym3 T = ps.B;
    T.t11 += x[4] / Pr; T.t22 += x[4] / Pr; T.t33 += x[4] / Pr;
    double det;
    sym3_inverse(T, A, det);
    c0 = log(x[0]) - 0.5 * log(kTwoPi * kTwoPi * kTwoPi * det);
}

// Residual (returns the scaled norm) and, if J != nullptr, the Jacobian, from
// the 35 centred moments M of g(x).
// low (optional): exact centred moments (sum w g, sum w g ut_d, sum w g |ut|^2/2)
// of the equilibrium actually used, replacing the first three orders of M in
// the residual and the Jacobian's leading terms.
template <typename MT>
__device__ __forceinline__ double assemble(const MT *M, const PointState &ps, const GasInfo &gs,
                                           const double x[5], const Sym3 &A, double R[5], double (*J)[5],
                                           const double *low = nullptr) {
#define MM(p1, p2, p3) ((double)M[midx(p1, p2, p3)])
    const double *U0 = ps.U0;
    const double hd = 0.5 * gs.delta;
    const double dl[3] = {x[1] - U0[0], x[2] - U0[1], x[3] - U0[2]};
    const double M0 = low ? low[0] : MM(0, 0, 0);
    const double Me[3] = {low ? low[1] : MM(1, 0, 0), low ? low[2] : MM(0, 1, 0), low ? low[3] : MM(0, 0, 1)};
    const double Se = low ? low[4] : 0.5 * (MM(2, 0, 0) + MM(0, 2, 0) + MM(0, 0, 2));
    const double eint = hd * x[4];
    const double dM0 = M0 - ps.rho;
    const double UMe = U0[0] * Me[0] + U0[1] * Me[1] + U0[2] * Me[2];
    R[0] = dM0;
#pragma unroll
    for (int d = 0; d < 3; ++d) R[1 + d] = fma(U0[d], dM0, Me[d]);
    R[4] = Se + UMe + ps.hU2 * dM0 + eint * M0 - ps.Eth;
    const double res = fmax(fabs(R[0]) * ps.sc_rho,
                            fmax(fmax(fabs(R[1]), fmax(fabs(R[2]), fabs(R[3]))) * ps.sc_mom, fabs(R[4]) * ps.sc_E));
    if (!J) return res;
    // Jacobian: moment combinations of v = A c = A ut - A dl
    const double Am[3][3] = {{A.t11, A.t12, A.t13}, {A.t12, A.t22, A.t23}, {A.t13, A.t23, A.t33}};
    double bt[3];
#pragma unroll
    for (int f = 0; f < 3; ++f) bt[f] = Am[f][0] * dl[0] + Am[f][1] * dl[1] + Am[f][2] * dl[2];
    double A2[3][3], bb2[3];
#pragma unroll
    for (int e1 = 0; e1 < 3; ++e1) {
#pragma unroll
        for (int e2 = 0; e2 < 3; ++e2)
            A2[e1][e2] = Am[e1][0] * Am[0][e2] + Am[e1][1] * Am[1][e2] + Am[e1][2] * Am[2][e2];
        bb2[e1] = Am[e1][0] * bt[0] + Am[e1][1] * bt[1] + Am[e1][2] * bt[2];
    }
    const double s0 = bt[0] * bt[0] + bt[1] * bt[1] + bt[2] * bt[2];
    double V[3], Vd[3][3], VE[3], W0, Wd[3], WE;
#pragma unroll
    for (int f = 0; f < 3; ++f) V[f] = Am[f][0] * Me[0] + Am[f][1] * Me[1] + Am[f][2] * Me[2] - bt[f] * M0;
    double Mij[3][3];
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int e = 0; e < 3; ++e) Mij[d][e] = M[midx((d == 0) + (e == 0), (d == 1) + (e == 1), (d == 2) + (e == 2))];
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int f = 0; f < 3; ++f)
            Vd[d][f] = Am[f][0] * Mij[d][0] + Am[f][1] * Mij[d][1] + Am[f][2] * Mij[d][2] - bt[f] * Me[d];
#pragma unroll
    for (int f = 0; f < 3; ++f) {
        double acc = 0.0;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
#pragma unroll
            for (int e = 0; e < 3; ++e)
                acc += Am[f][e] * M[midx(2 * (d == 0) + (e == 0), 2 * (d == 1) + (e == 1), 2 * (d == 2) + (e == 2))];
            acc -= bt[f] * Mij[d][d];
        }
        VE[f] = 0.5 * acc;
    }
    W0 = s0 * M0;
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        W0 -= 2.0 * bb2[e] * Me[e];
#pragma unroll
        for (int e2 = 0; e2 < 3; ++e2) W0 += A2[e][e2] * Mij[e][e2];
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        double acc = s0 * Me[d];
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            acc -= 2.0 * bb2[e] * Mij[d][e];
#pragma unroll
            for (int e2 = 0; e2 < 3; ++e2)
                acc += A2[e][e2] * M[midx((d == 0) + (e == 0) + (e2 == 0), (d == 1) + (e == 1) + (e2 == 1),
                                          (d == 2) + (e == 2) + (e2 == 2))];
        }
        Wd[d] = acc;
    }
    {
        double acc = 0.0;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            acc += s0 * Mij[d][d];
#pragma unroll
            for (int e = 0; e < 3; ++e) {
                acc -= 2.0 * bb2[e] * M[midx(2 * (d == 0) + (e == 0), 2 * (d == 1) + (e == 1), 2 * (d == 2) + (e == 2))];
#pragma unroll
                for (int e2 = 0; e2 < 3; ++e2)
                    acc += A2[e][e2] * M[midx(2 * (d == 0) + (e == 0) + (e2 == 0), 2 * (d == 1) + (e == 1) + (e2 == 1),
                                              2 * (d == 2) + (e == 2) + (e2 == 2))];
            }
        }
        WE = 0.5 * acc;
    }
    const double trA = A.t11 + A.t22 + A.t33;
    const double k2 = 0.5 / gs.Pr;
    const double ir = 1.0 / x[0];
    const double cE = ps.hU2 + eint;
    J[0][0] = M0 * ir;
#pragma unroll
    for (int d = 0; d < 3; ++d) J[1 + d][0] = fma(U0[d], M0, Me[d]) * ir;
    J[4][0] = (Se + UMe + cE * M0) * ir;
#pragma unroll
    for (int f = 0; f < 3; ++f) {
        J[0][1 + f] = V[f];
        double UV = 0.0;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            J[1 + d][1 + f] = fma(U0[d], V[f], Vd[d][f]);
            UV = fma(U0[d], Vd[d][f], UV);
        }
        J[4][1 + f] = VE[f] + UV + cE * V[f];
    }
    const double Z0 = W0 - trA * M0;
    double Zd[3], UZ = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) { Zd[d] = Wd[d] - trA * Me[d]; UZ = fma(U0[d], Zd[d], UZ); }
    const double ZE = WE - trA * Se;
    J[0][4] = k2 * Z0;
#pragma unroll
    for (int d = 0; d < 3; ++d) J[1 + d][4] = k2 * fma(U0[d], Z0, Zd[d]);
    J[4][4] = k2 * (ZE + UZ + cE * Z0) + hd * M0;
#undef MM
    return res;
}

// Newton update with step halving while rho', theta' <= 0 or T' is not SPD.
__device__ __forceinline__ bool newton_update(double J[5][5], const double R[5], double x[5], const Sym3 &B,
                                              double Pr) {
    double dx[5] = {-R[0], -R[1], -R[2], -R[3], -R[4]};
    if (!solve5(J, dx)) return false;
#pragma unroll
    for (int j = 0; j < 5; ++j)
        if (!isfinite(dx[j])) return false;
    double lam = 1.0;
    for (int h = 0; h < 60; ++h) {
        const double r0 = x[0] + lam * dx[0], t0 = x[4] + lam * dx[4];
        Sym3 Tt = B;
        Tt.t11 += t0 / Pr; Tt.t22 += t0 / Pr; Tt.t33 += t0 / Pr;
        Sym3 dummy;
        double dd;
        if (r0 > 0.0 && t0 > 0.0 && sym3_inverse(Tt, dummy, dd)) break;
        lam *= 0.5;
    }
#pragma unroll
    for (int j = 0; j < 5; ++j) x[j] = fma(lam, dx[j], x[j]);
    return true;
}

// ---- FP32-equilibrium moment correction (mixed form) ------------------------
// Error-free accumulation (Ogita, Rump & Oishi 2005, "Sum2"): TwoSum keeps
// the exact rounding error of each addition in c; the sum is s + c.
__device__ __forceinline__ void sum2(float &s, float &c, float v) {
    const float t = __fadd_rn(s, v);
    const float bp = __fsub_rn(t, s);
    const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(v, bp));
    s = t;
    c = __fadd_rn(c, e);
}

__device__ __forceinline__ float trapf(int j, int n) { return (j == 0 || j == n - 1) ? 0.5f : 1.0f; }

// packed FP32 (two IEEE operations per issue): x - y as one rounding of the
// exact difference, and sum2 on two independent (sum, error) pairs
__device__ __forceinline__ float2 qdup2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 qneg2(float2 v) { return make_float2(-v.x, -v.y); }
__device__ __forceinline__ float2 qsub2(float2 x, float2 y) { return __ffma2_rn(y, make_float2(-1.f, -1.f), x); }
__device__ __forceinline__ void qsum2x2(float2 &s, float2 &c, float2 v) {
    const float2 t = __fadd2_rn(s, v);
    const float2 bp = qsub2(t, s);
    const float2 e = __fadd2_rn(qsub2(s, qsub2(t, bp)), qsub2(v, bp));
    s = t;
    c = __fadd2_rn(c, e);
}

// add c * (sum + err) of a line pair into a plane pair, error-free up to O(eps^2)
__device__ __forceinline__ void plane_add(float &P, float &Pc, float c, float sum, float err) {
    const float ps = __fmul_rn(c, sum);
    sum2(P, Pc, ps);
    Pc = __fadd_rn(Pc, fmaf(c, sum, -ps));
    Pc = fmaf(c, err, Pc);
}

// The per-point FP32 parameters of the velocity passes, formed once per point
// (by the lane that does the point's algebra) so the passes on the whole
// warp run on the FP32 pipe only: the stage's equilibrium Eq32 (its ten
// parameters, the same conversions as the stage's own record) and the
// offsets U0_1, lo_2 - U0_2, lo_3 - U0_3 of the centred coordinates.
constexpr int QEF = 14;
__device__ __forceinline__ void point_eqf(const PointState &ps, double c0, const double x[5], const Sym3 &A,
                                          const VelGrid &vg, float ef[QEF]) {
    const double qd[10] = {c0, x[1], x[2], x[3], A.t11, A.t22, A.t33, A.t12, A.t13, A.t23};
    Eq32 e32;
    e32.load(qd);
    e32.get(ef);
    ef[10] = (float)ps.U0[0];
    ef[11] = (float)(vg.lo[1] - ps.U0[1]);
    ef[12] = (float)(vg.lo[2] - ps.U0[2]);
    ef[13] = (float)(vg.lo[0] + ((vg.n[0] - 1) / 2) * vg.h[0] - ps.U0[0]);   // centre of the first axis - U0_1
}

// Error-free FP32 pairs (s + c) for the index moments of a whole velocity
// grid: a plane's (sum, error) pairs times exact or exactly split weights
// join the pair (TwoSum, TwoProd), so the moments stay accurate to O(2^-48)
// without the FP64 pipe.
__device__ __forceinline__ void pair_add(float &s, float &c, float v, float ve) {
    const float t = __fadd_rn(s, v);
    const float bp = __fsub_rn(t, s);
    const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(v, bp));
    s = t;
    c = __fadd_rn(c, __fadd_rn(e, ve));
}
// J pair k += w * (P + Pc), w exact in FP32 (a small integer or half of one)
__device__ __forceinline__ void pair_axpy(float &s, float &c, float w, float P, float Pc) {
    const float p = __fmul_rn(w, P);
    pair_add(s, c, p, fmaf(w, Pc, fmaf(w, P, -p)));
}
// the plane j3's five plane pairs into the seven index-moment pairs
// J000 J100 J200 J010 J020 J001 J002 (Js[k], Jc[k])
__device__ __forceinline__ void plane_to_pairs(float (&Js)[7], float (&Jc)[7], float (&P)[5], float (&Pc)[5], int j3,
                                               int n3, int jc3) {
    const float c3 = (j3 == 0 || j3 == n3 - 1) ? 0.5f : 1.f, t3 = (float)(j3 - jc3);
    const float w5 = __fmul_rn(c3, t3), w6 = __fmul_rn(w5, t3);       // exact
#pragma unroll
    for (int i = 0; i < 5; ++i) pair_axpy(Js[i], Jc[i], c3, P[i], Pc[i]);
    pair_axpy(Js[5], Jc[5], w5, P[0], Pc[0]);
    pair_axpy(Js[6], Jc[6], w6, P[0], Pc[0]);
#pragma unroll
    for (int i = 0; i < 5; ++i) P[i] = Pc[i] = 0.f;
}
// sum of the seven pairs over the warp (every lane returns them)
__device__ __forceinline__ void pair_warp_sum(float (&Js)[7], float (&Jc)[7]) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int i = 0; i < 7; ++i) {
            const float s2 = __shfl_xor_sync(0xffffffffu, Js[i], o), c2 = __shfl_xor_sync(0xffffffffu, Jc[i], o);
            pair_add(Js[i], Jc[i], s2, c2);
        }
    }
}

// The error-free line sums of a velocity line without products in the
// walk: with A_k = sum_{j<=k} c g_j, B_k = sum_{m<=k} A_m, C_k = sum_{m<=k} B_m
// (error-free pair sums, taken in index order), at the line's end
//   sum_j c g_j            = A
//   sum_j (n - j) c g_j    = B
//   sum_j (n - j)^2 c g_j  = 2 C - B,
// so with jt = j - jc = K - (n - j), K = n - jc:
//   L1 = sum jt c g   = K A - B
//   L2 = sum jt^2 c g = K^2 A - (2K + 1) B + 2 C.
// The integer weights are exact in FP32 and each product joins its pair with
// its exact error, so L1 and L2 are accurate to O(2^-48) of the largest term.
__device__ __forceinline__ void pair_wadd(float &s, float &c, float w, float vs, float vc) {
    const float p = __fmul_rn(w, vs);
    pair_add(s, c, p, fmaf(w, vc, fmaf(w, vs, -p)));
}
__device__ __forceinline__ void line_sums_from_prefix(float K, float As, float Ac, float Bs, float Bc, float Cs,
                                                      float Cc, float &L1, float &C1, float &L2, float &C2) {
    L1 = 0.f; C1 = 0.f;
    pair_wadd(L1, C1, K, As, Ac);
    pair_wadd(L1, C1, -1.f, Bs, Bc);
    L2 = 0.f; C2 = 0.f;
    pair_wadd(L2, C2, __fmul_rn(K, K), As, Ac);
    pair_wadd(L2, C2, -fmaf(2.f, K, 1.f), Bs, Bc);
    pair_wadd(L2, C2, 2.f, Cs, Cc);
}

// Exact index moments J_abc = sum c g32 jt1^a jt2^b jt3^c of the stage's FP32
// equilibrium (jt = j - jc centred indices, c the trapezoid factors):
// J000 J100 J200 J010 J020 J001 J002 as (sum, error) pairs, reduced over the
// warp (every lane returns them).  Lane l takes a contiguous run of lines;
// the line sums are error-free (Sum2) sums of exact products, the lines of
// one plane (j3 = const) accumulate as (sum, error) pairs with exact
// coefficients, and the planes as error-free pairs, so s + c is accurate to
// O(2^-48) of the sums.  ef: the point's parameters (point_eqf).
__device__ __forceinline__ void correction_sums(const QPrimeArgs &a, int lane, const float *ef, const float *su1,
                                                float (&Js)[7], float (&Jc)[7]) {
    const VelGrid &vg = a.vg;
    const int n1 = vg.n[0], n2 = vg.n[1], n3 = vg.n[2];
    const int jc[3] = {(n1 - 1) / 2, (n2 - 1) / 2, (n3 - 1) / 2};
    Eq32 e32;
    e32.set(ef);
#pragma unroll
    for (int i = 0; i < 7; ++i) Js[i] = Jc[i] = 0.f;
    float P[5] = {0.f, 0.f, 0.f, 0.f, 0.f}, Pc[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    const int nl = n2 * n3, chunk = (nl + 31) / 32;
    const int l0 = min(nl, lane * chunk), l1 = min(nl, l0 + chunk);
    int j3cur = l0 < l1 ? l0 / n2 : -1;
    for (int line = l0; line < l1; ++line) {
        const int j2 = line % n2, j3 = line / n2;
        if (j3 != j3cur) { plane_to_pairs(Js, Jc, P, Pc, j3cur, n3, jc[2]); j3cur = j3; }
        const float4 *vl32 = a.vtab32 + (size_t)line * n1;
        float lin, cst;
        e32.line(vl32[0].y, vl32[0].z, lin, cst);
        float L0 = 0.f, C0 = 0.f, Bs = 0.f, Bc = 0.f, Cs = 0.f, Cc = 0.f;
        for (int j1 = 0; j1 < n1; ++j1) {
            const float g = e32.g(su1[j1], lin, cst);
            const float cg = (j1 == 0 || j1 == n1 - 1) ? __fmul_rn(0.5f, g) : g;     // exact
            sum2(L0, C0, cg);
            sum2(Bs, Bc, L0);
            Bc = __fadd_rn(Bc, C0);
            sum2(Cs, Cc, Bs);
            Cc = __fadd_rn(Cc, Bc);
        }
        float L1, C1, L2, C2;
        line_sums_from_prefix((float)(n1 - jc[0]), L0, C0, Bs, Bc, Cs, Cc, L1, C1, L2, C2);
        const float c2 = trapf(j2, n2), t2 = (float)(j2 - jc[1]);
        const float b = __fmul_rn(c2, t2), bb = __fmul_rn(b, t2);                  // exact
        plane_add(P[0], Pc[0], c2, L0, C0);
        plane_add(P[1], Pc[1], c2, L1, C1);
        plane_add(P[2], Pc[2], c2, L2, C2);
        plane_add(P[3], Pc[3], b, L0, C0);
        plane_add(P[4], Pc[4], bb, L0, C0);
    }
    if (j3cur >= 0) plane_to_pairs(Js, Jc, P, Pc, j3cur, n3, jc[2]);
    pair_warp_sum(Js, Jc);
}

// the index moments in FP64 from their pairs
__device__ __forceinline__ void pairs_to_jm(const float *Jp, double Jm[7]) {
#pragma unroll
    for (int k = 0; k < 7; ++k) Jm[k] = (double)Jp[2 * k] + (double)Jp[2 * k + 1];
}

// gamma from G gamma = T - S (one thread), with S the moments of g32 from the
// index moments Jm, T the centred moments of f itself and G from the
// solve's moments.
// S_i = sum w phi_i g32 in ut = u - U0 coordinates (u_d = uc_d + jt_d h_d) from
// the index moments J000 J100 J200 J010 J020 J001 J002.
__device__ __forceinline__ void exact_low_moments(const VelGrid &vg, const PointState &ps, const double Jm[7],
                                                  double S[5]) {
    const int jc[3] = {(vg.n[0] - 1) / 2, (vg.n[1] - 1) / 2, (vg.n[2] - 1) / 2};
    const double W = vg.h[0] * vg.h[1] * vg.h[2];
    const double o[3] = {vg.lo[0] + jc[0] * vg.h[0] - ps.U0[0], vg.lo[1] + jc[1] * vg.h[1] - ps.U0[1],
                         vg.lo[2] + jc[2] * vg.h[2] - ps.U0[2]};
    const double J1[3] = {Jm[1], Jm[3], Jm[5]}, J2[3] = {Jm[2], Jm[4], Jm[6]};
    S[0] = W * Jm[0];
    double s4 = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        S[1 + d] = W * (o[d] * Jm[0] + vg.h[d] * J1[d]);
        s4 += o[d] * o[d] * Jm[0] + 2.0 * o[d] * vg.h[d] * J1[d] + vg.h[d] * vg.h[d] * J2[d];
    }
    S[4] = 0.5 * W * s4;
}

template <typename MT>
__device__ __forceinline__ void correction_fit(const QPrimeArgs &a, const PointState &ps, const double x[5],
                                               const double Jm[7], const MT *Gsrc, double gam[5]) {
    double S[5];
    exact_low_moments(a.vg, ps, Jm, S);
    // targets: the centred moments of f, with the G equilibrium's share of
    // the energy (delta theta'/2 per unit mass) taken out of phi_4
    const double *m = ps.m;
    const double gfac = 0.5 * a.gas.delta * x[4];
    double T[5];
    T[0] = m[0];
    T[1] = m[1] - ps.U0[0] * m[0];
    T[2] = m[2] - ps.U0[1] * m[0];
    T[3] = m[3] - ps.U0[2] * m[0];
    T[4] = ps.Eth - gfac * m[0];
    // G_ij = sum w phi_i phi_j g from the solve's moments (accuracy not critical)
#define MM(p1, p2, p3) ((double)Gsrc[midx(p1, p2, p3)])
    double Gm[5][5];
    Gm[0][0] = MM(0, 0, 0);
    Gm[0][1] = MM(1, 0, 0); Gm[0][2] = MM(0, 1, 0); Gm[0][3] = MM(0, 0, 1);
    Gm[0][4] = 0.5 * (MM(2, 0, 0) + MM(0, 2, 0) + MM(0, 0, 2));
#undef MM
#pragma unroll
    for (int d = 0; d < 3; ++d) {
#pragma unroll
        for (int e = 0; e < 3; ++e)
            Gm[1 + d][1 + e] = Gsrc[midx((d == 0) + (e == 0), (d == 1) + (e == 1), (d == 2) + (e == 2))];
        double acc = 0.0;
#pragma unroll
        for (int e = 0; e < 3; ++e) acc += Gsrc[midx((d == 0) + 2 * (e == 0), (d == 1) + 2 * (e == 1), (d == 2) + 2 * (e == 2))];
        Gm[1 + d][4] = 0.5 * acc;
    }
    {
        double acc = 0.0;
#pragma unroll
        for (int e = 0; e < 3; ++e)
#pragma unroll
            for (int f = 0; f < 3; ++f)
                acc += Gsrc[midx(2 * (e == 0) + 2 * (f == 0), 2 * (e == 1) + 2 * (f == 1), 2 * (e == 2) + 2 * (f == 2))];
        Gm[4][4] = 0.25 * acc;
    }
#pragma unroll
    for (int i = 0; i < 5; ++i)
#pragma unroll
        for (int j = 0; j < i; ++j) Gm[i][j] = Gm[j][i];
    double rhs[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) rhs[i] = T[i] - S[i];
#pragma unroll
    for (int i = 0; i < 5; ++i) gam[i] = 0.0;
    if (solve5(Gm, rhs)) {
#pragma unroll
        for (int i = 0; i < 5; ++i) gam[i] = isfinite(rhs[i]) ? rhs[i] : 0.0;
    }
}

// One thread per point: the solution, the equilibrium record, the training
// log; statistics and log slots are aggregated over the warp (call from all
// 32 lanes; `valid` marks the lanes that hold a point).
__device__ __forceinline__ void point_epilogue(const QPrimeArgs &a, int p, bool valid, const PointState &ps,
                                               const double x[5], const Sym3 &A, double c0, const double gam[5],
                                               int tot, bool conv, double res) {
    const unsigned vmask = __ballot_sync(0xffffffffu, valid);
    const unsigned lmask = __ballot_sync(0xffffffffu, valid && conv && a.log != nullptr);
    const int lane = threadIdx.x & 31;
    if (a.stats) {
        const unsigned isum = __reduce_add_sync(0xffffffffu, valid ? (unsigned)tot : 0u);
        const unsigned imax = __reduce_max_sync(0xffffffffu, valid ? (unsigned)tot : 0u);
        double r = valid ? (res >= 0.0 ? res : 1.0e300) : 0.0;
        if (!(r == r)) r = 1.0e300;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r = fmax(r, __shfl_xor_sync(0xffffffffu, r, o));
        if (lane == 0 && vmask) {
            atomicAdd(&a.stats->iter_sum, (unsigned long long)isum);
            atomicAdd(&a.stats->solves, (unsigned long long)__popc(vmask));
            atomicMax(&a.stats->iter_max, (int)imax);
            atomic_max_nonneg_double(&a.stats->res_max_bits, r);
        }
    }
    unsigned long long lbase = 0;
    if (lmask) {
        if (lane == 0) lbase = atomicAdd(a.log_count, (unsigned long long)__popc(lmask));
        lbase = __shfl_sync(0xffffffffu, lbase, 0);
    }
    if (!valid) return;
    const double hd = 0.5 * a.gas.delta;
    if (a.qp) {
#pragma unroll
        for (int j = 0; j < 5; ++j) a.qp[(size_t)p * 5 + j] = x[j];
    }
    if (a.iters) a.iters[p] = tot;
    if (a.eq) {
        double *q = a.eq + (size_t)p * BGK_NEQ;
        q[0] = c0; q[1] = x[1]; q[2] = x[2]; q[3] = x[3];
        q[4] = A.t11; q[5] = A.t22; q[6] = A.t33; q[7] = A.t12; q[8] = A.t13; q[9] = A.t23;
        q[10] = 1.0 / ps.tau;
        q[11] = hd * x[4];
#pragma unroll
        for (int i = 0; i < 5; ++i) q[12 + i] = gam[i];
        q[17] = ps.U0[0]; q[18] = ps.U0[1]; q[19] = ps.U0[2];
        if (a.eq32) {
            // the FP32 values the stage kernels derive from this record, with
            // the same conversions (Eq32::load and plain roundings)
            double qr[BGK_NEQ];
#pragma unroll
            for (int i = 0; i < BGK_NEQ; ++i) qr[i] = q[i];
            Eq32 e;
            e.load(qr);
            float g[5];
#pragma unroll
            for (int i = 0; i < 5; ++i) g[i] = (float)qr[12 + i];
            float4 *r = reinterpret_cast<float4 *>(a.eq32 + (size_t)p * BGK_NEQ32);
            r[0] = make_float4(e.E0, e.V1, e.A11, (float)qr[10]);
            r[1] = make_float4(g[1], 0.5f * g[4], (float)qr[17], (float)qr[11]);
            r[2] = make_float4(e.V2, e.V3, e.A12, e.A13);
            r[3] = make_float4(e.A22, e.A23, e.A33, g[0]);
            r[4] = make_float4(g[2], g[3], (float)qr[18], (float)qr[19]);
            r[5] = make_float4(g[4], 0.f, 0.f, 0.f);
        }
    }
    if (!conv) atomicOr(a.status, BGK_DEV_NOCONV);
    if (a.log && conv) {
        const unsigned long long slot = lbase + __popc(lmask & ((1u << lane) - 1u));
        if ((long long)slot < a.log_max) {
            float *r = a.log + (size_t)slot * MLP_LOG_STRIDE;
#pragma unroll
            for (int f = 0; f < MLP_IN; ++f) r[f] = ps.feat[f];
            const double st = sqrt(ps.theta);
            r[MLP_IN + 0] = (float)(x[0] / ps.rho - 1.0);
            r[MLP_IN + 1] = (float)((x[1] - ps.U0[0]) / st);
            r[MLP_IN + 2] = (float)((x[2] - ps.U0[1]) / st);
            r[MLP_IN + 3] = (float)((x[3] - ps.U0[2]) / st);
            r[MLP_IN + 4] = (float)(x[4] / ps.theta - 1.0);
        }
    }
}

// ---- velocity-sum engines ------------------------------------------------------
// FP64: table w1 ut1^m in shared memory, FP64 walk and fold.
struct Engine64 {
    double (*tab)[5];
    __device__ void init(double (*t)[5], const VelGrid &vg, const PointState &ps, int lane) {
        tab = t;
        const double s1 = vg.lo[0] - ps.U0[0], h1 = vg.h[0];
        for (int j = lane; j < vg.n[0]; j += 32) {
            const double ut = fma((double)j, h1, s1);
            const double w = (j == 0 || j == vg.n[0] - 1) ? 0.5 * h1 : h1;
            tab[j][0] = w; tab[j][1] = w * ut; tab[j][2] = w * ut * ut;
            tab[j][3] = w * ut * ut * ut; tab[j][4] = w * ut * ut * ut * ut;
        }
        __syncwarp();
    }
    __device__ void moments(const VelGrid &vg, const PointState &ps, const double x[5], const Sym3 &A, double c0,
                            int lane, double M[35]) const {
        const int n1 = vg.n[0], n2 = vg.n[1], n3 = vg.n[2];
        const double h1 = vg.h[0], h2 = vg.h[1], h3 = vg.h[2];
        const double s1 = vg.lo[0] - ps.U0[0];
        const double dl[3] = {x[1] - ps.U0[0], x[2] - ps.U0[1], x[3] - ps.U0[2]};
        const double rho1 = exp(-A.t11 * h1 * h1);
        const double ia11 = 1.0 / A.t11, ih1 = 1.0 / h1;
#pragma unroll
        for (int i = 0; i < 35; ++i) M[i] = 0.0;
        for (int line = lane; line < n2 * n3; line += 32) {
            const int j2 = line % n2, j3 = line / n2;
            const double ut2 = fma((double)j2, h2, vg.lo[1] - ps.U0[1]);
            const double ut3 = fma((double)j3, h3, vg.lo[2] - ps.U0[2]);
            const double w23 = ((j2 == 0 || j2 == n2 - 1) ? 0.5 * h2 : h2) * ((j3 == 0 || j3 == n3 - 1) ? 0.5 * h3 : h3);
            const double c2 = ut2 - dl[1], c3 = ut3 - dl[2];
            const double lin = A.t12 * c2 + A.t13 * c3;
            const double cst = A.t22 * c2 * c2 + 2.0 * A.t23 * c2 * c3 + A.t33 * c3 * c3;
            const double jf = (-lin * ia11 + dl[0] - s1) * ih1;
            const int js = (int)rint(fmin(fmax(jf, 0.0), (double)(n1 - 1)));
            const double c1s = fma((double)js, h1, s1) - dl[0];
            const double G = exp(c0 - 0.5 * (A.t11 * c1s * c1s + 2.0 * c1s * lin + cst));
            const double D = fmin(fmax(-h1 * (A.t11 * (c1s + 0.5 * h1) + lin), -700.0), 700.0);
            const double rup = exp(D);
            const double rdn = rho1 / rup;
            double Tm[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
            int j = js, dir = 1;
            double g = G, r = rup;
            const int nup = n1 - js;
            for (int t = 0; t < n1; ++t) {
                if (t == nup) { j = js - 1; dir = -1; g = G * rdn; r = rdn * rho1; }
                const double *tb = tab[j];
#pragma unroll
                for (int q = 0; q < 5; ++q) Tm[q] = fma(g, tb[q], Tm[q]);
                g *= r;
                r *= rho1;
                j += dir;
            }
            double pu2[5], pu3[5];
            pu2[0] = w23; pu3[0] = 1.0;
#pragma unroll
            for (int q = 1; q < 5; ++q) { pu2[q] = pu2[q - 1] * ut2; pu3[q] = pu3[q - 1] * ut3; }
            // slots in midx order: (p2, p3) outer, p1 inner (a running index keeps them compile-time)
            int idx = 0;
#pragma unroll
            for (int aa = 0; aa <= 4; ++aa)
#pragma unroll
                for (int bb = 0; bb <= 4 - aa; ++bb) {
                    const double P = pu2[aa] * pu3[bb];
#pragma unroll
                    for (int mm = 0; mm <= 4 - aa - bb; ++mm, ++idx) M[idx] = fma(P, Tm[mm], M[idx]);
                }
        }
#pragma unroll
        for (int i = 0; i < 35; ++i) M[i] = warp_sum(M[i]);
    }
};

// FP32: same walk in FP32, monomials formed on the fly (no table), anchors
// from the FP32 exp2 unit; the 35 moments accumulate in FP32 per lane and
// are reduced across the warp in FP32 (every lane returns them).
struct Engine32 {
    __device__ void moments(const VelGrid &vg, const PointState &ps, const double x[5], const Sym3 &Ad, double c0d,
                            int lane, float (&Mo)[35]) const {
        const int n1 = vg.n[0], n2 = vg.n[1], n3 = vg.n[2];
        const float h1 = (float)vg.h[0];
        const float s1 = (float)(vg.lo[0] - ps.U0[0]);
        const float o2 = (float)(vg.lo[1] - ps.U0[1]), o3 = (float)(vg.lo[2] - ps.U0[2]);
        const float h2 = (float)vg.h[1], h3 = (float)vg.h[2];
        const float dl0 = (float)(x[1] - ps.U0[0]), dl1 = (float)(x[2] - ps.U0[1]), dl2 = (float)(x[3] - ps.U0[2]);
        const float A11 = (float)Ad.t11, A22 = (float)Ad.t22, A33 = (float)Ad.t33;
        const float A12 = (float)Ad.t12, A13 = (float)Ad.t13, A23 = (float)Ad.t23;
        const float c0 = (float)c0d;
        const float L2E = 1.4426950408889634f;
        const float rho1 = Eq32::ex2(-A11 * h1 * h1 * L2E);
        const float ia11 = 1.f / A11, ih1 = 1.f / h1;
        float M[35];
#pragma unroll
        for (int i = 0; i < 35; ++i) M[i] = 0.f;
        for (int line = lane; line < n2 * n3; line += 32) {
            const int j2 = line % n2, j3 = line / n2;
            const float ut2 = fmaf((float)j2, h2, o2), ut3 = fmaf((float)j3, h3, o3);
            const float w23 = ((j2 == 0 || j2 == n2 - 1) ? 0.5f * h2 : h2) * ((j3 == 0 || j3 == n3 - 1) ? 0.5f * h3 : h3) * h1;
            const float c2 = ut2 - dl1, c3 = ut3 - dl2;
            const float lin = A12 * c2 + A13 * c3;
            const float cst = A22 * c2 * c2 + 2.f * A23 * c2 * c3 + A33 * c3 * c3;
            const float jf = (-lin * ia11 + dl0 - s1) * ih1;
            const int js = (int)rintf(fminf(fmaxf(jf, 0.f), (float)(n1 - 1)));
            const float c1s = fmaf((float)js, h1, s1) - dl0;
            const float G = Eq32::ex2((c0 - 0.5f * (A11 * c1s * c1s + 2.f * c1s * lin + cst)) * L2E);
            const float D = fminf(fmaxf(-h1 * (A11 * (c1s + 0.5f * h1) + lin), -80.f), 80.f);
            const float rup = Eq32::ex2(D * L2E);
            const float rdn = rho1 / rup;
            float Tm[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
            // walk up from js, then down from js-1; ut1 advances with j
            float g = G, r = rup, ut = fmaf((float)js, h1, s1), step = h1;
            int j = js;
            const int nup = n1 - js;
            for (int t = 0; t < n1; ++t) {
                if (t == nup) { j = js - 1; step = -h1; g = G * rdn; r = rdn * rho1; ut = fmaf((float)j, h1, s1); }
                const float gw = (j == 0 || j == n1 - 1) ? 0.5f * g : g;
                const float t1 = gw * ut, t2 = t1 * ut, t3 = t2 * ut;
                Tm[0] += gw; Tm[1] += t1; Tm[2] += t2; Tm[3] += t3; Tm[4] = fmaf(t3, ut, Tm[4]);
                g *= r;
                r *= rho1;
                ut += step;
                j += (step > 0.f) ? 1 : -1;
            }
            float pu2[5], pu3[5];
            pu2[0] = w23; pu3[0] = 1.f;
#pragma unroll
            for (int q = 1; q < 5; ++q) { pu2[q] = pu2[q - 1] * ut2; pu3[q] = pu3[q - 1] * ut3; }
            int idx = 0;
#pragma unroll
            for (int aa = 0; aa <= 4; ++aa)
#pragma unroll
                for (int bb = 0; bb <= 4 - aa; ++bb) {
                    const float P = pu2[aa] * pu3[bb];
#pragma unroll
                    for (int mm = 0; mm <= 4 - aa - bb; ++mm, ++idx) M[idx] = fmaf(P, Tm[mm], M[idx]);
                }
        }
        // the lane partials carry FP32 rounding already; the tree sum in FP32
        // keeps the reduction off the FP64 pipe
#pragma unroll
        for (int i = 0; i < 35; ++i) Mo[i] = warp_sumf(M[i]);
    }
};

// One pass that serves both the Newton residual and the correction: the
// stage's exact FP32 equilibrium g32 (Eq32) is evaluated once per velocity
// and accumulated (a) into the error-free index moments J000..J002 (as in
// correction_sums), which give the exact discrete moments of g32 and so the
// residual of the equilibrium actually used, and (b) into plain FP32 line
// sums T_m = sum_j1 w1 g32 ut1^m, m <= 4, folded per line into the 35 centred
// moments (as in Engine32) for the Jacobian and the correction's G.  All on
// the FP32 pipe; every lane returns the moments M (FP32 sums) and the index
// moment pairs.  tab: the warp's [2 n1] first-axis table, filled here for
// the point: node j1's (c1, c1, ut, ut) and (ut^3, ut^3, w1, w1), c1 = u1 -
// V1, ut = u1 - U0_1, w1 the trapezoid factor -- what the walk would
// otherwise form per velocity, as pairs for its packed instructions.
__device__ __forceinline__ void fused_pass(const QPrimeArgs &a, int lane, const float *ef, const float *su1,
                                           float4 *tab, float (&M)[35], float (&Js)[7], float (&Jc)[7]) {
    const VelGrid &vg = a.vg;
    const int n1 = vg.n[0], n2 = vg.n[1], n3 = vg.n[2];
    const int jc[3] = {(n1 - 1) / 2, (n2 - 1) / 2, (n3 - 1) / 2};
    Eq32 e32;
    e32.set(ef);
    const float U0x = ef[10], o2 = ef[11], o3 = ef[12], dlt = ef[13];
    const float h1 = (float)vg.h[0], h2 = (float)vg.h[1], h3 = (float)vg.h[2];
    const float K = (float)(n1 - jc[0]);
    __syncwarp();
    for (int j = lane; j < n1; j += 32) {
        const float u1 = su1[j];
        const float c1 = __fsub_rn(u1, e32.V1);
        const float ut = __fsub_rn(u1, U0x), ut3 = ut * ut * ut;
        const float w1 = (j == 0 || j == n1 - 1) ? 0.5f : 1.f;
        tab[2 * j] = make_float4(c1, c1, ut, ut);
        tab[2 * j + 1] = make_float4(ut3, ut3, w1, w1);
    }
    __syncwarp();
#pragma unroll
    for (int i = 0; i < 35; ++i) M[i] = 0.f;
#pragma unroll
    for (int i = 0; i < 7; ++i) Js[i] = Jc[i] = 0.f;
    float P[5] = {0.f, 0.f, 0.f, 0.f, 0.f}, Pc[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    const int nl = n2 * n3, chunk = (nl + 31) / 32;
    const int l0 = min(nl, lane * chunk), l1 = min(nl, l0 + chunk);
    int j3cur = l0 < l1 ? l0 / n2 : -1;
    // the end of a line: its error-free sums into the plane pairs (in line
    // order, flushing finished planes) and its Jacobian sums into the moments
    auto end_line = [&](int line, float L0, float C0, float L1, float C1, float L2, float C2, float T3, float T4) {
        // the Jacobian line sums of order <= 2 from the exact index sums:
        // ut = u1 - U0_1 = dlt + h1 jt on the grid
        const float S0 = __fadd_rn(L0, C0), S1 = __fadd_rn(L1, C1), S2 = __fadd_rn(L2, C2);
        const float Tm[5] = {S0, fmaf(h1, S1, dlt * S0), fmaf(h1 * h1, S2, fmaf(2.f * dlt * h1, S1, dlt * dlt * S0)),
                             T3, T4};
        const int j2 = line % n2, j3 = line / n2;
        if (j3 != j3cur) { plane_to_pairs(Js, Jc, P, Pc, j3cur, n3, jc[2]); j3cur = j3; }
        const float c2 = trapf(j2, n2), jt2 = (float)(j2 - jc[1]);
        const float b = __fmul_rn(c2, jt2), bb = __fmul_rn(b, jt2);                  // exact
        plane_add(P[0], Pc[0], c2, L0, C0);
        plane_add(P[1], Pc[1], c2, L1, C1);
        plane_add(P[2], Pc[2], c2, L2, C2);
        plane_add(P[3], Pc[3], b, L0, C0);
        plane_add(P[4], Pc[4], bb, L0, C0);
        // fold the line sums into the 35 centred moments
        const float ut2 = fmaf((float)j2, h2, o2), ut3 = fmaf((float)j3, h3, o3);
        const float w23 = ((j2 == 0 || j2 == n2 - 1) ? 0.5f * h2 : h2) * ((j3 == 0 || j3 == n3 - 1) ? 0.5f * h3 : h3) * h1;
        float pu2[5], pu3[5];
        pu2[0] = w23; pu3[0] = 1.f;
#pragma unroll
        for (int q = 1; q < 5; ++q) { pu2[q] = pu2[q - 1] * ut2; pu3[q] = pu3[q - 1] * ut3; }
        int idx = 0;
#pragma unroll
        for (int aa = 0; aa <= 4; ++aa)
#pragma unroll
            for (int bb2 = 0; bb2 <= 4 - aa; ++bb2) {
                const float Pp = pu2[aa] * pu3[bb2];
#pragma unroll
                for (int mm = 0; mm <= 4 - aa - bb2; ++mm, ++idx) M[idx] = fmaf(Pp, Tm[mm], M[idx]);
            }
    };
    // two lines of the lane's run at a time on packed FP32: they share u1,
    // the equilibrium's point parameters and the weights, so every operation
    // of a line's walk is the scalar one (the equilibrium values bit for bit
    // those of the stage's Eq32), paired with the other line's
    for (int line = l0; line < l1; line += 2) {
        const bool two = line + 1 < l1;
        const float4 *vl32 = a.vtab32 + (size_t)line * n1;
        float linA, cstA, linB = 0.f, cstB = 0.f;
        e32.line(vl32[0].y, vl32[0].z, linA, cstA);
        if (two) e32.line(vl32[n1].y, vl32[n1].z, linB, cstB);
        const float2 lin2 = make_float2(linA, linB), cst2 = make_float2(cstA, cstB);
        const float2 A11 = qdup2(e32.A11), E0 = qdup2(e32.E0);
        // error-free prefix sums A (= L0), B, C of the line (line_sums_from_prefix)
        float2 L0 = qdup2(0.f), C0 = L0, Bs = L0, Bc = L0, Cs = L0, Cc = L0;
        float2 T3 = L0, T4 = L0;
        // unrolled by two: one velocity's table loads, exponent and
        // equilibrium overlap the previous one's dependent sum chains
#pragma unroll 2
        for (int j1 = 0; j1 < n1; ++j1) {
            const float4 ta = tab[2 * j1], tb = tab[2 * j1 + 1];
            const float2 c1 = make_float2(ta.x, ta.y);
            const float2 ex = __ffma2_rn(c1, __ffma2_rn(A11, c1, lin2), cst2);
            const float2 g = __fmul2_rn(E0, make_float2(Eq32::ex2(ex.x), Eq32::ex2(ex.y)));
            const float2 cg = __fmul2_rn(make_float2(tb.z, tb.w), g);                     // exact
            qsum2x2(L0, C0, cg);
            qsum2x2(Bs, Bc, L0);
            Bc = __fadd2_rn(Bc, C0);
            qsum2x2(Cs, Cc, Bs);
            Cc = __fadd2_rn(Cc, Bc);
            // Jacobian line sums of order 3 and 4 (plain FP32)
            const float2 t3 = __fmul2_rn(cg, make_float2(tb.x, tb.y));
            T3 = __fadd2_rn(T3, t3);
            T4 = __ffma2_rn(t3, make_float2(ta.z, ta.w), T4);
        }
        {
            float L1, C1, L2, C2;
            line_sums_from_prefix(K, L0.x, C0.x, Bs.x, Bc.x, Cs.x, Cc.x, L1, C1, L2, C2);
            end_line(line, L0.x, C0.x, L1, C1, L2, C2, T3.x, T4.x);
        }
        if (two) {
            float L1, C1, L2, C2;
            line_sums_from_prefix(K, L0.y, C0.y, Bs.y, Bc.y, Cs.y, Cc.y, L1, C1, L2, C2);
            end_line(line + 1, L0.y, C0.y, L1, C1, L2, C2, T3.y, T4.y);
        }
    }
    if (j3cur >= 0) plane_to_pairs(Js, Jc, P, Pc, j3cur, n3, jc[2]);
    pair_warp_sum(Js, Jc);
#pragma unroll
    for (int i = 0; i < 35; ++i) M[i] = warp_sumf(M[i]);
}

// One block solves a batch of QB points.  The velocity sums run one warp per
// point (QW warps take the batch's points in turn); the per-point algebra
// (prologue, Newton step, correction fit, epilogue) runs one lane of warp 0
// per point, so the FP64 work of a point issues once rather than on 32 lanes.
constexpr int QB = 32;
constexpr int QW = 8;

template <bool F32>
struct QPShared {
    using MT = typename std::conditional<F32, float, double>::type;
    PointState ps[QB];
    double x[QB][5];
    double A[QB][6];
    double c0[QB];
    double res[QB];
    MT M[QB][35];            // the velocity pass's moments (FP32 sums with the FP32 engine)
    float Jp[QB][14];        // exact index moments of g32 as (sum, error) pairs
    float ef[QB][QEF];       // the FP32 pass parameters (point_eqf)
    int it[QB], tot[QB];
    int conv[QB], from_guess[QB], active[QB];
    int fused[QB];           // next evaluation by the fused pass (FP32-sum engine)
    int exact[QB];           // Jm holds the exact moments of the last evaluation
    int any_active;
};

__device__ __forceinline__ Sym3 load_sym3(const double *t) { return Sym3{t[0], t[1], t[2], t[3], t[4], t[5]}; }

template <bool F32>
__global__ void __launch_bounds__(QB * QW, 2) k_qprime(QPrimeArgs a) {
    __shared__ QPShared<F32> S;
    __shared__ float su1[BGK_MAXV];          // u1 of the first-axis velocity nodes (the same on every line)
    extern __shared__ double dyn_tab[];      // FP64 engine: [QW][n1][5] tables w1 ut1^m; FP32: [QW][2 n1] float4
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int p0 = blockIdx.x * QB;
    const int nb = min(QB, a.P - p0);
    const double tol = F32 ? a.tol32 : a.tol;
    const double Pr = a.gas.Pr;
    for (int j = threadIdx.x; j < a.vg.n[0]; j += blockDim.x) su1[j] = __ldg(a.vtab32 + j).x;
    // -- prologue: one lane per point
    if (wib == 0 && lane < nb) point_prologue(a, p0 + lane, S.ps[lane]);
    __syncthreads();
    // -- starting points: one warp per point (the network runs on the warp)
    for (int i = wib; i < nb; i += QW) {
        double x[5];
        bool left;
        const bool fg = initial_guess(a, p0 + i, lane, S.ps[i], x, left);
        if (lane == 0) {
#pragma unroll
            for (int j = 0; j < 5; ++j) S.x[i][j] = x[j];
            S.from_guess[i] = fg;
            S.it[i] = 0; S.tot[i] = 0; S.conv[i] = 0; S.active[i] = 1;
            S.res[i] = 1.0e300;
            // from the learned guess the first evaluation is expected to be the
            // last: the fused pass gives its residual and its correction at once
            S.fused[i] = F32 && fg && a.mixed && a.eq;
            S.exact[i] = 0;
            if (left && a.fallbacks) atomicAdd(a.fallbacks, 1ull);
        }
    }
    __syncthreads();
    // -- Newton iterations over the batch until every point has stopped
    for (;;) {
        if (wib == 0 && lane < nb && S.active[lane]) {
            Sym3 A;
            double c0;
            equilibrium_params(S.ps[lane], Pr, S.x[lane], A, c0);
            S.A[lane][0] = A.t11; S.A[lane][1] = A.t22; S.A[lane][2] = A.t33;
            S.A[lane][3] = A.t12; S.A[lane][4] = A.t13; S.A[lane][5] = A.t23;
            S.c0[lane] = c0;
            if (F32 && S.fused[lane]) point_eqf(S.ps[lane], c0, S.x[lane], A, a.vg, S.ef[lane]);
        }
        __syncthreads();
        for (int i = wib; i < nb; i += QW) {
            if (!S.active[i]) continue;
            if constexpr (F32) {
                float M[35];
                if (S.fused[i]) {
                    float Js[7], Jc[7];
                    fused_pass(a, lane, S.ef[i], su1, reinterpret_cast<float4 *>(dyn_tab) + (size_t)wib * 2 * a.vg.n[0], M,
                               Js, Jc);
                    if (lane == 0) {
#pragma unroll
                        for (int j = 0; j < 7; ++j) { S.Jp[i][2 * j] = Js[j]; S.Jp[i][2 * j + 1] = Jc[j]; }
                    }
                } else {
                    double x[5];
#pragma unroll
                    for (int j = 0; j < 5; ++j) x[j] = S.x[i][j];
                    Engine32 e32;
                    e32.moments(a.vg, S.ps[i], x, load_sym3(S.A[i]), S.c0[i], lane, M);
                }
                if (lane == 0) {
#pragma unroll
                    for (int j = 0; j < 35; ++j) S.M[i][j] = M[j];
                    S.exact[i] = S.fused[i];
                }
            } else {
                double x[5], M[35];
#pragma unroll
                for (int j = 0; j < 5; ++j) x[j] = S.x[i][j];
                Engine64 e64;
                e64.init(reinterpret_cast<double (*)[5]>(dyn_tab + (size_t)wib * a.vg.n[0] * 5), a.vg, S.ps[i], lane);
                e64.moments(a.vg, S.ps[i], x, load_sym3(S.A[i]), S.c0[i], lane, M);
                if (lane == 0) {
#pragma unroll
                    for (int j = 0; j < 35; ++j) S.M[i][j] = M[j];
                    S.exact[i] = 0;
                }
            }
            __syncwarp();
        }
        __syncthreads();
        if (wib == 0) {
            bool act = false;
            if (lane < nb && S.active[lane]) {
                const PointState &ps = S.ps[lane];
                double x[5];
#pragma unroll
                for (int j = 0; j < 5; ++j) x[j] = S.x[lane][j];
                const Sym3 A = load_sym3(S.A[lane]);
                double R[5], J[5][5], low[5];
                const bool ex = S.exact[lane];
                if (ex) {
                    double Jm[7];
                    pairs_to_jm(S.Jp[lane], Jm);
                    exact_low_moments(a.vg, ps, Jm, low);
                }
                // the residual first; the Jacobian only if an update may follow
                const double res = assemble(S.M[lane], ps, a.gas, x, A, R, nullptr, ex ? low : nullptr);
                // The exact residual of the mixed form measures the stage's FP32
                // equilibrium, whose mean is U' rounded to FP32: its spacing
                // 2^-23 |U'| bounds the reachable momentum residual
                // |R_rhoU| / (rho sqrt(theta')).  At high speed (|U'| of tens of
                // thermal speeds) that floor exceeds tol32, so the momentum rows
                // stop at a few spacings -- the linear term of the exact moment
                // correction that follows absorbs such a mean shift to first
                // order -- while density and energy converge to tol32.
                bool done = res <= tol;
                if (F32 && !done) {
                    const double um = fmax(fabs(x[1]), fmax(fabs(x[2]), fabs(x[3])));
                    const double tol_mom = fmax(tol, 8.0 * 0x1p-24 * um / sqrt(fmax(x[4], 1e-300)));
                    done = fabs(R[0]) * ps.sc_rho <= tol && fabs(R[4]) * ps.sc_E <= tol &&
                           fmax(fabs(R[1]), fmax(fabs(R[2]), fabs(R[3]))) * ps.sc_mom <= tol_mom;
                }
                if (!done) assemble(S.M[lane], ps, a.gas, x, A, R, J, ex ? low : nullptr);
                S.res[lane] = res;
                int it = S.it[lane];
                act = true;
                if (done) {
                    S.conv[lane] = 1;
                    act = false;
                } else if (S.from_guess[lane] && ((it == 0 && !(res <= 1e-3)) || it >= a.max_iter || !(res == res))) {
                    // the learned guess is judged by its own residual: one that is
                    // not small (or a solve that runs out of updates from it)
                    // restarts from q
                    x[0] = ps.rho; x[1] = ps.U0[0]; x[2] = ps.U0[1]; x[3] = ps.U0[2]; x[4] = ps.theta;
                    S.from_guess[lane] = 0;
                    S.fused[lane] = 0;                   // from q, an update is expected first
                    it = 0;
                    if (a.fallbacks) atomicAdd(a.fallbacks, 1ull);
                } else if (it >= a.max_iter || !(res == res) || !newton_update(J, R, x, ps.B, Pr)) {
                    act = false;
                } else {
                    ++it;
                    ++S.tot[lane];
                    // after an update the next evaluation is usually the last
                    S.fused[lane] = F32 && a.mixed && a.eq;
                }
                S.it[lane] = it;
#pragma unroll
                for (int j = 0; j < 5; ++j) S.x[lane][j] = x[j];
                S.active[lane] = act;
            }
            const bool any = __any_sync(0xffffffffu, act);
            if (lane == 0) S.any_active = any;
        }
        __syncthreads();
        if (!S.any_active) break;
    }
    // -- mixed form: exact moments of the stage's FP32 equilibrium, one warp per point
    const bool fit = a.mixed && a.eq;
    if (fit) {
        // the parameters of the equilibrium the stage will use (the final x)
        if (wib == 0 && lane < nb && !S.exact[lane])
            point_eqf(S.ps[lane], S.c0[lane], S.x[lane], load_sym3(S.A[lane]), a.vg, S.ef[lane]);
        __syncthreads();
        for (int i = wib; i < nb; i += QW) {
            if (S.exact[i]) continue;            // the fused pass measured them already
            float Js[7], Jc[7];
            correction_sums(a, lane, S.ef[i], su1, Js, Jc);
            if (lane == 0) {
#pragma unroll
                for (int j = 0; j < 7; ++j) { S.Jp[i][2 * j] = Js[j]; S.Jp[i][2 * j + 1] = Jc[j]; }
            }
        }
        __syncthreads();
    }
    // -- correction fit and epilogue: one lane per point
    if (wib == 0) {
        const bool valid = lane < nb;
        const int i = valid ? lane : 0;
        double x[5], gam[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
        for (int j = 0; j < 5; ++j) x[j] = S.x[i][j];
        if (fit && valid) {
            double Jm[7];
            pairs_to_jm(S.Jp[i], Jm);
            correction_fit(a, S.ps[i], x, Jm, S.M[i], gam);
        }
        point_epilogue(a, p0 + i, valid, S.ps[i], x, load_sym3(S.A[i]), S.c0[i], gam, S.tot[i], S.conv[i] != 0,
                       S.res[i]);
    }
}

}  // namespace

// ---- tensor variant of the discrete ES equilibrium (monatomic) -------------
// The discrete Gaussian g = exp(b . phi(ut)), ut = u - U (the point's
// velocity), phi = (1, ut, ut_i ut_j (i <= j)), whose discrete moments are
// (rho, 0, rho T) with T = theta/Pr I + (1 - 1/Pr) Pi/rho the ES target: the
// paper's remark that ES-BGK may need a solve of marginally higher dimension
// (section "Numerical method").  Newton on the ten natural parameters b from
// the d+2 solution's record (written by k_qprime): R = sum w phi g - t and
// J = sum w phi phi^T g are the centred moments of order <= 4 that the
// velocity-sum engines already produce.  One warp per point; the 10x10
// algebra on lane 0.  The mixed form then fits its FP32-equilibrium
// correction as k_qprime does.

// exponents (p1, p2, p3) of phi_a: 1, ut1, ut2, ut3, ut1^2, ut2^2, ut3^2, ut1 ut2, ut1 ut3, ut2 ut3
__device__ __forceinline__ void tensor_phi(int a, int &p1, int &p2, int &p3) {
    const int e1[10] = {0, 1, 0, 0, 2, 0, 0, 1, 1, 0};
    const int e2[10] = {0, 0, 1, 0, 0, 2, 0, 1, 0, 1};
    const int e3[10] = {0, 0, 0, 1, 0, 0, 2, 0, 1, 1};
    p1 = e1[a]; p2 = e2[a]; p3 = e3[a];
}

// Gaussian elimination with partial pivoting, N x N, compile-time indices.
template <int N>
__device__ __forceinline__ bool solve_n(double (&J)[N][N], double (&r)[N]) {
#pragma unroll
    for (int c = 0; c < N; ++c) {
        int piv = c;
        double best = fabs(J[c][c]);
#pragma unroll
        for (int i = c + 1; i < N; ++i) {
            const double v = fabs(J[i][c]);
            if (v > best) { best = v; piv = i; }
        }
        if (!(best > 0.0)) return false;
#pragma unroll
        for (int i = c + 1; i < N; ++i) {
            if (i == piv) {
#pragma unroll
                for (int j = 0; j < N; ++j) {
                    const double t = J[c][j]; J[c][j] = J[i][j]; J[i][j] = t;
                }
                const double t = r[c]; r[c] = r[i]; r[i] = t;
            }
        }
        const double inv = 1.0 / J[c][c];
#pragma unroll
        for (int i = c + 1; i < N; ++i) {
            const double l = J[i][c] * inv;
#pragma unroll
            for (int j = c + 1; j < N; ++j) J[i][j] = fma(-l, J[c][j], J[i][j]);
            r[i] = fma(-l, r[c], r[i]);
        }
    }
#pragma unroll
    for (int c = N - 1; c >= 0; --c) {
        double sacc = r[c];
#pragma unroll
        for (int j = c + 1; j < N; ++j) sacc = fma(-J[c][j], r[j], sacc);
        r[c] = sacc / J[c][c];
    }
    return true;
}

// (c0, U', A) <-> natural parameters b in the frame ut = u - U0
__device__ __forceinline__ void tensor_to_b(const PointState &ps, double c0, const double U[3], const Sym3 &A,
                                            double b[10]) {
    const double ur[3] = {U[0] - ps.U0[0], U[1] - ps.U0[1], U[2] - ps.U0[2]};
    const double au[3] = {A.t11 * ur[0] + A.t12 * ur[1] + A.t13 * ur[2], A.t12 * ur[0] + A.t22 * ur[1] + A.t23 * ur[2],
                          A.t13 * ur[0] + A.t23 * ur[1] + A.t33 * ur[2]};
    b[0] = c0 - 0.5 * (ur[0] * au[0] + ur[1] * au[1] + ur[2] * au[2]);
    b[1] = au[0]; b[2] = au[1]; b[3] = au[2];
    b[4] = -0.5 * A.t11; b[5] = -0.5 * A.t22; b[6] = -0.5 * A.t33;
    b[7] = -A.t12; b[8] = -A.t13; b[9] = -A.t23;
}

__device__ __forceinline__ bool tensor_from_b(const PointState &ps, const double b[10], double &c0, double U[3],
                                              Sym3 &A) {
    A = Sym3{-2.0 * b[4], -2.0 * b[5], -2.0 * b[6], -b[7], -b[8], -b[9]};
    Sym3 T;
    double det;
    if (!sym3_inverse(A, T, det)) return false;
    const double ur[3] = {T.t11 * b[1] + T.t12 * b[2] + T.t13 * b[3], T.t12 * b[1] + T.t22 * b[2] + T.t23 * b[3],
                          T.t13 * b[1] + T.t23 * b[2] + T.t33 * b[3]};
    c0 = b[0] + 0.5 * (b[1] * ur[0] + b[2] * ur[1] + b[3] * ur[2]);
    U[0] = ps.U0[0] + ur[0]; U[1] = ps.U0[1] + ur[1]; U[2] = ps.U0[2] + ur[2];
    return true;
}

struct TensorShared {
    PointState ps[QW];
    double par[QW][10];       // c0, U'(3), A(6)
    double M[QW][35];
    int go[QW];
};

template <bool F32>
__global__ void __launch_bounds__(QW * 32) k_qprime_tensor(QPrimeArgs a) {
    __shared__ TensorShared S;
    __shared__ float su1[BGK_MAXV];
    extern __shared__ double dyn_tab[];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int j = threadIdx.x; j < a.vg.n[0]; j += blockDim.x) su1[j] = __ldg(a.vtab32 + j).x;
    __syncthreads();
    const int p = blockIdx.x * QW + wib;
    if (p >= a.P) return;                       // whole warps; no block barrier follows
    PointState &ps = S.ps[wib];
    if (lane == 0) point_prologue(a, p, ps);
    __syncwarp();
    // targets in the frame ut = u - U0, and the start: the d+2 solution's record
    double t[10], b[10];
    double res = 1.0e300;
    int it = 0;
    bool conv = false;
    if (lane == 0) {
        const double ip = 1.0 / a.gas.Pr;
        t[0] = ps.m[0];
        t[1] = ps.m[1] - ps.U0[0] * ps.m[0];
        t[2] = ps.m[2] - ps.U0[1] * ps.m[0];
        t[3] = ps.m[3] - ps.U0[2] * ps.m[0];
        const double rt = ps.rho * ps.theta * ip;
        t[4] = fma(ps.rho, ps.B.t11, rt); t[5] = fma(ps.rho, ps.B.t22, rt); t[6] = fma(ps.rho, ps.B.t33, rt);
        t[7] = ps.rho * ps.B.t12; t[8] = ps.rho * ps.B.t13; t[9] = ps.rho * ps.B.t23;
        const double *q = a.eq + (size_t)p * BGK_NEQ;
#pragma unroll
        for (int j = 0; j < 10; ++j) S.par[wib][j] = q[j];
        const Sym3 A0{q[4], q[5], q[6], q[7], q[8], q[9]};
        const double U[3] = {q[1], q[2], q[3]};
        tensor_to_b(ps, q[0], U, A0, b);
    }
    __syncwarp();
    Engine64 e64;
    if (!F32) e64.init(reinterpret_cast<double (*)[5]>(dyn_tab + (size_t)wib * a.vg.n[0] * 5), a.vg, ps, lane);
    for (;;) {
        const double *pr = S.par[wib];
        const Sym3 A{pr[4], pr[5], pr[6], pr[7], pr[8], pr[9]};
        const double x[5] = {0.0, pr[1], pr[2], pr[3], 0.0};
        double M[35];
        if (F32) {
            Engine32 e32;
            float Mf[35];
            e32.moments(a.vg, ps, x, A, pr[0], lane, Mf);
#pragma unroll
            for (int j = 0; j < 35; ++j) M[j] = Mf[j];
        } else {
            e64.moments(a.vg, ps, x, A, pr[0], lane, M);
        }
        if (lane == 0) {
#pragma unroll
            for (int j = 0; j < 35; ++j) S.M[wib][j] = M[j];
            double R[10], J[10][10];
#pragma unroll
            for (int i = 0; i < 10; ++i) {
                int a1, a2, a3;
                tensor_phi(i, a1, a2, a3);
                R[i] = M[midx(a1, a2, a3)] - t[i];
#pragma unroll
                for (int j = 0; j < 10; ++j) {
                    int b1, b2, b3;
                    tensor_phi(j, b1, b2, b3);
                    J[i][j] = M[midx(a1 + b1, a2 + b2, a3 + b3)];
                }
            }
            const double sq = 1.0 / (ps.rho * ps.theta);
            double r_mom = 0.0, r_oth = fabs(R[0]) * ps.sc_rho;
#pragma unroll
            for (int i = 1; i < 4; ++i) r_mom = fmax(r_mom, fabs(R[i]) * ps.sc_mom);
#pragma unroll
            for (int i = 4; i < 10; ++i) r_oth = fmax(r_oth, fabs(R[i]) * sq);
            res = fmax(r_mom, r_oth);
            const double tol = F32 ? a.tol32 : a.tol;
            double tol_mom = tol;
            if (F32) {        // the momentum rows' FP32 floor, as in k_qprime
                const double um = fmax(fabs(pr[1]), fmax(fabs(pr[2]), fabs(pr[3])));
                tol_mom = fmax(tol, 8.0 * 0x1p-24 * um * sqrt(fmax(A.t11 + A.t22 + A.t33, 0.0) / 3.0));
            }
            bool go = false;
            if (r_oth <= tol && r_mom <= tol_mom) {
                conv = true;
            } else if (it < a.max_iter && res == res) {
                double db[10];
#pragma unroll
                for (int i = 0; i < 10; ++i) db[i] = -R[i];
                if (solve_n<10>(J, db)) {
                    double lam = 1.0, bt[10], c0n = 0.0, Un[3];
                    Sym3 An;
                    bool ok = false;
                    for (int h = 0; h < 60 && !ok; ++h) {
#pragma unroll
                        for (int i = 0; i < 10; ++i) bt[i] = fma(lam, db[i], b[i]);
                        ok = tensor_from_b(ps, bt, c0n, Un, An);
                        if (!ok) lam *= 0.5;
                    }
                    if (ok) {
#pragma unroll
                        for (int i = 0; i < 10; ++i) b[i] = bt[i];
                        S.par[wib][0] = c0n;
                        S.par[wib][1] = Un[0]; S.par[wib][2] = Un[1]; S.par[wib][3] = Un[2];
                        S.par[wib][4] = An.t11; S.par[wib][5] = An.t22; S.par[wib][6] = An.t33;
                        S.par[wib][7] = An.t12; S.par[wib][8] = An.t13; S.par[wib][9] = An.t23;
                        ++it;
                        go = true;
                    }
                }
            }
            S.go[wib] = go;
        }
        __syncwarp();
        if (!S.go[wib]) break;
    }
    // the converged Gaussian: x = (rho', U', theta' = tr T'/3) for the record and qp
    const double *pr = S.par[wib];
    const Sym3 A{pr[4], pr[5], pr[6], pr[7], pr[8], pr[9]};
    Sym3 T;
    double detA;
    sym3_inverse(A, T, detA);
    double x[5];
    x[0] = exp(pr[0]) * sqrt(kTwoPi * kTwoPi * kTwoPi / detA);
    x[1] = pr[1]; x[2] = pr[2]; x[3] = pr[3];
    x[4] = (T.t11 + T.t22 + T.t33) / 3.0;
    double gam[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    if (a.mixed && a.eq) {
        float ef[QEF], Js[7], Jc[7], Jp[14];
        point_eqf(ps, pr[0], x, A, a.vg, ef);
        correction_sums(a, lane, ef, su1, Js, Jc);
#pragma unroll
        for (int j = 0; j < 7; ++j) { Jp[2 * j] = Js[j]; Jp[2 * j + 1] = Jc[j]; }
        double Jm[7];
        pairs_to_jm(Jp, Jm);
        if (lane == 0) correction_fit(a, ps, x, Jm, S.M[wib], gam);
    }
    const int tot = __shfl_sync(0xffffffffu, it, 0);
    const bool cv = __shfl_sync(0xffffffffu, (int)conv, 0) != 0;
    const double rs = __shfl_sync(0xffffffffu, res, 0);
    point_epilogue(a, p, lane == 0, ps, x, A, pr[0], gam, tot, cv, rs);
}

cudaError_t launch_qprime_tensor(const QPrimeArgs &a, bool fp32_sums, cudaStream_t s) {
    const unsigned grid = (unsigned)((a.P + QW - 1) / QW);
    if (fp32_sums) {
        k_qprime_tensor<true><<<grid, QW * 32, 0, s>>>(a);
    } else {
        const size_t dyn = (size_t)QW * a.vg.n[0] * 5 * sizeof(double);
        k_qprime_tensor<false><<<grid, QW * 32, dyn, s>>>(a);
    }
    return cudaGetLastError();
}

// raise a kernel's dynamic shared-memory limit to `bytes` once per device
template <typename K>
cudaError_t allow_dyn_smem(K kernel, SmemLimit &lim, size_t bytes) {
    size_t *attr = lim.slot();
    if (!attr) return cudaErrorInvalidDevice;
    if (bytes > *attr) {
        const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (e != cudaSuccess) return e;
        *attr = bytes;
    }
    return cudaSuccess;
}

cudaError_t launch_qprime(const QPrimeArgs &a, bool fp32_sums, cudaStream_t s) {
    const unsigned grid = (unsigned)((a.P + QB - 1) / QB);
    if (fp32_sums) {
        static SmemLimit lim32;
        const size_t dyn = (size_t)QW * 2 * a.vg.n[0] * sizeof(float4);      // the fused pass's tables
        const cudaError_t e = allow_dyn_smem(k_qprime<true>, lim32, dyn);
        if (e != cudaSuccess) return e;
        k_qprime<true><<<grid, QB * QW, dyn, s>>>(a);
    } else {
        static SmemLimit lim64;
        const size_t dyn = (size_t)QW * a.vg.n[0] * 5 * sizeof(double);
        const cudaError_t e = allow_dyn_smem(k_qprime<false>, lim64, dyn);
        if (e != cudaSuccess) return e;
        k_qprime<false><<<grid, QB * QW, dyn, s>>>(a);
    }
    return cudaGetLastError();
}
