// FP64 kernels of one explicit Runge--Kutta stage of the Boltzmann--ES-BGK
// residual (Dzanic & Martinelli, arXiv 2312.06567, section "Methodology").
//
//   moments   raw velocity moments of f, partial over velocity blocks
//   qprime    reduce the partials to Q, build the ES tensor and tau, and solve
//             the discrete compatibility condition for Q' by Newton's method
//             (one warp per point, lanes split the velocity sums)
//   stage     FR divergence (nodal derivative + upwind interface jump lifted
//             with the DG correction function) + BGK source + Shu--Osher
//             combination, with the moment partials of the output in the
//             epilogue (one thread per solution point, looping over a block
//             of velocities so the point's equilibrium record stays in
//             registers)
#include "bgk_internal.cuh"

namespace {

constexpr double kTwoPi = 6.283185307179586476925286766559;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ void atomic_max_nonneg_double(unsigned long long *addr, double v) {
    if (!(v >= 0.0)) v = 1.0e300;      // NaN / negative: record as "huge"
    atomicMax(addr, (unsigned long long)__double_as_longlong(v));
}

// ---------------------------------------------------------------------------
// Raw moments (section "Governing equations": Q = int psi f, Pi = int f c c):
// slots 0: w F, 1..3: w u_d F, 4..6: w u_d^2 F, 7: w u1u2 F, 8: w u1u3 F,
// 9: w u2u3 F, 10: w G.  One thread per point, one velocity block per blockIdx.y.
__global__ void __launch_bounds__(256) k_moments_f64(MomentArgs64 a) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.P) return;
    const int vb = blockIdx.y;
    const int k0 = vb * a.Kblk;
    const int k1 = min(a.Nu, k0 + a.Kblk);
    double m[BGK_NMOM];
#pragma unroll
    for (int j = 0; j < BGK_NMOM; ++j) m[j] = 0.0;
    for (int k = k0; k < k1; ++k) {
        const double *v = a.vtab + (size_t)k * BGK_VTAB;
        const double u1 = __ldg(v + 0), u2 = __ldg(v + 1), u3 = __ldg(v + 2), w = __ldg(v + 3);
        const double wF = w * __ldg(a.f + (size_t)k * a.P + p);
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
        if (a.C == 2) m[10] = fma(w, __ldg(a.f + ((size_t)a.Nu + k) * a.P + p), m[10]);
    }
#pragma unroll
    for (int j = 0; j < BGK_NMOM; ++j) a.part[((size_t)vb * BGK_NMOM + j) * a.P + p] = m[j];
}

__global__ void k_reduce_moments(const double *part, int n_vblk, int P, double *m_out) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    for (int j = 0; j < BGK_NMOM; ++j) {
        double s = 0.0;
        for (int vb = 0; vb < n_vblk; ++vb) s += part[((size_t)vb * BGK_NMOM + j) * P + p];
        m_out[(size_t)p * BGK_NMOM + j] = s;
    }
}

// ---------------------------------------------------------------------------
// Q' solve.  Unknowns x = (rho', U', theta'); T'(theta') = theta'/Pr I + B with
// B = (1 - 1/Pr) Pi/rho of f; g = rho'/sqrt(det(2 pi T')) exp(-c^T T'^-1 c / 2),
// c = u - U'.  Residual R = sum_k w_k psi~_k g_k - Q with
// psi~ = (1, u, |u|^2/2 + delta theta'/2); analytic Jacobian:
//   dg/drho' = g/rho',  dg/dU' = g A c,  dg/dtheta' = g (|A c|^2 - tr A)/(2 Pr).
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

__global__ void __launch_bounds__(256) k_qprime_f64(QPrimeArgs a) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= a.P) return;                 // whole warps exit together
    const int p = warp;

    // 1. reduce the moment partials of this point
    double m[BGK_NMOM];
#pragma unroll
    for (int j = 0; j < BGK_NMOM; ++j) m[j] = 0.0;
    for (int vb = lane; vb < a.n_vblk; vb += 32) {
#pragma unroll
        for (int j = 0; j < BGK_NMOM; ++j) m[j] += a.part[((size_t)vb * BGK_NMOM + j) * a.P + p];
    }
#pragma unroll
    for (int j = 0; j < BGK_NMOM; ++j) m[j] = warp_sum(m[j]);

    // 2. macroscopic state, ES tensor, collision time
    const GasInfo &gs = a.gas;
    const double rho = m[0];
    const double U1 = m[1] / rho, U2 = m[2] / rho, U3 = m[3] / rho;
    const double E = 0.5 * (m[4] + m[5] + m[6]) + m[10];
    const double pres = (gs.gamma - 1.0) * (E - 0.5 * rho * (U1 * U1 + U2 * U2 + U3 * U3));
    const double theta = pres / rho;
    const double es = (1.0 - 1.0 / gs.Pr) / rho;
    Sym3 B;
    B.t11 = es * (m[4] - rho * U1 * U1);
    B.t22 = es * (m[5] - rho * U2 * U2);
    B.t33 = es * (m[6] - rho * U3 * U3);
    B.t12 = es * (m[7] - rho * U1 * U2);
    B.t13 = es * (m[8] - rho * U1 * U3);
    B.t23 = es * (m[9] - rho * U2 * U3);
    double mu = gs.mu_ref;
    if (gs.theta_S >= 0.0) {
        const double r = theta / gs.theta_ref;
        mu = gs.mu_ref * r * sqrt(r) * (gs.theta_ref + gs.theta_S) / (theta + gs.theta_S);
    }
    const double tau = mu / (gs.Pr * pres);
    const double sc_rho = 1.0 / rho, sc_mom = 1.0 / (rho * sqrt(theta)), sc_E = 1.0 / fabs(E);
    const double Q[5] = {rho, m[1], m[2], m[3], E};

    // 3. Newton
    double x[5];
    if (a.guess) {
#pragma unroll
        for (int j = 0; j < 5; ++j) x[j] = a.guess[(size_t)p * 5 + j];
    } else {
        x[0] = rho; x[1] = U1; x[2] = U2; x[3] = U3; x[4] = theta;
    }
    const double hd = 0.5 * gs.delta;
    int it = 0;
    bool conv = false;
    double res = 1.0e300;
    Sym3 A;
    double c0 = 0.0;
    for (;;) {
        Sym3 T = B;
        T.t11 += x[4] / gs.Pr; T.t22 += x[4] / gs.Pr; T.t33 += x[4] / gs.Pr;
        double det;
        sym3_inverse(T, A, det);
        c0 = log(x[0]) - 0.5 * log(kTwoPi * kTwoPi * kTwoPi * det);
        // lane-strided velocity sums: g, g u, g e | g v, g u v, g e v | g vv, g u vv, g e vv
        double s_g = 0, s_gu[3] = {0, 0, 0}, s_ge = 0;
        double s_gv[3] = {0, 0, 0}, s_guv[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, s_gev[3] = {0, 0, 0};
        double s_gvv = 0, s_guvv[3] = {0, 0, 0}, s_gevv = 0;
        for (int k = lane; k < a.Nu; k += 32) {
            const double *vt = a.vtab + (size_t)k * BGK_VTAB;
            const double u[3] = {__ldg(vt + 0), __ldg(vt + 1), __ldg(vt + 2)};
            const double w = __ldg(vt + 3), e = __ldg(vt + 4);
            const double c1 = u[0] - x[1], c2 = u[1] - x[2], c3 = u[2] - x[3];
            const double v[3] = {A.t11 * c1 + A.t12 * c2 + A.t13 * c3,
                                 A.t12 * c1 + A.t22 * c2 + A.t23 * c3,
                                 A.t13 * c1 + A.t23 * c2 + A.t33 * c3};
            const double qf = c1 * v[0] + c2 * v[1] + c3 * v[2];
            const double g = w * exp(c0 - 0.5 * qf);
            const double vv = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
            const double ge = g * e, gvv = g * vv;
            s_g += g;
            s_ge += ge;
            s_gvv += gvv;
            s_gevv = fma(ge, vv, s_gevv);
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const double gu = g * u[d];
                s_gu[d] += gu;
                s_gv[d] = fma(g, v[d], s_gv[d]);
                s_gev[d] = fma(ge, v[d], s_gev[d]);
                s_guvv[d] = fma(gu, vv, s_guvv[d]);
#pragma unroll
                for (int f = 0; f < 3; ++f) s_guv[d][f] = fma(gu, v[f], s_guv[d][f]);
            }
        }
        s_g = warp_sum(s_g); s_ge = warp_sum(s_ge); s_gvv = warp_sum(s_gvv); s_gevv = warp_sum(s_gevv);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            s_gu[d] = warp_sum(s_gu[d]); s_gv[d] = warp_sum(s_gv[d]);
            s_gev[d] = warp_sum(s_gev[d]); s_guvv[d] = warp_sum(s_guvv[d]);
#pragma unroll
            for (int f = 0; f < 3; ++f) s_guv[d][f] = warp_sum(s_guv[d][f]);
        }
        const double eint = hd * x[4];                       // delta theta' / 2
        double R[5] = {s_g - Q[0], s_gu[0] - Q[1], s_gu[1] - Q[2], s_gu[2] - Q[3],
                       s_ge + eint * s_g - Q[4]};
        res = fmax(fabs(R[0]) * sc_rho,
                   fmax(fmax(fabs(R[1]), fmax(fabs(R[2]), fabs(R[3]))) * sc_mom, fabs(R[4]) * sc_E));
        if (res <= a.tol) { conv = true; break; }
        if (it >= a.max_iter || !(res == res)) break;
        const double trA = A.t11 + A.t22 + A.t33;
        const double k2 = 0.5 / gs.Pr;
        double J[5][5];
        const double ir = 1.0 / x[0];
        J[0][0] = s_g * ir;
        J[4][0] = (s_ge + eint * s_g) * ir;
#pragma unroll
        for (int d = 0; d < 3; ++d) J[1 + d][0] = s_gu[d] * ir;
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            J[0][1 + f] = s_gv[f];
#pragma unroll
            for (int d = 0; d < 3; ++d) J[1 + d][1 + f] = s_guv[d][f];
            J[4][1 + f] = s_gev[f] + eint * s_gv[f];
        }
        J[0][4] = k2 * (s_gvv - trA * s_g);
#pragma unroll
        for (int d = 0; d < 3; ++d) J[1 + d][4] = k2 * (s_guvv[d] - trA * s_gu[d]);
        J[4][4] = k2 * ((s_gevv - trA * s_ge) + eint * (s_gvv - trA * s_g)) + hd * s_g;
        double dx[5] = {-R[0], -R[1], -R[2], -R[3], -R[4]};
        if (!solve5(J, dx)) break;
        bool finite = true;
#pragma unroll
        for (int j = 0; j < 5; ++j) finite = finite && isfinite(dx[j]);
        if (!finite) break;
        double lam = 1.0;
        for (int h = 0; h < 60; ++h) {
            const double r0 = x[0] + lam * dx[0], t0 = x[4] + lam * dx[4];
            Sym3 Tt = B;
            Tt.t11 += t0 / gs.Pr; Tt.t22 += t0 / gs.Pr; Tt.t33 += t0 / gs.Pr;
            Sym3 dummy;
            double dd;
            if (r0 > 0.0 && t0 > 0.0 && sym3_inverse(Tt, dummy, dd)) break;
            lam *= 0.5;
        }
#pragma unroll
        for (int j = 0; j < 5; ++j) x[j] = fma(lam, dx[j], x[j]);
        ++it;
    }

    if (lane == 0) {
        if (a.qp) {
#pragma unroll
            for (int j = 0; j < 5; ++j) a.qp[(size_t)p * 5 + j] = x[j];
        }
        if (a.iters) a.iters[p] = it;
        if (a.eq) {
            double *q = a.eq + (size_t)p * BGK_NEQ;
            q[0] = c0; q[1] = x[1]; q[2] = x[2]; q[3] = x[3];
            q[4] = A.t11; q[5] = A.t22; q[6] = A.t33; q[7] = A.t12; q[8] = A.t13; q[9] = A.t23;
            q[10] = 1.0 / tau;
            q[11] = hd * x[4];
        }
        if (!conv) atomicOr(a.status, BGK_DEV_NOCONV);
        if (a.stats) {
            atomicAdd(&a.stats->iter_sum, (unsigned long long)it);
            atomicAdd(&a.stats->solves, 1ull);
            atomicMax(&a.stats->iter_max, it);
            atomic_max_nonneg_double(&a.stats->res_max_bits, res);
        }
    }
}

// ---------------------------------------------------------------------------
// Fused stage.  Per point (e, s) and velocity k, along each reference
// direction d the 1-D FR derivative of the line through s is
//   u_d sum_j D[i][j] f_j + u_d (f^+ - f^-) dg(xi_i)
// where the jump is taken only at the inflow face (the upwind flux makes the
// outflow jump zero): for u_d > 0 the left face (f^- = sum lm f, f^+ the
// left neighbour's right trace, dg = g_L'), for u_d < 0 the right face
// (f^- = sum lp f, f^+ the right neighbour's left trace, dg = g_R').
// div = sum_d (2/h_d) (...).  R = -div + (g' - f)/tau.
template <int Q, int C>
__global__ void __launch_bounds__(256) k_stage_f64(StageArgs<double> a) {
    constexpr int NS = Q * Q * Q;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.P) return;
    const int vb = blockIdx.y;
    const int k0 = vb * a.Kblk;
    const int k1 = min(a.Nu, k0 + a.Kblk);
    const int e = p / NS, s = p - e * NS;
    const int id[3] = {s % Q, (s / Q) % Q, s / (Q * Q)};
    const int stride[3] = {1, Q, Q * Q};
    const int n1 = a.mesh.n[0], n2 = a.mesh.n[1], n3 = a.mesh.n[2];
    const int ec[3] = {e % n1, (e / n1) % n2, e / (n1 * n2)};
    const int estr[3] = {1, n1, n1 * n2};
    const int nn[3] = {n1, n2, n3};
    int eL[3], eR[3], base[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        eL[d] = ec[d] > 0 ? e - estr[d] : (a.mesh.periodic[d] ? e + (nn[d] - 1) * estr[d] : -1);
        eR[d] = ec[d] < nn[d] - 1 ? e + estr[d] : (a.mesh.periodic[d] ? e - (nn[d] - 1) * estr[d] : -1);
        base[d] = s - id[d] * stride[d];
    }
    const double *q = a.eq + (size_t)p * BGK_NEQ;
    const double c0 = q[0], V1 = q[1], V2 = q[2], V3 = q[3];
    const double A11 = q[4], A22 = q[5], A33 = q[6], A12 = q[7], A13 = q[8], A23 = q[9];
    const double itau = q[10], gfac = q[11];
    double m[BGK_NMOM];
#pragma unroll
    for (int j = 0; j < BGK_NMOM; ++j) m[j] = 0.0;
    const size_t slab = (size_t)a.P;

    for (int k = k0; k < k1; ++k) {
        const double *vt = a.vtab + (size_t)k * BGK_VTAB;
        const double u[3] = {__ldg(vt + 0), __ldg(vt + 1), __ldg(vt + 2)};
        const double w = __ldg(vt + 3);
        const double c1 = u[0] - V1, c2 = u[1] - V2, c3 = u[2] - V3;
        const double qf = 0.5 * (A11 * c1 * c1 + A22 * c2 * c2 + A33 * c3 * c3) +
                          (A12 * c1 * c2 + A13 * c1 * c3 + A23 * c2 * c3);
        const double g = exp(c0 - qf);
        double outv[C];
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const double *fs = a.f_s + ((size_t)c * a.Nu + k) * slab;
            const double fself = __ldg(fs + p);
            double div = 0.0;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const double ud = u[d];
                const double *own = fs + (size_t)e * NS + base[d];
                double line[Q];
#pragma unroll
                for (int j = 0; j < Q; ++j) line[j] = __ldg(own + j * stride[d]);
                double dfd = 0.0;
#pragma unroll
                for (int j = 0; j < Q; ++j) dfd = fma(a.fr.D[id[d]][j], line[j], dfd);
                double corr = 0.0;
                if (ud != 0.0) {
                    const bool left = ud > 0.0;
                    const int en = left ? eL[d] : eR[d];
                    double fm = 0.0, fp = 0.0;
#pragma unroll
                    for (int j = 0; j < Q; ++j) fm = fma(left ? a.fr.lm[j] : a.fr.lp[j], line[j], fm);
                    if (en >= 0) {
                        const double *nb = fs + (size_t)en * NS + base[d];
#pragma unroll
                        for (int j = 0; j < Q; ++j)
                            fp = fma(left ? a.fr.lp[j] : a.fr.lm[j], __ldg(nb + j * stride[d]), fp);
                    } else {
                        const int face = 2 * d + (left ? 0 : 1);
                        fp = __ldg(a.bcval + ((size_t)face * C + c) * a.Nu + k);
                    }
                    corr = (fp - fm) * (left ? a.fr.dgL[id[d]] : a.fr.dgR[id[d]]);
                }
                div = fma(a.mesh.two_over_h[d] * ud, dfd + corr, div);
            }
            const double eqv = (c == 0) ? g : gfac * g;
            const double R = fma(eqv - fself, itau, -div);
            double out = fma(a.c, R, a.b * fself);
            if (a.a != 0.0) out = fma(a.a, __ldg(a.f_n + ((size_t)c * a.Nu + k) * slab + p), out);
            a.f_out[((size_t)c * a.Nu + k) * slab + p] = out;
            outv[c] = out;
        }
        if (a.part) {
            const double wF = w * outv[0];
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
            if (C == 2) m[10] = fma(w, outv[C - 1], m[10]);
        }
    }
    if (a.part) {
#pragma unroll
        for (int j = 0; j < BGK_NMOM; ++j) a.part[((size_t)vb * BGK_NMOM + j) * a.P + p] = m[j];
    }
}

__global__ void k_maxwellian_f64(double *f, const double *qin, const double *vtab, int Nu, int P,
                                 int C, double delta) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)Nu * P) return;
    const int k = (int)(i / P), p = (int)(i - (size_t)k * P);
    const double *q = qin + (size_t)p * 5;
    const double rho = q[0], th = q[4];
    const double *vt = vtab + (size_t)k * BGK_VTAB;
    const double c1 = vt[0] - q[1], c2 = vt[1] - q[2], c3 = vt[2] - q[3];
    const double F = rho / (kTwoPi * th * sqrt(kTwoPi * th)) *
                     exp(-(c1 * c1 + c2 * c2 + c3 * c3) / (2.0 * th));
    f[(size_t)k * P + p] = F;
    if (C == 2) f[((size_t)Nu + k) * P + p] = 0.5 * delta * th * F;
}

}  // namespace

cudaError_t launch_moments_f64(const MomentArgs64 &a, int n_vblk, cudaStream_t s) {
    dim3 grid((a.P + 255) / 256, n_vblk);
    k_moments_f64<<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_reduce_moments(const double *part, int n_vblk, int P, double *m_out,
                                  cudaStream_t s) {
    k_reduce_moments<<<(P + 255) / 256, 256, 0, s>>>(part, n_vblk, P, m_out);
    return cudaGetLastError();
}

cudaError_t launch_qprime_f64(const QPrimeArgs &a, cudaStream_t s) {
    const long long threads = (long long)a.P * 32;
    k_qprime_f64<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}

template <int Q>
static cudaError_t stage_q(const StageArgs<double> &a, int C, dim3 grid, cudaStream_t s) {
    if (C == 1) k_stage_f64<Q, 1><<<grid, 256, 0, s>>>(a);
    else k_stage_f64<Q, 2><<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_stage_f64(const StageArgs<double> &a, int C, int n_vblk, cudaStream_t s) {
    dim3 grid((a.P + 255) / 256, n_vblk);
    switch (a.fr.q) {
        case 2: return stage_q<2>(a, C, grid, s);
        case 3: return stage_q<3>(a, C, grid, s);
        case 4: return stage_q<4>(a, C, grid, s);
        case 5: return stage_q<5>(a, C, grid, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_maxwellian_f64(double *f, const double *q, const double *vtab, int Nu, int P,
                                  int C, double delta, cudaStream_t s) {
    const size_t n = (size_t)Nu * P;
    k_maxwellian_f64<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(f, q, vtab, Nu, P, C, delta);
    return cudaGetLastError();
}
