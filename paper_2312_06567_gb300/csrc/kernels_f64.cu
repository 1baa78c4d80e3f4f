// FP64 kernels of one explicit Runge--Kutta stage of the Boltzmann--ES-BGK
// residual (Dzanic & Martinelli, arXiv 2312.06567, section "Methodology").
//
//   moments   raw velocity moments of f, partial over velocity blocks
//   (the Q' solve is in kernels_qprime.cu)
//   stage     FR divergence (nodal derivative + upwind interface jump lifted
//             with the DG correction function) + BGK source + Shu--Osher
//             combination, with the moment partials of the output in the
//             epilogue (one thread per solution point, looping over a block
//             of velocity lines so the point's equilibrium record stays in
//             registers)
#include "bgk_internal.cuh"

namespace {

constexpr double kTwoPi = 6.283185307179586476925286766559;

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

// Discrete entropy of the F component, partial over velocity blocks
// (section "Numerical method": the discrete-velocity BGK step obeys a
// discrete H-theorem): part[vb][p] = sum_{k in block vb} w_k F ln F in FP64;
// a non-positive F has no entropy and is counted in *nonpos instead.
template <typename T>
__global__ void __launch_bounds__(256) k_entropy_partial(const T *f, const double *vtab, int Nu, int P, int Kblk,
                                                         double *part, unsigned int *nonpos) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const int vb = blockIdx.y;
    const int k0 = vb * Kblk, k1 = min(Nu, k0 + Kblk);
    double h = 0.0;
    unsigned int bad = 0;
    for (int k = k0; k < k1; ++k) {
        const double F = (double)f[(size_t)k * P + p];
        if (F > 0.0) h = fma(__ldg(vtab + (size_t)k * BGK_VTAB + 3) * F, log(F), h);
        else ++bad;
    }
    part[(size_t)vb * P + p] = h;
    if (bad) atomicAdd(nonpos, bad);
}

__global__ void k_reduce_entropy(const double *part, int n_vblk, int P, double *h_out) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    double s = 0.0;
    for (int vb = 0; vb < n_vblk; ++vb) s += part[(size_t)vb * P + p];
    h_out[p] = s;
}

__global__ void k_sum_partials(const double *part, int n_vblk, int P, double *out) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    for (int j = 0; j < BGK_NMOM; ++j) {
        double s = 0.0;
        for (int vb = 0; vb < n_vblk; ++vb) s += part[((size_t)vb * BGK_NMOM + j) * P + p];
        out[(size_t)j * P + p] = s;
    }
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
// Fused stage.  Along each reference direction d the 1-D FR derivative at
// node i of the line through the thread's node is
//   u_d [ sum_j D_ij f_j + (f^+ - f^-) dg(xi_i) ]
// with the jump only at the inflow face (upwind: the outflow jump is zero).
// With f^- = sum_j l_j f_j this is u_d [ sum_j Dt_ij f_j + dg_i f^+ ] where
// Dt = D - dg (x) l is the derivative with the inflow trace folded in:
// Dt_L = D - g_L' (x) l(-1) when u_d > 0, Dt_R = D - g_R' (x) l(+1) when
// u_d < 0 (either when u_d = 0, whose contribution vanishes).  f^+ is the
// neighbour's trace at the shared face (l(+1) of the left neighbour, l(-1)
// of the right one) or the Dirichlet exterior value.
// div = sum_d (2/h_d) u_d [...],  R = -div + (g' - f)/tau.
// g' = exp(c0 - c^T A c / 2) is advanced along each first-axis velocity line
// by the ratio recurrence (exact exp at the line start and wherever the
// exponent is below -650, where the recurrence would underflow).
// The block holds EB whole elements; their values for the current velocity
// are staged in shared memory (double buffered, one barrier per velocity).
//
// Curvilinear elements (CURV): the transformed flux Ft_d = a_d f with
// a_d = u . S^d at each node (S^d = J grad xi_d), per direction and line
//   dFt/dxi(xi_i) = sum_j D_ij Ft_j + J_R g_R'(xi_i) + J_L g_L'(xi_i),
//   J_R = F^I_R - sum_j l_j(+1) Ft_j,   F^I_R = A_R (A_R > 0 ? f^-_R : f^+_R),
//   J_L = -F^I_L,out - sum_j l_j(-1) Ft_j,  F^I_L,out = -A_L (-A_L > 0 ? f^-_L : f^+_L),
// A = u . S_face at the line's flux nodes (face vectors oriented +xi_d), and
// div = (1/J) sum_d dFt_d/dxi.  Both faces contribute (the trace of a f is
// not A times the trace of f).  The element's own flux values are staged in
// shared memory beside f.  Boundary faces: Dirichlet (prescribed exterior
// Maxwellian), diffuse wall (rho_w times the wall Maxwellian), closed (no flux).
template <int Q, int C, bool CURV>
__global__ void __launch_bounds__(256) k_stage_f64(StageArgs<double> a) {
    constexpr int NS = Q * Q * Q;
    constexpr int EB = 256 / NS;
    constexpr int NT = EB * NS;
    __shared__ double sf[2][C][NT];
    __shared__ double sFt[CURV ? 2 : 1][CURV ? C : 1][CURV ? 3 : 1][CURV ? NT : 1];
    __shared__ double sD[2][Q][Q];        // Dt_L, Dt_R (CURV: D, unused)
    __shared__ double sdg[2][Q];          // g_L', g_R'
    __shared__ double sl[2][Q];           // neighbour trace weights: l(+1) for left inflow, l(-1) for right
    const int tid = threadIdx.x;
    if (tid < Q * Q) {
        const int i = tid / Q, j = tid % Q;
        if (CURV) {
            sD[0][i][j] = a.fr.D[i][j];
            sD[1][i][j] = a.fr.D[i][j];
        } else {
            sD[0][i][j] = a.fr.D[i][j] - a.fr.dgL[i] * a.fr.lm[j];
            sD[1][i][j] = a.fr.D[i][j] - a.fr.dgR[i] * a.fr.lp[j];
        }
    }
    if (tid < Q) {
        sdg[0][tid] = a.fr.dgL[tid]; sdg[1][tid] = a.fr.dgR[tid];
        sl[0][tid] = a.fr.lp[tid];   sl[1][tid] = a.fr.lm[tid];
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
    // curvilinear: the node's metric vectors, 1/J and the face vectors of the
    // flux nodes on its three lines (faces 2d and 2d + 1)
    double Sm[CURV ? 3 : 1][3], invJ = 0.0, Fv[CURV ? 6 : 1][3];
    if constexpr (CURV) {
#pragma unroll
        for (int d = 0; d < 3; ++d)
#pragma unroll
            for (int c = 0; c < 3; ++c) Sm[d][c] = 0.0;
#pragma unroll
        for (int fc = 0; fc < 6; ++fc) Fv[fc][0] = Fv[fc][1] = Fv[fc][2] = 0.0;
        if (active) {
            const double *g = a.geo + (size_t)p * BGK_NGEO;
#pragma unroll
            for (int d = 0; d < 3; ++d)
#pragma unroll
                for (int c = 0; c < 3; ++c) Sm[d][c] = g[3 * d + c];
            invJ = g[9];
            const int fpi[3] = {id[1] + Q * id[2], id[0] + Q * id[2], id[0] + Q * id[1]};
#pragma unroll
            for (int fc = 0; fc < 6; ++fc) {
                const double *v = a.fvec + (((size_t)e * 6 + fc) * Q * Q + fpi[fc / 2]) * 3;
                Fv[fc][0] = v[0]; Fv[fc][1] = v[1]; Fv[fc][2] = v[2];
            }
        }
    }
    double c0 = 0, V1 = 0, V2 = 0, V3 = 0, A11 = 1, A22 = 1, A33 = 1, A12 = 0, A13 = 0, A23 = 0;
    double itau = 0, gfac = 0;
    if (active) {
        const double *q = a.eq + (size_t)p * BGK_NEQ;
        c0 = q[0]; V1 = q[1]; V2 = q[2]; V3 = q[3];
        A11 = q[4]; A22 = q[5]; A33 = q[6]; A12 = q[7]; A13 = q[8]; A23 = q[9];
        itau = q[10]; gfac = q[11];
    }
    const double h1 = a.vg.h[0];
    const double ah = -0.5 * A11 * h1 * h1;              // q(j) = q0 + j D0 + ah j (j - 1)
    const double rho1 = exp(2.0 * ah);
    const int vn1 = a.vg.n[0];
    const double ab = a.a + a.b;
    double m[BGK_NMOM];
#pragma unroll
    for (int j = 0; j < BGK_NMOM; ++j) m[j] = 0.0;
    const size_t slab = (size_t)a.P;
    __syncthreads();

    int buf = 0;
    for (int kl = k0; kl < k1; kl += vn1) {           // one first-axis velocity line
        const double *vl = a.vtab + (size_t)kl * BGK_VTAB;
        const double u2 = __ldg(vl + 1), u3 = __ldg(vl + 2);
        const double sc2 = a.mesh.two_over_h[1] * u2, sc3 = a.mesh.two_over_h[2] * u3;
        const double c1_0 = __ldg(vl + 0) - V1, c2 = u2 - V2, c3 = u3 - V3;
        const double lin = A12 * c2 + A13 * c3;
        const double cst = A22 * c2 * c2 + 2.0 * A23 * c2 * c3 + A33 * c3 * c3;
        const double q0 = c0 - 0.5 * (A11 * c1_0 * c1_0 + 2.0 * c1_0 * lin + cst);
        const double D0 = -h1 * (A11 * (c1_0 + 0.5 * h1) + lin);
        const float q0f = (float)q0, D0f = (float)D0, ahf = (float)ah;
        double g = 0.0, r = 0.0;
        bool rec = false;
        double T0 = 0, T1 = 0, T2 = 0, TG = 0;
        for (int j1 = 0; j1 < vn1; ++j1) {
            const int k = kl + j1;
            const double *vt = a.vtab + (size_t)k * BGK_VTAB;
            double fself[C];
            double ad[3] = {0.0, 0.0, 0.0};
            if (active) {
                if constexpr (CURV) {
                    const double uu[3] = {__ldg(vt + 0), u2, u3};
#pragma unroll
                    for (int d = 0; d < 3; ++d) ad[d] = fma(uu[0], Sm[d][0], fma(uu[1], Sm[d][1], uu[2] * Sm[d][2]));
                }
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    fself[c] = __ldg(a.f_s + ((size_t)c * a.Nu + k) * slab + p);
                    sf[buf][c][tid] = fself[c];
                    if constexpr (CURV) {
#pragma unroll
                        for (int d = 0; d < 3; ++d) sFt[buf][c][d][tid] = ad[d] * fself[c];
                    }
                }
            }
            // equilibrium value at this velocity
            const float qf = q0f + (float)j1 * (D0f + ahf * (float)(j1 - 1));
            if (qf < -650.0f) {
                g = exp(q0 + j1 * (D0 + ah * (j1 - 1)));
                rec = false;
            } else if (!rec) {
                g = exp(q0 + j1 * (D0 + ah * (j1 - 1)));
                r = exp(fmin(D0 + 2.0 * ah * j1, 700.0));
                rec = true;
            }
            __syncthreads();
            if (active) {
                const double u[3] = {__ldg(vt + 0), u2, u3};
                const double sc[3] = {__ldg(vt + 7), sc2, sc3};       // (2/h_d) u_d
                double outv[C];
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    const double *fs = a.f_s + ((size_t)c * a.Nu + k) * slab;
                    const double *sfc = sf[buf][c];
                    double div = 0.0;
                    if constexpr (CURV) {
#pragma unroll
                        for (int d = 0; d < 3; ++d) {
                            const double *own = sfc + le * NS + base[d];
                            const double *ownF = sFt[buf][c][d] + le * NS + base[d];
                            double dF = 0.0, trL = 0.0, trR = 0.0, fmL = 0.0, fmR = 0.0;
#pragma unroll
                            for (int j = 0; j < Q; ++j) {
                                const double Fj = ownF[j * stride[d]], fj = own[j * stride[d]];
                                dF = fma(sD[0][id[d]][j], Fj, dF);
                                trL = fma(sl[1][j], Fj, trL);        // sl[1] = l(-1)
                                trR = fma(sl[0][j], Fj, trR);        // sl[0] = l(+1)
                                fmL = fma(sl[1][j], fj, fmL);
                                fmR = fma(sl[0][j], fj, fmR);
                            }
                            const double AL = fma(u[0], Fv[2 * d][0], fma(u[1], Fv[2 * d][1], u[2] * Fv[2 * d][2]));
                            const double AR = fma(u[0], Fv[2 * d + 1][0], fma(u[1], Fv[2 * d + 1][1], u[2] * Fv[2 * d + 1][2]));
                            double FI[2];                          // outward common flux, left and right
#pragma unroll
                            for (int side = 0; side < 2; ++side) {
                                const double un = side ? AR : -AL;
                                const double fm = side ? fmR : fmL;
                                const int en = en_[d][side];
                                const int kind = a.mesh.face_kind[2 * d + side];
                                if (en < 0 && kind == BGK_FK_CLOSED) { FI[side] = 0.0; continue; }
                                if (un > 0.0) { FI[side] = un * fm; continue; }
                                double fp = 0.0;
                                // the neighbour's trace on the shared face: l(+1) of the left one, l(-1) of the right
                                if (en >= e0 && en < e0 + EB) {
                                    const double *nb = sfc + (en - e0) * NS + base[d];
#pragma unroll
                                    for (int j = 0; j < Q; ++j) fp = fma(sl[side][j], nb[j * stride[d]], fp);
                                } else if (en >= 0) {
                                    const double *nb = fs + (size_t)en * NS + base[d];
#pragma unroll
                                    for (int j = 0; j < Q; ++j) fp = fma(sl[side][j], __ldg(nb + j * stride[d]), fp);
                                } else {
                                    fp = __ldg(a.bcval + ((size_t)(2 * d + side) * C + c) * a.Nu + k);
                                    if (kind == BGK_FK_DIFFUSE) {
                                        const int fpi = d == 0 ? id[1] + Q * id[2] : (d == 1 ? id[0] + Q * id[2] : id[0] + Q * id[1]);
                                        fp *= __ldg(a.rho_w + ((size_t)e * 6 + 2 * d + side) * Q * Q + fpi);
                                    }
                                }
                                FI[side] = un * fp;
                            }
                            const double JR = FI[1] - trR, JL = -FI[0] - trL;
                            div += fma(JR, sdg[1][id[d]], fma(JL, sdg[0][id[d]], dF));
                        }
                        div *= invJ;
                    } else {
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        const int side = u[d] > 0.0 ? 0 : 1;
                        const double *own = sfc + le * NS + base[d];
                        double t = 0.0;
#pragma unroll
                        for (int j = 0; j < Q; ++j) t = fma(sD[side][id[d]][j], own[j * stride[d]], t);
                        const int en = side ? en_[d][1] : en_[d][0];
                        double fp = 0.0;
                        if (en >= e0 && en < e0 + EB) {
                            const double *nb = sfc + (en - e0) * NS + base[d];
#pragma unroll
                            for (int j = 0; j < Q; ++j) fp = fma(sl[side][j], nb[j * stride[d]], fp);
                        } else if (en >= 0) {
                            const double *nb = fs + (size_t)en * NS + base[d];
#pragma unroll
                            for (int j = 0; j < Q; ++j) fp = fma(sl[side][j], __ldg(nb + j * stride[d]), fp);
                        } else if (a.mesh.specular[2 * d + side]) {
                            // the element's own trace on this face at the mirrored velocity
                            const double *mr = a.f_s + ((size_t)c * a.Nu + mirror_velocity(k, d, a.vg.n)) * slab +
                                               (size_t)e * NS + base[d];
#pragma unroll
                            for (int j = 0; j < Q; ++j) fp = fma(sl[1 - side][j], __ldg(mr + j * stride[d]), fp);
                        } else {
                            fp = __ldg(a.bcval + ((size_t)(2 * d + side) * C + c) * a.Nu + k);
                        }
                        t = fma(sdg[side][id[d]], fp, t);
                        div = fma(sc[d], t, div);
                    }
                    }
                    const double eqv = (c == 0) ? g : gfac * g;
                    const double R = fma(eqv - fself[c], itau, -div);
                    // (a + b) f + a (f^n - f) + c R keeps a + b = 1 exact for SSP-RK3
                    double out = ab == 1.0 ? fself[c] : ab * fself[c];
                    if (a.a != 0.0)
                        out = fma(a.a, __ldg(a.f_n + ((size_t)c * a.Nu + k) * slab + p) - fself[c], out);
                    out = fma(a.c, R, out);
                    a.f_out[((size_t)c * a.Nu + k) * slab + p] = out;
                    outv[c] = out;
                }
                T0 = fma(__ldg(vt + 3), outv[0], T0);
                T1 = fma(__ldg(vt + 5), outv[0], T1);
                T2 = fma(__ldg(vt + 6), outv[0], T2);
                if (C == 2) TG = fma(__ldg(vt + 3), outv[C - 1], TG);
            }
            if (rec) { g *= r; r *= rho1; }
            buf ^= 1;
        }
        // fold the line sums: T_m = sum_j w u1^m F over the line
        m[0] += T0; m[1] += T1; m[2] = fma(u2, T0, m[2]); m[3] = fma(u3, T0, m[3]);
        m[4] += T2; m[5] = fma(u2 * u2, T0, m[5]); m[6] = fma(u3 * u3, T0, m[6]);
        m[7] = fma(u2, T1, m[7]); m[8] = fma(u3, T1, m[8]); m[9] = fma(u2 * u3, T0, m[9]);
        m[10] += TG;
    }
    if (a.part && active) {
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

template <typename T>
cudaError_t launch_entropy(const T *f, const double *vtab, int Nu, int P, int Kblk, int n_vblk, double *part,
                           double *h_out, unsigned int *nonpos, cudaStream_t s) {
    dim3 grid((P + 255) / 256, n_vblk);
    k_entropy_partial<T><<<grid, 256, 0, s>>>(f, vtab, Nu, P, Kblk, part, nonpos);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_reduce_entropy<<<(P + 255) / 256, 256, 0, s>>>(part, n_vblk, P, h_out);
    return cudaGetLastError();
}
template cudaError_t launch_entropy<double>(const double *, const double *, int, int, int, int, double *, double *,
                                            unsigned int *, cudaStream_t);
template cudaError_t launch_entropy<float>(const float *, const double *, int, int, int, int, double *, double *,
                                           unsigned int *, cudaStream_t);

cudaError_t launch_sum_partials(const double *part, int n_vblk, int P, double *out, cudaStream_t s) {
    k_sum_partials<<<(P + 255) / 256, 256, 0, s>>>(part, n_vblk, P, out);
    return cudaGetLastError();
}

cudaError_t launch_reduce_moments(const double *part, int n_vblk, int P, double *m_out,
                                  cudaStream_t s) {
    k_reduce_moments<<<(P + 255) / 256, 256, 0, s>>>(part, n_vblk, P, m_out);
    return cudaGetLastError();
}

template <int Q>
static cudaError_t stage_q(const StageArgs<double> &a, int C, int n_vblk, cudaStream_t s) {
    constexpr int NS = Q * Q * Q, EB = 256 / NS;
    dim3 grid((a.mesh.Ne + EB - 1) / EB, n_vblk);
    if (a.geo) {
        if (C == 1) k_stage_f64<Q, 1, true><<<grid, EB * NS, 0, s>>>(a);
        else k_stage_f64<Q, 2, true><<<grid, EB * NS, 0, s>>>(a);
    } else {
        if (C == 1) k_stage_f64<Q, 1, false><<<grid, EB * NS, 0, s>>>(a);
        else k_stage_f64<Q, 2, false><<<grid, EB * NS, 0, s>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_stage_f64(const StageArgs<double> &a, int C, int n_vblk, cudaStream_t s) {
    switch (a.fr.q) {
        case 2: return stage_q<2>(a, C, n_vblk, s);
        case 3: return stage_q<3>(a, C, n_vblk, s);
        case 4: return stage_q<4>(a, C, n_vblk, s);
        case 5: return stage_q<5>(a, C, n_vblk, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_maxwellian_f64(double *f, const double *q, const double *vtab, int Nu, int P,
                                  int C, double delta, cudaStream_t s) {
    const size_t n = (size_t)Nu * P;
    k_maxwellian_f64<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(f, q, vtab, Nu, P, C, delta);
    return cudaGetLastError();
}
