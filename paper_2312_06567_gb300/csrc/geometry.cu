// Host-side metric terms of curvilinear hexahedral elements (section
// "Numerical method": the FR flux correction uses the outward normals of the
// flux nodes; on a curved element the equation is mapped to the reference
// cube, J d_t f + sum_d d/dxi_d ((u . S^d) f) = J S with S^d = J grad xi_d).
//
// Per element, from the solution-node coordinates (the nodal interpolant of
// degree p is the element's geometry):
//   - S^d in the conservative curl form, (S^i)_n = -[curl_xi (X_l grad_xi X_m)]_i
//     with (n, m, l) cyclic, the products and derivatives taken on the
//     element's Gauss--Lobatto--Legendre points and the resulting polynomial
//     evaluated at the Gauss--Legendre solution nodes.  Its divergence
//     vanishes identically, and on a face it depends only on the face's own
//     geometry, so a continuous mesh preserves a uniform state exactly;
//   - J = det(dX/dxi) at the solution nodes;
//   - face vectors: the trace of S^d on each face, averaged with the
//     neighbour's trace of the same face (identical for a continuous mesh;
//     the average keeps the common flux single-valued in any case).
#include <cmath>
#include <string>
#include <vector>

#include "bgk_internal.cuh"

namespace {

// P_n and P_n' by the three-term recurrence.
void legendre_pd(int n, double x, double &pn, double &dpn) {
    double p0 = 1.0, p1 = x, d0 = 0.0, d1 = 1.0;
    if (n == 0) { pn = 1.0; dpn = 0.0; return; }
    for (int k = 1; k < n; ++k) {
        const double p2 = ((2 * k + 1) * x * p1 - k * p0) / (k + 1);
        const double d2 = d0 + (2 * k + 1) * p1;
        p0 = p1; p1 = p2; d0 = d1; d1 = d2;
    }
    pn = p1; dpn = d1;
}

// GLL points: -1, the roots of P'_{q-1} (Newton with P'' from Legendre's
// equation), +1.
std::vector<double> gll(int q) {
    std::vector<double> x(q);
    const int N = q - 1;
    x[0] = -1.0; x[N] = 1.0;
    for (int i = 1; i < N; ++i) {
        double t = -std::cos(M_PI * i / N);
        for (int it = 0; it < 100; ++it) {
            double pn, dpn;
            legendre_pd(N, t, pn, dpn);
            const double d2 = (2.0 * t * dpn - N * (N + 1.0) * pn) / (1.0 - t * t);
            const double dt = dpn / d2;
            t -= dt;
            if (std::fabs(dt) < 1e-16) break;
        }
        x[i] = t;
    }
    return x;
}

// Barycentric weights b_j = 1 / prod_{m != j} (x_j - x_m).
std::vector<double> bary(const std::vector<double> &x) {
    const int q = (int)x.size();
    std::vector<double> b(q);
    for (int j = 0; j < q; ++j) {
        double pr = 1.0;
        for (int m = 0; m < q; ++m)
            if (m != j) pr *= x[j] - x[m];
        b[j] = 1.0 / pr;
    }
    return b;
}

// L[i][j] = l_j(t_i) for the Lagrange basis on x (q x q, row-major).
std::vector<double> interp(const std::vector<double> &x, const std::vector<double> &t) {
    const int q = (int)x.size(), r = (int)t.size();
    std::vector<double> L((size_t)r * q);
    for (int i = 0; i < r; ++i)
        for (int j = 0; j < q; ++j) {
            double v = 1.0;
            for (int m = 0; m < q; ++m)
                if (m != j) v *= (t[i] - x[m]) / (x[j] - x[m]);
            L[(size_t)i * q + j] = v;
        }
    return L;
}

// D[i][j] = l_j'(x_i).
std::vector<double> deriv(const std::vector<double> &x) {
    const int q = (int)x.size();
    const std::vector<double> b = bary(x);
    std::vector<double> D((size_t)q * q, 0.0);
    for (int i = 0; i < q; ++i) {
        double diag = 0.0;
        for (int j = 0; j < q; ++j)
            if (j != i) {
                D[(size_t)i * q + j] = (b[j] / b[i]) / (x[i] - x[j]);
                diag -= D[(size_t)i * q + j];
            }
        D[(size_t)i * q + i] = diag;
    }
    return D;
}

// Nodal arrays of one element: g[(i3 * q + i2) * q + i1].
struct Elem {
    int q;
    explicit Elem(int q_) : q(q_) {}
    int at(int i1, int i2, int i3) const { return (i3 * q + i2) * q + i1; }
    // apply the q x q matrix M along axis ax (0: i1, 1: i2, 2: i3)
    std::vector<double> along(const std::vector<double> &g, const std::vector<double> &M, int ax) const {
        std::vector<double> o(g.size(), 0.0);
        for (int i3 = 0; i3 < q; ++i3)
            for (int i2 = 0; i2 < q; ++i2)
                for (int i1 = 0; i1 < q; ++i1) {
                    const int id[3] = {i1, i2, i3};
                    double s = 0.0;
                    for (int j = 0; j < q; ++j) {
                        int jd[3] = {i1, i2, i3};
                        jd[ax] = j;
                        s += M[(size_t)id[ax] * q + j] * g[at(jd[0], jd[1], jd[2])];
                    }
                    o[at(i1, i2, i3)] = s;
                }
        return o;
    }
    std::vector<double> all3(const std::vector<double> &g, const std::vector<double> &M) const {
        return along(along(along(g, M, 0), M, 1), M, 2);
    }
};

}  // namespace

// x[P][3] node coordinates (P = Ne * Ns, element e = e1 + n1 (e2 + n2 e3),
// node s = i1 + q (i2 + q i3)).  Outputs geo[P][BGK_NGEO] and
// fvec[Ne][6][q*q][3] (face 2d + (side > 0), face point indexed by the two
// other node indices, lower axis fastest).  Returns false (with err) on a
// non-positive Jacobian.
bool build_curved_geometry(const FROps &fr, const int n[3], const int periodic[3], const double *x,
                           std::vector<double> &geo, std::vector<double> &fvec, std::string &err) {
    const int q = fr.q, Ns = q * q * q;
    const int Ne = n[0] * n[1] * n[2];
    std::vector<double> xg(fr.xi, fr.xi + q);
    const std::vector<double> xl = gll(q);
    const std::vector<double> to_gll = interp(xg, xl), to_gl = interp(xl, xg);
    const std::vector<double> DL = deriv(xl), DG = deriv(xg);
    const Elem E(q);
    geo.assign((size_t)Ne * Ns * BGK_NGEO, 0.0);
    std::vector<double> own((size_t)Ne * 6 * q * q * 3, 0.0);
    static const int cyc[3][3] = {{0, 1, 2}, {1, 2, 0}, {2, 0, 1}};
    for (int e = 0; e < Ne; ++e) {
        std::vector<double> X[3], XL[3];
        for (int c = 0; c < 3; ++c) {
            X[c].resize(Ns);
            for (int s = 0; s < Ns; ++s) X[c][s] = x[((size_t)e * Ns + s) * 3 + c];
            XL[c] = E.all3(X[c], to_gll);
        }
        std::vector<double> dXL[3][3], dXG[3][3];     // [j][c] = d_j X_c
        for (int j = 0; j < 3; ++j)
            for (int c = 0; c < 3; ++c) {
                dXL[j][c] = E.along(XL[c], DL, j);
                dXG[j][c] = E.along(X[c], DG, j);
            }
        std::vector<double> S[3][3];                  // [i][c] at the Gauss nodes
        for (int t = 0; t < 3; ++t) {
            const int nn = cyc[t][0], m = cyc[t][1], l = cyc[t][2];
            std::vector<double> V[3];
            for (int j = 0; j < 3; ++j) {
                V[j].resize(Ns);
                for (int s = 0; s < Ns; ++s) V[j][s] = XL[l][s] * dXL[j][m][s];
            }
            for (int r = 0; r < 3; ++r) {
                const int i = cyc[r][0], j = cyc[r][1], k = cyc[r][2];
                const std::vector<double> a = E.along(V[k], DL, j), b = E.along(V[j], DL, k);
                std::vector<double> SLn(Ns);
                for (int s = 0; s < Ns; ++s) SLn[s] = -(a[s] - b[s]);
                S[i][nn] = E.all3(SLn, to_gl);
            }
        }
        for (int s = 0; s < Ns; ++s) {
            const double a11 = dXG[0][0][s], a12 = dXG[1][0][s], a13 = dXG[2][0][s];
            const double a21 = dXG[0][1][s], a22 = dXG[1][1][s], a23 = dXG[2][1][s];
            const double a31 = dXG[0][2][s], a32 = dXG[1][2][s], a33 = dXG[2][2][s];
            const double J = a11 * (a22 * a33 - a23 * a32) - a12 * (a21 * a33 - a23 * a31) + a13 * (a21 * a32 - a22 * a31);
            if (!(J > 0.0)) {
                err = "non-positive Jacobian at a solution node of element " + std::to_string(e);
                return false;
            }
            double *g = &geo[((size_t)e * Ns + s) * BGK_NGEO];
            for (int i = 0; i < 3; ++i)
                for (int c = 0; c < 3; ++c) g[3 * i + c] = S[i][c][s];
            const int i1 = s % q, i2 = (s / q) % q, i3 = s / (q * q);
            g[9] = 1.0 / J;
            g[10] = fr.wq[i1] * fr.wq[i2] * fr.wq[i3] * J;
        }
        // own traces of S^d on the faces of the element
        for (int d = 0; d < 3; ++d)
            for (int side = 0; side < 2; ++side) {
                const double *lw = side ? fr.lp : fr.lm;
                for (int b = 0; b < q; ++b)
                    for (int a = 0; a < q; ++a) {
                        for (int c = 0; c < 3; ++c) {
                            double t = 0.0;
                            for (int j = 0; j < q; ++j) {
                                int id[3];
                                if (d == 0) { id[0] = j; id[1] = a; id[2] = b; }
                                else if (d == 1) { id[0] = a; id[1] = j; id[2] = b; }
                                else { id[0] = a; id[1] = b; id[2] = j; }
                                t += lw[j] * S[d][c][E.at(id[0], id[1], id[2])];
                            }
                            own[((((size_t)e * 6 + 2 * d + side) * q * q) + a + q * b) * 3 + c] = t;
                        }
                    }
            }
    }
    fvec = own;
    const int estr[3] = {1, n[0], n[0] * n[1]};
    for (int e = 0; e < Ne; ++e) {
        const int ec[3] = {e % n[0], (e / n[0]) % n[1], e / (n[0] * n[1])};
        for (int d = 0; d < 3; ++d)
            for (int side = 0; side < 2; ++side) {
                int nb;
                if (side == 0) nb = ec[d] > 0 ? e - estr[d] : (periodic[d] ? e + (n[d] - 1) * estr[d] : -1);
                else nb = ec[d] < n[d] - 1 ? e + estr[d] : (periodic[d] ? e - (n[d] - 1) * estr[d] : -1);
                if (nb < 0) continue;
                for (int i = 0; i < q * q * 3; ++i) {
                    const size_t mine = ((size_t)e * 6 + 2 * d + side) * q * q * 3 + i;
                    const size_t theirs = ((size_t)nb * 6 + 2 * d + 1 - side) * q * q * 3 + i;
                    fvec[mine] = 0.5 * (own[mine] + own[theirs]);
                }
            }
    }
    return true;
}
