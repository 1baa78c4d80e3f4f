// Macroscopic post-processing per solution point: rho, U, theta, p, Mach,
// the local mean free path lambda = (mu(theta)/rho) sqrt(pi/(2 theta)), the
// FR density gradient norm and the gradient-length local Knudsen number
// Kn_GLL = lambda ||grad rho|| / rho (Dzanic & Martinelli, arXiv 2312.06567,
// section "Results": continuum breakdown above 0.05).  The gradient is that
// of the FR-corrected density polynomial along each reference direction:
// the nodal derivative plus the correction-function derivatives times the
// differences between the central common interface value (at a Dirichlet
// face, the average with the face state's density; at a specular, diffuse
// or collapsed face the element's own trace: none of them prescribes a
// density) and the element's trace.  On the box d/dx_d = (2/h_d) d/dxi_d; on
// a curvilinear mesh the chain rule grad rho = (1/J) sum_d S^d d rho/d xi_d
// with the node's metric terms S^d = J grad xi_d.
// FP64; one thread per point.
#include "bgk_internal.cuh"

namespace {

// geo: the curvilinear node records [P][BGK_NGEO] (S^1, S^2, S^3, 1/J, ...) or null on the box
__global__ void k_macro(const double *mom, double *out, int P, MeshInfo mesh, FROps fr, GasInfo gas,
                        double3 bc_lo, double3 bc_hi, const double *geo) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const int q = fr.q, NS = q * q * q;
    const int e = p / NS, s = p - e * NS;
    const double *m = mom + (size_t)p * BGK_NMOM;
    const double rho = m[0];
    const double U[3] = {m[1] / rho, m[2] / rho, m[3] / rho};
    const double E = 0.5 * (m[4] + m[5] + m[6]) + m[10];
    const double u2 = U[0] * U[0] + U[1] * U[1] + U[2] * U[2];
    const double pres = (gas.gamma - 1.0) * (E - 0.5 * rho * u2);
    const double theta = pres / rho;
    double mu = gas.mu_ref;
    if (gas.theta_S >= 0.0) {
        const double r = theta / gas.theta_ref;
        mu = gas.mu_ref * r * sqrt(r) * (gas.theta_ref + gas.theta_S) / (theta + gas.theta_S);
    }
    const double lam = mu / rho * sqrt(3.14159265358979323846 / (2.0 * theta));
    const double mach = sqrt(u2 / (gas.gamma * theta));
    // FR gradient of rho
    const int id[3] = {s % q, (s / q) % q, s / (q * q)};
    const int stride[3] = {1, q, q * q};
    const int n1 = mesh.n[0], n2 = mesh.n[1], n3 = mesh.n[2];
    const int ec[3] = {e % n1, (e / n1) % n2, e / (n1 * n2)};
    const int estr[3] = {1, n1, n1 * n2};
    const int nn[3] = {n1, n2, n3};
    const double face_lo[3] = {bc_lo.x, bc_lo.y, bc_lo.z}, face_hi[3] = {bc_hi.x, bc_hi.y, bc_hi.z};
    double dxi[3];
    for (int d = 0; d < 3; ++d) {
        const int base = s - id[d] * stride[d];
        const int i = id[d];
        double der = 0.0, trL = 0.0, trR = 0.0;
        for (int j = 0; j < q; ++j) {
            const double r = mom[((size_t)e * NS + base + j * stride[d]) * BGK_NMOM];
            der = fma(fr.D[i][j], r, der);
            trL = fma(fr.lm[j], r, trL);
            trR = fma(fr.lp[j], r, trR);
        }
        // the neighbours' traces on the shared faces (or the Dirichlet face density)
        double outL, outR;
        const int eL = ec[d] > 0 ? e - estr[d] : (mesh.periodic[d] ? e + (nn[d] - 1) * estr[d] : -1);
        const int eR = ec[d] < nn[d] - 1 ? e + estr[d] : (mesh.periodic[d] ? e - (nn[d] - 1) * estr[d] : -1);
        if (eL >= 0) {
            outL = 0.0;
            for (int j = 0; j < q; ++j) outL = fma(fr.lp[j], mom[((size_t)eL * NS + base + j * stride[d]) * BGK_NMOM], outL);
        } else {
            // a Dirichlet face prescribes the density; the other faces give the element's own trace
            outL = (mesh.face_kind[2 * d] == BGK_FK_DIRICHLET && !mesh.specular[2 * d]) ? face_lo[d] : trL;
        }
        if (eR >= 0) {
            outR = 0.0;
            for (int j = 0; j < q; ++j) outR = fma(fr.lm[j], mom[((size_t)eR * NS + base + j * stride[d]) * BGK_NMOM], outR);
        } else {
            outR = (mesh.face_kind[2 * d + 1] == BGK_FK_DIRICHLET && !mesh.specular[2 * d + 1]) ? face_hi[d] : trR;
        }
        const double cL = 0.5 * (trL + outL), cR = 0.5 * (trR + outR);
        der += (cL - trL) * fr.dgL[i] + (cR - trR) * fr.dgR[i];
        dxi[d] = der;
    }
    double g2 = 0.0;
    if (geo) {
        const double *g = geo + (size_t)p * BGK_NGEO;
        for (int c = 0; c < 3; ++c) {
            const double gc = g[9] * (g[c] * dxi[0] + g[3 + c] * dxi[1] + g[6 + c] * dxi[2]);
            g2 = fma(gc, gc, g2);
        }
    } else {
        for (int d = 0; d < 3; ++d) {
            const double gd = mesh.two_over_h[d] * dxi[d];
            g2 = fma(gd, gd, g2);
        }
    }
    const double gn = sqrt(g2);
    double *o = out + (size_t)p * BGK_NMACRO;
    o[0] = rho; o[1] = U[0]; o[2] = U[1]; o[3] = U[2]; o[4] = theta; o[5] = pres;
    o[6] = mach; o[7] = lam; o[8] = gn; o[9] = lam * gn / rho;
}

}  // namespace

cudaError_t launch_macro(const double *mom, double *out, int P, const MeshInfo &mesh, const FROps &fr,
                         const GasInfo &gas, const double face_rho[6], const double *geo, cudaStream_t s) {
    const double3 lo = make_double3(face_rho[0], face_rho[2], face_rho[4]);
    const double3 hi = make_double3(face_rho[1], face_rho[3], face_rho[5]);
    k_macro<<<(P + 255) / 256, 256, 0, s>>>(mom, out, P, mesh, fr, gas, lo, hi, geo);
    return cudaGetLastError();
}
