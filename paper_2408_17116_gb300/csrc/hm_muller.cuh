// N-Mueller formulation of a dielectric body (Sec. II.A, Eqs. 7-9 with
// alpha = -eps2/eps1, beta = -mu2/mu1, mu_r = 1): the far (Nystrom) entries of one
// target node / source node pair, written for both host and device so the fill and
// ACA entry generators and a host check share one definition.
//
// Rows per target node: E-u, E-v, H-u, H-v (the equations tested with sqrt|G| a^b,
// Eqs. 17-18, i.e. t_u = -a_v, t_v = a_u applied to the vector inside n x [ ]).
// Columns per source node: Jbar^u, Jbar^v, M^u, M^v with Jbar = eta0 J and
// F^a = sqrt|G| x contravariant component (Eq. 11).  With R = r_i - r_j,
// K_S = G1 - eps_r G2, grad(G1 - G2) = gD R, grad(G1 - eps_r G2) = gE R:
//   E-row b, J^a:  w_j j k K_S (t_b.a_a) - (1/(j k)) sum_{j' on the a-line of j} w_j' gD' (t_b.R') D_a[j', j]
//   E-row b, M^a:  w_j gE t_b.(R x a_a)
//   H-row b, J^a: -w_j gD t_b.(R x a_a)
//   H-row b, M^a:  as E-row b, J^a
// where the divergence terms carry the spectral derivative of the source patch's
// Chebyshev interpolant along the grid line through node j (D_a[j', j] =
// d ell_j / d a at node j').  The identity terms of the jump relations are not part
// of these far entries.
#pragma once
#include "hm_device.cuh"

struct MullerMedia {
    double k;     // exterior wavenumber
    zc epsr;      // interior relative permittivity
    zc k2;        // interior wavenumber k sqrt(eps_r), Im <= 0
};

// exp(-j kc R) for a complex wavenumber kc (Im kc <= 0: decaying)
__host__ __device__ __forceinline__ zc expmj(zc kc, double R)
{
    double amp = exp(kc.y * R), s, c;
#ifdef __CUDA_ARCH__
    sincos(kc.x * R, &s, &c);
#else
    s = sin(kc.x * R);
    c = cos(kc.x * R);
#endif
    return zmake(amp * c, -amp * s);
}

// G(R) and g(R) (grad G = g R) for wavenumber kc: G = e/(4 pi R), g = -(1 + j kc R) e/(4 pi R^3)
__host__ __device__ __forceinline__ void green_pair(zc kc, double R, zc &G, zc &g)
{
    const double fpi = 4.0 * 3.14159265358979323846;
    zc e = expmj(kc, R);
    G = zscale(e, 1.0 / (fpi * R));
    zc f = zmake(1.0 - kc.y * R, kc.x * R);  // 1 + j kc R
    g = zscale(zmul(f, e), -1.0 / (fpi * R * R * R));
}

// The 16 far entries out[row * 4 + col] for target node ni and source node nj of a
// patch with nc x nc nodes (node index p nc^2 + kv nc + lu).  X: node table SoA
// [14][nnode] (r, a_u, a_v, n, sqrtG, w).  d1[l' * nc + l]: derivative of the l-th
// Chebyshev cardinal function at node l'.
__host__ __device__ inline void muller_far_pair(const double *X, int nnode, int nc, const double *d1,
                                                const MullerMedia &md, int ni, int nj, zc *out)
{
    const int n = nnode, nc2 = nc * nc;
    const int p = nj / nc2, loc = nj - p * nc2, kv = loc / nc, lu = loc - kv * nc;
    double t[2][3], a[2][3];
    for (int q = 0; q < 3; ++q) {
        t[0][q] = -X[(6 + q) * n + ni];
        t[1][q] = X[(3 + q) * n + ni];
        a[0][q] = X[(3 + q) * n + nj];
        a[1][q] = X[(6 + q) * n + nj];
    }
    const zc kk = zmake(md.k, 0.0);
    const zc jk = zmake(0.0, md.k), inv_jk = zmake(0.0, -1.0 / md.k);  // j k and 1/(j k)
    // point terms at (ni, nj)
    double R3[3];
    for (int q = 0; q < 3; ++q) R3[q] = X[q * n + ni] - X[q * n + nj];
    double R = sqrt(R3[0] * R3[0] + R3[1] * R3[1] + R3[2] * R3[2]);
    zc G1, g1, G2, g2;
    green_pair(kk, R, G1, g1);
    green_pair(md.k2, R, G2, g2);
    const double wj = X[13 * n + nj];
    zc KS = zsub(G1, zmul(md.epsr, G2)), gD = zsub(g1, g2), gE = zsub(g1, zmul(md.epsr, g2));
    for (int b = 0; b < 2; ++b)
        for (int aa = 0; aa < 2; ++aa) {
            double ta = t[b][0] * a[aa][0] + t[b][1] * a[aa][1] + t[b][2] * a[aa][2];
            double cr[3] = {R3[1] * a[aa][2] - R3[2] * a[aa][1], R3[2] * a[aa][0] - R3[0] * a[aa][2],
                            R3[0] * a[aa][1] - R3[1] * a[aa][0]};
            double tc = t[b][0] * cr[0] + t[b][1] * cr[1] + t[b][2] * cr[2];
            zc sl = zscale(zmul(jk, KS), wj * ta);
            out[b * 4 + aa] = sl;
            out[b * 4 + 2 + aa] = zscale(gE, wj * tc);
            out[(2 + b) * 4 + aa] = zscale(gD, -wj * tc);
            out[(2 + b) * 4 + 2 + aa] = sl;
        }
    // divergence terms: sum over the source nodes on the u-line (a = u) and the v-line (a = v)
    for (int aa = 0; aa < 2; ++aa) {
        zc acc[2] = {zmake(0, 0), zmake(0, 0)};
        for (int l2 = 0; l2 < nc; ++l2) {
            const int jp = p * nc2 + (aa == 0 ? kv * nc + l2 : l2 * nc + lu);
            const double dd = aa == 0 ? d1[l2 * nc + lu] : d1[l2 * nc + kv];
            double Rp[3];
            for (int q = 0; q < 3; ++q) Rp[q] = X[q * n + ni] - X[q * n + jp];
            double Rn = sqrt(Rp[0] * Rp[0] + Rp[1] * Rp[1] + Rp[2] * Rp[2]);
            zc Ga, ga, Gb, gb;
            green_pair(kk, Rn, Ga, ga);
            green_pair(md.k2, Rn, Gb, gb);
            zc gd = zscale(zsub(ga, gb), X[13 * n + jp] * dd);
            for (int b = 0; b < 2; ++b) {
                double tR = t[b][0] * Rp[0] + t[b][1] * Rp[1] + t[b][2] * Rp[2];
                acc[b] = zadd(acc[b], zscale(gd, tR));
            }
        }
        for (int b = 0; b < 2; ++b) {
            zc dv = zmul(inv_jk, acc[b]);
            out[b * 4 + aa] = zsub(out[b * 4 + aa], dv);
            out[(2 + b) * 4 + 2 + aa] = zsub(out[(2 + b) * 4 + 2 + aa], dv);
        }
    }
}
