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

// Medium of relative permittivity eps_re + j eps_im inside (k2 = k0 sqrt(eps_r), the root
// with Im <= 0: a decaying wave for exp(j w t)); host function (hm_muller_dev.cu).
MullerMedia muller_media(double k0, double eps_re, double eps_im);

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

// ---------------------------------------------------------------------------
// Integrand of the N-Mueller self/near integrals at one source point r' = r(u,v)
// with tangents a_u, a_v, for target r_i with tangents (tu = a_u(r_i), tv = a_v(r_i)):
// the coefficients of the cardinal function ell_j (cl) and of its derivative along
// the source direction of the column (cd, divergence terms only), per unit du dv:
//   E-row b, J^a: cl = j k K_S (t_b.a_a),  cd = -(1/(j k)) gD (t_b.R)
//   E-row b, M^a: cl = gE t_b.(R x a_a)
//   H-row b, J^a: cl = -gD t_b.(R x a_a)
//   H-row b, M^a: as E-row b, J^a.
// ---------------------------------------------------------------------------
__host__ __device__ inline void muller_point(const double *ri, const double *tu, const double *tv, const double *r,
                                             const double *ru, const double *rv, const MullerMedia &md, zc *cl,
                                             zc *cd)
{
    double R3[3] = {ri[0] - r[0], ri[1] - r[1], ri[2] - r[2]};
    double R = sqrt(R3[0] * R3[0] + R3[1] * R3[1] + R3[2] * R3[2]);
    zc G1, g1, G2, g2;
    green_pair(zmake(md.k, 0.0), R, G1, g1);
    green_pair(md.k2, R, G2, g2);
    zc KS = zsub(G1, zmul(md.epsr, G2)), gD = zsub(g1, g2), gE = zsub(g1, zmul(md.epsr, g2));
    const zc jk = zmake(0.0, md.k), inv_jk = zmake(0.0, -1.0 / md.k);
    double t[2][3] = {{-tv[0], -tv[1], -tv[2]}, {tu[0], tu[1], tu[2]}};
    const double *a[2] = {ru, rv};
    for (int b = 0; b < 2; ++b) {
        double tR = t[b][0] * R3[0] + t[b][1] * R3[1] + t[b][2] * R3[2];
        zc sd = zmul(inv_jk, zscale(gD, -tR));
        for (int aa = 0; aa < 2; ++aa) {
            const double *av = a[aa];
            double ta = t[b][0] * av[0] + t[b][1] * av[1] + t[b][2] * av[2];
            double cr[3] = {R3[1] * av[2] - R3[2] * av[1], R3[2] * av[0] - R3[0] * av[2], R3[0] * av[1] - R3[1] * av[0]};
            double tc = t[b][0] * cr[0] + t[b][1] * cr[1] + t[b][2] * cr[2];
            zc sl = zscale(zmul(jk, KS), ta);
            cl[b * 4 + aa] = sl;
            cd[b * 4 + aa] = sd;
            cl[b * 4 + 2 + aa] = zscale(gE, tc);
            cd[b * 4 + 2 + aa] = zmake(0, 0);
            cl[(2 + b) * 4 + aa] = zscale(gD, -tc);
            cd[(2 + b) * 4 + aa] = zmake(0, 0);
            cl[(2 + b) * 4 + 2 + aa] = sl;
            cd[(2 + b) * 4 + 2 + aa] = sd;
        }
    }
}

// ---------------------------------------------------------------------------
// Pieces of the self/near quadrature rule on the source patch's parameter square,
// split at the point (uc, vc) nearest the singularity (the same construction as the
// MFIE near-field kernel): for a near target (eps > 0) four tensor rectangles with
// graded axes (a sinh-mapped Gauss panel of length min(L, t0) clustered at the corner
// on the scale eps, then a plain Gauss panel on [t0, L]); for a self target (eps = 0)
// on each corner rectangle a Duffy square (two triangles, Jacobian s) on its physically
// square part and a tensor strip (plain across, graded along) on the remainder.
// ---------------------------------------------------------------------------
struct NearAxis {
    int graded;              // 1: graded (sinh panel + plain panel), 0: plain Gauss
    double eps, L, start, sgn;
};
struct NearPiece {
    int type;                // 0 tensor (axes A = u, B = v); 1 Duffy u = uc + du s, v = vc + dv s t;
                             // 2 Duffy v = vc + dv s, u = uc + du s t
    double uc, vc, du, dv;   // Duffy corner and signed side lengths
    NearAxis A, B;           // tensor axes
};

// Returns the number of pieces written to pc (at most 12).  gu, gv: |a_u|, |a_v| at
// (uc, vc) (they decide the physically square part of a self rectangle).
__host__ __device__ inline int near_pieces(double uc, double vc, double eps, double gu, double gv, NearPiece *pc)
{
    int np = 0;
    for (int corner = 0; corner < 4; ++corner) {
        double du = (corner & 1) ? (-1.0 - uc) : (1.0 - uc);
        double dv = (corner & 2) ? (-1.0 - vc) : (1.0 - vc);
        if (fabs(du) < 1e-14 || fabs(dv) < 1e-14) continue;
        double su = du > 0 ? 1.0 : -1.0, sv = dv > 0 ? 1.0 : -1.0;
        if (eps > 0.0) {
            NearPiece &p = pc[np++];
            p.type = 0;
            p.A = NearAxis{1, eps, fabs(du), uc, su};
            p.B = NearAxis{1, eps, fabs(dv), vc, sv};
            continue;
        }
        double pa = fabs(du) * gu, pb = fabs(dv) * gv;
        double ddu = du, ddv = dv;
        int strip = 0;
        if (pb > pa) {
            ddv = sv * pa / gv;
            if (fabs(dv) - fabs(ddv) > 1e-14) strip = 1;
        } else {
            ddu = su * pb / gu;
            if (fabs(du) - fabs(ddu) > 1e-14) strip = 2;
        }
        for (int tri = 1; tri <= 2; ++tri) {
            NearPiece &p = pc[np++];
            p.type = tri;
            p.uc = uc;
            p.vc = vc;
            p.du = ddu;
            p.dv = ddv;
        }
        if (strip) {
            NearPiece &p = pc[np++];
            p.type = 0;
            if (strip == 1) {
                p.A = NearAxis{0, 0.0, fabs(du), uc, su};
                p.B = NearAxis{1, fabs(ddv), fabs(dv) - fabs(ddv), vc + ddv, sv};
            } else {
                p.A = NearAxis{1, fabs(ddu), fabs(du) - fabs(ddu), uc + ddu, su};
                p.B = NearAxis{0, 0.0, fabs(dv), vc, sv};
            }
        }
    }
    return np;
}

// Points and weights of one axis on [0,1]-mapped Gauss tables: gi (qi points) for the
// graded inner panel and the plain axis, go (qo points) for the outer panel.  Returns
// the number of points (<= qi + qo).
__host__ __device__ inline int near_axis_points(const NearAxis &ax, const double *gix, const double *giw, int qi,
                                                const double *gox, const double *gow, int qo, double t0, double *x,
                                                double *w)
{
    int n = 0;
    if (!ax.graded) {
        for (int i = 0; i < qi; ++i) {
            x[n] = ax.start + ax.sgn * ax.L * gix[i];
            w[n] = ax.L * giw[i];
            ++n;
        }
        return n;
    }
    double Lin = fmin(ax.L, t0);
    double mu = asinh(Lin / ax.eps);
    for (int i = 0; i < qi; ++i) {
        double z = mu * gix[i];
        x[n] = ax.start + ax.sgn * ax.eps * sinh(z);
        w[n] = ax.eps * mu * cosh(z) * giw[i];
        ++n;
    }
    if (ax.L > t0) {
        for (int i = 0; i < qo; ++i) {
            x[n] = ax.start + ax.sgn * (t0 + (ax.L - t0) * gox[i]);
            w[n] = (ax.L - t0) * gow[i];
            ++n;
        }
    }
    return n;
}

// ---------------------------------------------------------------------------
// Right-hand side of one node for the plane wave E = pol exp(-jk khat.r):
// E-row b: t_b . E_inc, H-row b: t_b . (eta0 H_inc) = t_b . (khat x pol) exp(-jk khat.r).
// X: node table SoA [14][nnode].  out[4]: (E-u, E-v, H-u, H-v).
// ---------------------------------------------------------------------------
__host__ __device__ inline void muller_rhs_node(const double *X, int nnode, int i, double k, const double *kh,
                                                const double *po, zc *out)
{
    const int n = nnode;
    double h0[3] = {kh[1] * po[2] - kh[2] * po[1], kh[2] * po[0] - kh[0] * po[2], kh[0] * po[1] - kh[1] * po[0]};
    double ph = -k * (kh[0] * X[i] + kh[1] * X[n + i] + kh[2] * X[2 * n + i]);
    zc e = zmake(cos(ph), sin(ph));
    double au[3] = {X[3 * n + i], X[4 * n + i], X[5 * n + i]};
    double av[3] = {X[6 * n + i], X[7 * n + i], X[8 * n + i]};
    out[0] = zscale(e, -(av[0] * po[0] + av[1] * po[1] + av[2] * po[2]));
    out[1] = zscale(e, au[0] * po[0] + au[1] * po[1] + au[2] * po[2]);
    out[2] = zscale(e, -(av[0] * h0[0] + av[1] * h0[1] + av[2] * h0[2]));
    out[3] = zscale(e, au[0] * h0[0] + au[1] * h0[1] + au[2] * h0[2]);
}

// Contribution of node j to the radiation vectors in direction rh:
// NJ += w_j (Jbar^u a_u + Jbar^v a_v) exp(jk rh.r_j), NM likewise with M (x: 4 values).
// The far field is E_far = -jk/(4 pi) [(I - rh rh) NJ - rh x NM].
__host__ __device__ inline void muller_radiation_add(const double *X, int nnode, int j, double k, const double *rh,
                                                     const zc *x, zc *NJ, zc *NM)
{
    const int n = nnode;
    double ph = k * (rh[0] * X[j] + rh[1] * X[n + j] + rh[2] * X[2 * n + j]);
    zc e = zscale(zmake(cos(ph), sin(ph)), X[13 * n + j]);
    zc ju = zmul(x[0], e), jv = zmul(x[1], e), mu = zmul(x[2], e), mv = zmul(x[3], e);
    for (int d = 0; d < 3; ++d) {
        double au = X[(3 + d) * n + j], av = X[(6 + d) * n + j];
        NJ[d] = zadd(NJ[d], zadd(zscale(ju, au), zscale(jv, av)));
        NM[d] = zadd(NM[d], zadd(zscale(mu, au), zscale(mv, av)));
    }
}

__host__ __device__ inline void muller_far_field(const double *rh, double k, const zc *NJ, const zc *NM, zc *E)
{
    zc rn = zadd(zadd(zscale(NJ[0], rh[0]), zscale(NJ[1], rh[1])), zscale(NJ[2], rh[2]));
    zc rxm[3] = {zsub(zscale(NM[2], rh[1]), zscale(NM[1], rh[2])), zsub(zscale(NM[0], rh[2]), zscale(NM[2], rh[0])),
                 zsub(zscale(NM[1], rh[0]), zscale(NM[0], rh[1]))};
    zc pre = zmake(0.0, -k / (4.0 * 3.14159265358979323846));
    for (int d = 0; d < 3; ++d) E[d] = zmul(pre, zsub(zsub(NJ[d], zscale(rn, rh[d])), rxm[d]));
}
