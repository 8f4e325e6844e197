// Host evaluation of the N-Mueller far entries (hm_muller.cuh) for one target node
// and one source patch, with the library's own geometry: the check of that entry
// generator against an independent implementation, before the device fill uses it.
#include <algorithm>
#include <cmath>
#include <vector>

#include "hm_internal.h"
#include "hm_muller.cuh"

// Derivative of the l-th cardinal function of the first-kind Chebyshev interpolant
// (Eq. 12 with Eq. 13) at node l':  d1[l' nc + l] = sum_{n>=1} (alpha_n / nc) T_n(x_l) T_n'(x_l'),
// T_n' = n U_{n-1}.
static void cardinal_derivatives(int nc, const double *x, double *d1)
{
    for (int lp = 0; lp < nc; ++lp) {
        double U[HM_NC_MAX + 1];
        U[0] = 1.0;
        if (nc > 1) U[1] = 2.0 * x[lp];
        for (int j = 2; j < nc; ++j) U[j] = 2.0 * x[lp] * U[j - 1] - U[j - 2];
        for (int l = 0; l < nc; ++l) {
            double T[HM_NC_MAX];
            cheb_T(nc, x[l], T);
            double s = 0.0;
            for (int n = 1; n < nc; ++n) s += 2.0 / nc * T[n] * n * U[n - 1];
            d1[lp * nc + l] = s;
        }
    }
}

// Host geometry of a set of bodies: the node table SoA [14][nnode] (r, a_u, a_v, n,
// sqrt|G|, Fejer weight) the device computes in its node kernel.
static void host_geometry(const hm_body *bodies, int nbodies, int nc, std::vector<DevBody> &B,
                          std::vector<DevPatch> &P, std::vector<double> &x, std::vector<double> &X)
{
    const int nc2 = nc * nc;
    B.clear();
    P.clear();
    for (int b = 0; b < nbodies; ++b) {
        const hm_body &hb = bodies[b];
        if (hb.m < 1) throw HmError{HM_ERR_ARG, "bad body"};
        DevBody d{};
        for (int a = 0; a < 3; ++a) {
            d.c[a] = hb.center[a];
            for (int e = 0; e < 3; ++e) {
                d.M[3 * a + e] = hb.rot[3 * a + e] * hb.semi_axes[e];
                d.Minv[3 * a + e] = hb.rot[3 * e + a] / hb.semi_axes[a];
            }
        }
        d.m = hb.m;
        B.push_back(d);
        for (int f = 0; f < 6; ++f)
            for (int i = 0; i < hb.m; ++i)
                for (int j = 0; j < hb.m; ++j) P.push_back(DevPatch{b, f, i, j});
    }
    const int nnode = (int)P.size() * nc2;
    std::vector<double> w(nc);
    x.assign(nc, 0.0);
    cheb_nodes_host(nc, x.data());
    fejer_weights_host(nc, w.data());
    X.assign(14 * (size_t)nnode, 0.0);
    for (int id = 0; id < nnode; ++id) {
        const int pp = id / nc2, loc = id - pp * nc2, kv = loc / nc, lu = loc - kv * nc;
        double r[3], ru[3], rv[3];
        patch_eval(B[P[pp].body], P[pp], x[lu], x[kv], r, ru, rv);
        double nn[3] = {ru[1] * rv[2] - ru[2] * rv[1], ru[2] * rv[0] - ru[0] * rv[2], ru[0] * rv[1] - ru[1] * rv[0]};
        double sg = std::sqrt(nn[0] * nn[0] + nn[1] * nn[1] + nn[2] * nn[2]);
        for (int d = 0; d < 3; ++d) {
            X[(0 + d) * (size_t)nnode + id] = r[d];
            X[(3 + d) * (size_t)nnode + id] = ru[d];
            X[(6 + d) * (size_t)nnode + id] = rv[d];
            X[(9 + d) * (size_t)nnode + id] = nn[d] / sg;
        }
        X[12 * (size_t)nnode + id] = sg;
        X[13 * (size_t)nnode + id] = w[lu] * w[kv];
    }
}

static MullerMedia host_media(double k0, double eps_re, double eps_im)
{
    MullerMedia md;
    md.k = k0;
    md.epsr = zmake(eps_re, eps_im);
    // k2 = k sqrt(eps_r), the root with Im <= 0 (a decaying wave for exp(j w t))
    double mod = std::sqrt(std::sqrt(eps_re * eps_re + eps_im * eps_im));
    double arg = 0.5 * std::atan2(eps_im, eps_re);
    md.k2 = zmake(k0 * mod * std::cos(arg), k0 * mod * std::sin(arg));
    if (md.k2.y > 0) md.k2.y = -md.k2.y;
    return md;
}

// Cardinal functions ell_l(x) and derivatives at an arbitrary x (Eq. 12 with Eq. 13).
static void cardinals(int nc, const double *nodes, double x, double *ell, double *dell)
{
    double T[HM_NC_MAX], U[HM_NC_MAX + 1], Tl[HM_NC_MAX];
    cheb_T(nc, x, T);
    U[0] = 1.0;
    if (nc > 1) U[1] = 2.0 * x;
    for (int j = 2; j < nc; ++j) U[j] = 2.0 * x * U[j - 1] - U[j - 2];
    for (int l = 0; l < nc; ++l) {
        cheb_T(nc, nodes[l], Tl);
        double s = Tl[0] * T[0] / nc, ds = 0.0;
        for (int n = 1; n < nc; ++n) {
            s += 2.0 / nc * Tl[n] * T[n];
            ds += 2.0 / nc * Tl[n] * n * U[n - 1];
        }
        ell[l] = s;
        dell[l] = ds;
    }
}

// Gauss-Legendre on [0, 1], ascending.
static void gauss01(int q, std::vector<double> &x, std::vector<double> &w)
{
    std::vector<double> xx(q), ww(q);
    gauss_legendre_host(q, xx.data(), ww.data());
    std::vector<int> o(q);
    for (int i = 0; i < q; ++i) o[i] = i;
    std::sort(o.begin(), o.end(), [&](int a, int b) { return xx[a] < xx[b]; });
    x.resize(q);
    w.resize(q);
    for (int i = 0; i < q; ++i) {
        x[i] = 0.5 * (xx[o[i]] + 1.0);
        w[i] = 0.5 * ww[o[i]];
    }
}

extern "C" hm_status hm_muller_near_block_host(const hm_body *bodies, int nbodies, int nodes_per_dir, double k0,
                                               double eps_re, double eps_im, int tn, int p, int qd, int qi, int qo,
                                               double t0, void *out)
{
    if (!bodies || nbodies <= 0 || nodes_per_dir < 2 || nodes_per_dir > HM_NC_MAX || !(k0 > 0.0) || !out)
        return HM_ERR_ARG;
    if (qd <= 0) qd = 24;
    if (qi <= 0) qi = 24;
    if (qo <= 0) qo = 16;
    if (!(t0 > 0.0)) t0 = 0.5;
    if (qd > 128 || qi > 128 || qo > 128) return HM_ERR_ARG;
    try {
        const int nc = nodes_per_dir, nc2 = nc * nc;
        std::vector<DevBody> B;
        std::vector<DevPatch> P;
        std::vector<double> x1d, X;
        host_geometry(bodies, nbodies, nc, B, P, x1d, X);
        const int nnode = (int)P.size() * nc2;
        if (tn < 0 || tn >= nnode || p < 0 || p >= (int)P.size()) return HM_ERR_ARG;
        const MullerMedia md = host_media(k0, eps_re, eps_im);
        double ri[3], tu[3], tv[3];
        for (int d = 0; d < 3; ++d) {
            ri[d] = X[(0 + d) * (size_t)nnode + tn];
            tu[d] = X[(3 + d) * (size_t)nnode + tn];
            tv[d] = X[(6 + d) * (size_t)nnode + tn];
        }
        // the point of p's chart nearest the singularity (the near-field kernel's choice)
        const DevPatch &Pp = P[p];
        const DevBody &Bp = B[Pp.body];
        double uc, vc, eps;
        if (tn / nc2 == p) {
            int loc = tn - p * nc2;
            uc = x1d[loc % nc];
            vc = x1d[loc / nc];
            eps = 0.0;
        } else {
            double u0, v0;
            if (patch_chart(Bp, Pp, ri, &u0, &v0)) {
                uc = std::fmin(1.0, std::fmax(-1.0, u0));
                vc = std::fmin(1.0, std::fmax(-1.0, v0));
                eps = std::fmax(std::hypot(u0 - uc, v0 - vc), 1e-6);
            } else {
                uc = vc = 0.0;
                eps = 1.0;
            }
        }
        double r[3], ru[3], rv[3];
        patch_eval(Bp, Pp, uc, vc, r, ru, rv);
        const double gu = std::sqrt(ru[0] * ru[0] + ru[1] * ru[1] + ru[2] * ru[2]);
        const double gv = std::sqrt(rv[0] * rv[0] + rv[1] * rv[1] + rv[2] * rv[2]);
        NearPiece pieces[12];
        const int npieces = near_pieces(uc, vc, eps, gu, gv, pieces);
        std::vector<double> gdx, gdw, gix, giw, gox, gow;
        gauss01(qd, gdx, gdw);
        gauss01(qi, gix, giw);
        gauss01(qo, gox, gow);
        zc *W = (zc *)out;
        for (int i = 0; i < 16 * nc2; ++i) W[i] = zmake(0, 0);
        double lu[HM_NC_MAX], dlu[HM_NC_MAX], lv[HM_NC_MAX], dlv[HM_NC_MAX];
        zc cl[16], cd[16];
        auto accumulate = [&](double u, double v, double wt) {
            patch_eval(Bp, Pp, u, v, r, ru, rv);
            muller_point(ri, tu, tv, r, ru, rv, md, cl, cd);
            cardinals(nc, x1d.data(), u, lu, dlu);
            cardinals(nc, x1d.data(), v, lv, dlv);
            for (int c = 0; c < 16; ++c) {
                zc kl = zscale(cl[c], wt), kd = zscale(cd[c], wt);
                const int dir = c & 1;
                for (int kb = 0; kb < nc; ++kb)
                    for (int la = 0; la < nc; ++la) {
                        double ell = lu[la] * lv[kb];
                        double dl = dir == 0 ? dlu[la] * lv[kb] : lu[la] * dlv[kb];
                        zc &o = W[(size_t)c * nc2 + kb * nc + la];
                        o = zadd(o, zadd(zscale(kl, ell), zscale(kd, dl)));
                    }
            }
        };
        std::vector<double> ax(qi + qo), aw(qi + qo), bx(qi + qo), bw(qi + qo);
        for (int ip = 0; ip < npieces; ++ip) {
            const NearPiece &pc = pieces[ip];
            if (pc.type == 0) {
                int na = near_axis_points(pc.A, gix.data(), giw.data(), qi, gox.data(), gow.data(), qo, t0, ax.data(),
                                          aw.data());
                int nb = near_axis_points(pc.B, gix.data(), giw.data(), qi, gox.data(), gow.data(), qo, t0, bx.data(),
                                          bw.data());
                for (int ia = 0; ia < na; ++ia)
                    for (int ib = 0; ib < nb; ++ib) accumulate(ax[ia], bx[ib], aw[ia] * bw[ib]);
            } else {
                for (int is = 0; is < qd; ++is)
                    for (int it = 0; it < qd; ++it) {
                        double sv = gdx[is], tv2 = gdx[it];
                        double wt = std::fabs(pc.du * pc.dv) * sv * gdw[is] * gdw[it];
                        if (pc.type == 1)
                            accumulate(pc.uc + pc.du * sv, pc.vc + pc.dv * sv * tv2, wt);
                        else
                            accumulate(pc.uc + pc.du * sv * tv2, pc.vc + pc.dv * sv, wt);
                    }
            }
        }
        return HM_OK;
    } catch (const HmError &e) {
        return e.st;
    } catch (...) {
        return HM_ERR_OOM;
    }
}

extern "C" hm_status hm_muller_far_block_host(const hm_body *bodies, int nbodies, int nodes_per_dir, double k0,
                                              double eps_re, double eps_im, int tn, int p, void *out)
{
    if (!bodies || nbodies <= 0 || nodes_per_dir < 2 || nodes_per_dir > HM_NC_MAX || !(k0 > 0.0) || !out)
        return HM_ERR_ARG;
    try {
        const int nc = nodes_per_dir, nc2 = nc * nc;
        std::vector<DevBody> B;
        std::vector<DevPatch> P;
        std::vector<double> x, X;
        host_geometry(bodies, nbodies, nc, B, P, x, X);
        const int npatch = (int)P.size(), nnode = npatch * nc2;
        if (tn < 0 || tn >= nnode || p < 0 || p >= npatch) return HM_ERR_ARG;
        std::vector<double> d1((size_t)nc * nc);
        cardinal_derivatives(nc, x.data(), d1.data());
        const MullerMedia md = host_media(k0, eps_re, eps_im);
        zc *o = (zc *)out;
        zc e[16];
        for (int j = 0; j < nc2; ++j) {
            muller_far_pair(X.data(), nnode, nc, d1.data(), md, tn, p * nc2 + j, e);
            for (int c = 0; c < 16; ++c) o[(size_t)c * nc2 + j] = e[c];
        }
        return HM_OK;
    } catch (const HmError &e) {
        return e.st;
    } catch (...) {
        return HM_ERR_OOM;
    }
}

extern "C" hm_status hm_muller_rhs_farfield_host(const hm_body *bodies, int nbodies, int nodes_per_dir, double k0,
                                                 const double *khat, const double *pol, void *rhs_out, const void *x,
                                                 int nang, const double *obs, void *efar_out)
{
    if (!bodies || nbodies <= 0 || nodes_per_dir < 2 || nodes_per_dir > HM_NC_MAX || !(k0 > 0.0)) return HM_ERR_ARG;
    try {
        const int nc = nodes_per_dir;
        std::vector<DevBody> B;
        std::vector<DevPatch> P;
        std::vector<double> x1d, X;
        host_geometry(bodies, nbodies, nc, B, P, x1d, X);
        const int nnode = (int)P.size() * nc * nc;
        if (rhs_out && khat && pol) {
            zc *o = (zc *)rhs_out;
            for (int i = 0; i < nnode; ++i) muller_rhs_node(X.data(), nnode, i, k0, khat, pol, o + 4 * (size_t)i);
        }
        if (x && nang > 0 && obs && efar_out) {
            const zc *xs = (const zc *)x;
            zc *E = (zc *)efar_out;
            for (int a = 0; a < nang; ++a) {
                zc NJ[3] = {zmake(0, 0), zmake(0, 0), zmake(0, 0)}, NM[3] = {zmake(0, 0), zmake(0, 0), zmake(0, 0)};
                for (int j = 0; j < nnode; ++j) muller_radiation_add(X.data(), nnode, j, k0, obs + 3 * a, xs + 4 * j, NJ, NM);
                muller_far_field(obs + 3 * a, k0, NJ, NM, E + 3 * (size_t)a);
            }
        }
        return HM_OK;
    } catch (const HmError &e) {
        return e.st;
    } catch (...) {
        return HM_ERR_OOM;
    }
}
