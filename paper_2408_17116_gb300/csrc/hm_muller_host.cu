// Host evaluation of the N-Mueller far entries (hm_muller.cuh) for one target node
// and one source patch, with the library's own geometry: the check of that entry
// generator against an independent implementation, before the device fill uses it.
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

extern "C" hm_status hm_muller_far_block_host(const hm_body *bodies, int nbodies, int nodes_per_dir, double k0,
                                              double eps_re, double eps_im, int tn, int p, void *out)
{
    if (!bodies || nbodies <= 0 || nodes_per_dir < 2 || nodes_per_dir > HM_NC_MAX || !(k0 > 0.0) || !out)
        return HM_ERR_ARG;
    try {
        const int nc = nodes_per_dir, nc2 = nc * nc;
        std::vector<DevBody> B;
        std::vector<DevPatch> P;
        for (int b = 0; b < nbodies; ++b) {
            const hm_body &hb = bodies[b];
            if (hb.m < 1) return HM_ERR_ARG;
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
        const int npatch = (int)P.size(), nnode = npatch * nc2;
        if (tn < 0 || tn >= nnode || p < 0 || p >= npatch) return HM_ERR_ARG;
        std::vector<double> x(nc), w(nc), d1((size_t)nc * nc), X(14 * (size_t)nnode);
        cheb_nodes_host(nc, x.data());
        fejer_weights_host(nc, w.data());
        cardinal_derivatives(nc, x.data(), d1.data());
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
        MullerMedia md;
        md.k = k0;
        md.epsr = zmake(eps_re, eps_im);
        // k2 = k sqrt(eps_r), the root with Im <= 0 (a decaying wave for exp(j w t))
        double mod = std::sqrt(std::sqrt(eps_re * eps_re + eps_im * eps_im));
        double arg = 0.5 * std::atan2(eps_im, eps_re);
        md.k2 = zmake(k0 * mod * std::cos(arg), k0 * mod * std::sin(arg));
        if (md.k2.y > 0) md.k2.y = -md.k2.y;
        zc *o = (zc *)out;
        zc e[16];
        for (int j = 0; j < nc2; ++j) {
            muller_far_pair(X.data(), nnode, nc, d1.data(), md, tn, p * nc2 + j, e);
            for (int c = 0; c < 16; ++c) o[(size_t)c * nc2 + j] = e[c];
        }
        return HM_OK;
    } catch (...) {
        return HM_ERR_OOM;
    }
}
