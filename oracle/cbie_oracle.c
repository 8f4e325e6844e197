/*
 * CBIE / MFIE oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 CPU implementation of what the solver computes, used only by
 * tests/, the smoke check and the CPU-baseline leg of the benchmark.  It shares no
 * code, header, table or helper with the CUDA library; the product path never
 * calls it.
 *
 * What it defines (paper: arXiv 2408.17116):
 *   - cube-mapped ellipsoid patches r^p(u,v), covariant basis a_u, a_v, unit normal
 *     and Jacobian sqrt|G| (Sec. II.B, Eq. 11 and Eq. 14);
 *   - first-kind Chebyshev nodes, Fejer's first quadrature rule, and the
 *     Chebyshev interpolant of nodal values built from Eq. 12 with the discrete
 *     transform of Eq. 13;
 *   - the MFIE for a PEC body (Eq. 10, second row) tested with sqrt|G| a^b
 *     (Eqs. 17-18): far entries by the Nystrom/Fejer rule, self and near entries as
 *     the exact integrals of kernel x Chebyshev interpolant (Eq. 20), the identity
 *     term 1/2 from the jump relation (Eq. 5);
 *   - the dense matrix, dense LU with partial pivoting (LAPACK semantics, ties to
 *     the lowest row), forward/back substitution;
 *   - plane-wave right-hand sides (Eq. 19/22 rows) and the far field / RCS.
 *
 * Readings where the paper is silent or garbled (each also listed in the design
 * notes):
 *   - MFIE sign: the standard form J/2 - n x PV(grad G x J) = n x H_inc derived from
 *     Eqs. 1, 2 and 5 (the printed Eq. 10 carries the opposite sign on the n x curl S
 *     term);  row u:  F^u/2 + a_v . K = -a_v . H_inc,   row v:  F^v/2 - a_u . K = a_u . H_inc;
 *   - Fejer's first rule uses first-kind nodes (no endpoints); in Eq. 13 the second
 *     argument is v_k and alpha_0 = 1, alpha_n = 2 for n >= 1;
 *   - near pair (q,p): q == p, or dist(bbox_q, bbox_p) < delta * max(diam_q, diam_p),
 *     bboxes over the (Nc+2)^2 grid {-1, nodes, +1}^2 of each patch;
 *   - the self/near integrals are computed here by an independent method: an
 *     adaptive quadtree on the parameter square driven by 3-D distance to the
 *     target, Gauss-Legendre on every accepted box, and the Duffy transformation on
 *     rectangles that have the singular node at a corner (self patches).
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

#define OR_PI 3.14159265358979323846

/* ------------------------------------------------------------------------- */
/* 1-D rules                                                                  */
/* ------------------------------------------------------------------------- */

/* First-kind Chebyshev nodes u_l = cos(pi (2l+1) / (2N)), l = 0..N-1 (Sec. II.B). */
void or_cheb_nodes(int n, double *x)
{
    for (int l = 0; l < n; ++l) x[l] = cos(OR_PI * (2.0 * l + 1.0) / (2.0 * n));
}

/* Fejer's first rule on [-1,1] at the first-kind nodes (Sec. II.B):
 * w_l = (2/N) [1 - 2 sum_{s=1}^{floor(N/2)} cos(2 s theta_l) / (4 s^2 - 1)]. */
void or_fejer_weights(int n, double *w)
{
    for (int l = 0; l < n; ++l) {
        double th = OR_PI * (2.0 * l + 1.0) / (2.0 * n);
        double s = 0.0;
        for (int j = 1; j <= n / 2; ++j) s += cos(2.0 * j * th) / (4.0 * j * j - 1.0);
        w[l] = (2.0 / n) * (1.0 - 2.0 * s);
    }
}

/* Gauss-Legendre nodes and weights on [-1,1] by Newton iteration on P_q. */
void or_gauss_legendre(int q, double *x, double *w)
{
    for (int i = 0; i < q; ++i) {
        double z = cos(OR_PI * (i + 0.75) / (q + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int n = 2; n <= q; ++n) {
                double p2 = ((2.0 * n - 1.0) * z * p1 - (n - 1.0) * p0) / n;
                p0 = p1;
                p1 = p2;
            }
            if (q == 1) { p1 = z; p0 = 1.0; }
            dp = q * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        double p0 = 1.0, p1 = z;
        for (int n = 2; n <= q; ++n) {
            double p2 = ((2.0 * n - 1.0) * z * p1 - (n - 1.0) * p0) / n;
            p0 = p1;
            p1 = p2;
        }
        if (q == 1) { p1 = z; p0 = 1.0; }
        dp = q * (z * p1 - p0) / (z * z - 1.0);
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

/* Cardinal functions of the Chebyshev interpolant: with Eq. 13 substituted into
 * Eq. 12, F(x) = sum_l F(x_l) ell_l(x) where
 *   ell_l(x) = sum_{n=0}^{N-1} (alpha_n / N) T_n(x_l) T_n(x),  alpha_0 = 1, alpha_n = 2. */
static void cheb_T(int n, double x, double *t)
{
    t[0] = 1.0;
    if (n > 1) t[1] = x;
    for (int j = 2; j < n; ++j) t[j] = 2.0 * x * t[j - 1] - t[j - 2];
}

void or_cheb_cardinal(int n, const double *nodes, double x, double *ell)
{
    double tx[64], tl[64];
    cheb_T(n, x, tx);
    for (int l = 0; l < n; ++l) {
        cheb_T(n, nodes[l], tl);
        double s = tl[0] * tx[0] / n;
        for (int j = 1; j < n; ++j) s += 2.0 * tl[j] * tx[j] / n;
        ell[l] = s;
    }
}

/* ------------------------------------------------------------------------- */
/* Geometry: cube-mapped ellipsoid patches                                    */
/* ------------------------------------------------------------------------- */

/* Face frames (e_f, e1, e2) with e1 x e2 = e_f so that a_u x a_v points outward. */
static const double FACE_N[6][3] = {{1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};
static const double FACE_E1[6][3] = {{0, 1, 0}, {0, 0, 1}, {0, 0, 1}, {1, 0, 0}, {1, 0, 0}, {0, 1, 0}};
static const double FACE_E2[6][3] = {{0, 0, 1}, {0, 1, 0}, {1, 0, 0}, {0, 0, 1}, {0, 1, 0}, {1, 0, 0}};

typedef struct {
    double center[3];
    double semi[3];
    double rot[9]; /* row-major rotation */
    int m;         /* patches per cube-face edge */
} or_body;

static void cross3(const double *a, const double *b, double *c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static double norm3(const double *a) { return sqrt(dot3(a, a)); }

/* r^p(u,v) and its covariant basis a_u = dr/du, a_v = dr/dv (Eq. 14).
 * Face f, sub-square (i,j) of m x m; s = -1 + (2i+1+u)/m, t = -1 + (2j+1+v)/m,
 * equiangular S = tan(pi s / 4), T = tan(pi t / 4), c = e_f + S e1 + T e2,
 * r = center + Rot diag(semi) c/|c|. */
static void body_map(const or_body *b, int f, int i, int j, double u, double v, double *r, double *ru, double *rv)
{
    double m = (double)b->m;
    double s = -1.0 + (2.0 * i + 1.0 + u) / m;
    double t = -1.0 + (2.0 * j + 1.0 + v) / m;
    double S = tan(OR_PI * s / 4.0), T = tan(OR_PI * t / 4.0);
    double dS = (OR_PI / 4.0) * (1.0 + S * S) / m;
    double dT = (OR_PI / 4.0) * (1.0 + T * T) / m;
    double c[3], cu[3], cv[3];
    for (int d = 0; d < 3; ++d) {
        c[d] = FACE_N[f][d] + S * FACE_E1[f][d] + T * FACE_E2[f][d];
        cu[d] = dS * FACE_E1[f][d];
        cv[d] = dT * FACE_E2[f][d];
    }
    double nc = norm3(c);
    double xh[3], xu[3], xv[3];
    double ccu = dot3(c, cu), ccv = dot3(c, cv);
    for (int d = 0; d < 3; ++d) {
        xh[d] = c[d] / nc;
        xu[d] = cu[d] / nc - c[d] * ccu / (nc * nc * nc);
        xv[d] = cv[d] / nc - c[d] * ccv / (nc * nc * nc);
    }
    /* apply Rot diag(semi) */
    for (int a = 0; a < 3; ++a) {
        double sr = 0, su = 0, sv = 0;
        for (int d = 0; d < 3; ++d) {
            double md = b->rot[3 * a + d] * b->semi[d];
            sr += md * xh[d];
            su += md * xu[d];
            sv += md * xv[d];
        }
        r[a] = b->center[a] + sr;
        ru[a] = su;
        rv[a] = sv;
    }
}

/* ------------------------------------------------------------------------- */
/* Oracle context                                                             */
/* ------------------------------------------------------------------------- */

typedef struct {
    int nbodies;
    or_body *bodies;
    int nc;            /* nodes per patch direction */
    int npatch;
    int *pbody, *pface, *pi, *pj; /* per patch */
    double k;          /* wavenumber */
    double eta0;
    double delta;      /* near criterion */
    double *nodes1d, *fejer;
    /* node table */
    int nnode;
    double *nr, *nau, *nav, *nn, *nsg, *nw;
    /* patch bboxes, near flags */
    double *bbmin, *bbmax;
    unsigned char *near;
    /* quadrature orders of the independent near integrator */
    int q, qd;
    double *glx, *glw, *gdx, *gdw; /* on [0,1] */
    double accept;     /* box acceptance ratio: dist >= accept * radius */
    /* dielectric body (N-Mueller formulation): relative permittivity of the interior and
     * its wavenumber k2 = k sqrt(eps_r); mu_r = 1 */
    int dielectric;
    cplx epsr, k2;
    /* PEC combined field equation: weight alpha of the EFIE row, and the 1-D spectral
     * differentiation matrix dmat[l * nc + l'] = ell_{l'}'(x_l) */
    int cfie;
    double alpha;
    double *dmat;
} or_ctx;

static void ctx_patch_map(const or_ctx *c, int p, double u, double v, double *r, double *ru, double *rv)
{
    body_map(&c->bodies[c->pbody[p]], c->pface[p], c->pi[p], c->pj[p], u, v, r, ru, rv);
}

void or_destroy(or_ctx *c);

/* bodies: nbodies x 15 doubles (center[3], semi-axes[3], rotation[9] row-major), ms: m per body. */
or_ctx *or_create(int nbodies, const double *bodies, const int *ms, int nc, double k, double delta, int q, int qd)
{
    if (nbodies <= 0 || nc < 2 || nc > 48) return NULL;
    or_ctx *c = (or_ctx *)calloc(1, sizeof(or_ctx));
    c->nbodies = nbodies;
    c->bodies = (or_body *)calloc(nbodies, sizeof(or_body));
    c->npatch = 0;
    for (int b = 0; b < nbodies; ++b) {
        memcpy(c->bodies[b].center, bodies + 15 * b, 3 * sizeof(double));
        memcpy(c->bodies[b].semi, bodies + 15 * b + 3, 3 * sizeof(double));
        memcpy(c->bodies[b].rot, bodies + 15 * b + 6, 9 * sizeof(double));
        c->bodies[b].m = ms[b];
        c->npatch += 6 * ms[b] * ms[b];
    }
    c->nc = nc;
    c->k = k;
    c->eta0 = sqrt(1.25663706212e-6 / 8.8541878128e-12);
    c->delta = delta;
    c->pbody = (int *)malloc(sizeof(int) * c->npatch);
    c->pface = (int *)malloc(sizeof(int) * c->npatch);
    c->pi = (int *)malloc(sizeof(int) * c->npatch);
    c->pj = (int *)malloc(sizeof(int) * c->npatch);
    int p = 0;
    for (int b = 0; b < nbodies; ++b)
        for (int f = 0; f < 6; ++f)
            for (int i = 0; i < ms[b]; ++i)
                for (int j = 0; j < ms[b]; ++j) {
                    c->pbody[p] = b;
                    c->pface[p] = f;
                    c->pi[p] = i;
                    c->pj[p] = j;
                    ++p;
                }
    c->nodes1d = (double *)malloc(sizeof(double) * nc);
    c->fejer = (double *)malloc(sizeof(double) * nc);
    or_cheb_nodes(nc, c->nodes1d);
    or_fejer_weights(nc, c->fejer);
    c->nnode = c->npatch * nc * nc;
    int nn = c->nnode;
    c->nr = (double *)malloc(sizeof(double) * 3 * nn);
    c->nau = (double *)malloc(sizeof(double) * 3 * nn);
    c->nav = (double *)malloc(sizeof(double) * 3 * nn);
    c->nn = (double *)malloc(sizeof(double) * 3 * nn);
    c->nsg = (double *)malloc(sizeof(double) * nn);
    c->nw = (double *)malloc(sizeof(double) * nn);
    for (int pp = 0; pp < c->npatch; ++pp)
        for (int kv = 0; kv < nc; ++kv)
            for (int lu = 0; lu < nc; ++lu) {
                int id = (pp * nc + kv) * nc + lu;
                double cr[3];
                ctx_patch_map(c, pp, c->nodes1d[lu], c->nodes1d[kv], c->nr + 3 * id, c->nau + 3 * id, c->nav + 3 * id);
                cross3(c->nau + 3 * id, c->nav + 3 * id, cr);
                double sg = norm3(cr);
                c->nsg[id] = sg;
                for (int d = 0; d < 3; ++d) c->nn[3 * id + d] = cr[d] / sg;
                c->nw[id] = c->fejer[lu] * c->fejer[kv];
            }
    /* patch bboxes over the grid {-1, nodes, +1}^2 */
    c->bbmin = (double *)malloc(sizeof(double) * 3 * c->npatch);
    c->bbmax = (double *)malloc(sizeof(double) * 3 * c->npatch);
    double *g = (double *)malloc(sizeof(double) * (nc + 2));
    g[0] = -1.0;
    for (int l = 0; l < nc; ++l) g[l + 1] = c->nodes1d[l];
    g[nc + 1] = 1.0;
    for (int pp = 0; pp < c->npatch; ++pp) {
        for (int d = 0; d < 3; ++d) {
            c->bbmin[3 * pp + d] = 1e300;
            c->bbmax[3 * pp + d] = -1e300;
        }
        for (int a = 0; a < nc + 2; ++a)
            for (int b2 = 0; b2 < nc + 2; ++b2) {
                double r[3], ru[3], rv[3];
                ctx_patch_map(c, pp, g[a], g[b2], r, ru, rv);
                for (int d = 0; d < 3; ++d) {
                    if (r[d] < c->bbmin[3 * pp + d]) c->bbmin[3 * pp + d] = r[d];
                    if (r[d] > c->bbmax[3 * pp + d]) c->bbmax[3 * pp + d] = r[d];
                }
            }
    }
    free(g);
    c->near = (unsigned char *)calloc((size_t)c->npatch * c->npatch, 1);
    for (int qq = 0; qq < c->npatch; ++qq)
        for (int pp = 0; pp < c->npatch; ++pp) {
            double dist2 = 0, dq = 0, dp = 0;
            for (int d = 0; d < 3; ++d) {
                double gap = fmax(0.0, fmax(c->bbmin[3 * qq + d] - c->bbmax[3 * pp + d], c->bbmin[3 * pp + d] - c->bbmax[3 * qq + d]));
                dist2 += gap * gap;
                double eq = c->bbmax[3 * qq + d] - c->bbmin[3 * qq + d];
                double ep = c->bbmax[3 * pp + d] - c->bbmin[3 * pp + d];
                dq += eq * eq;
                dp += ep * ep;
            }
            double diam = sqrt(fmax(dq, dp));
            c->near[(size_t)qq * c->npatch + pp] = (qq == pp) || (sqrt(dist2) < delta * diam);
        }
    c->q = q;
    c->qd = qd;
    c->glx = (double *)malloc(sizeof(double) * q);
    c->glw = (double *)malloc(sizeof(double) * q);
    c->gdx = (double *)malloc(sizeof(double) * qd);
    c->gdw = (double *)malloc(sizeof(double) * qd);
    or_gauss_legendre(q, c->glx, c->glw);
    or_gauss_legendre(qd, c->gdx, c->gdw);
    for (int i = 0; i < q; ++i) { c->glx[i] = 0.5 * (c->glx[i] + 1.0); c->glw[i] *= 0.5; }
    for (int i = 0; i < qd; ++i) { c->gdx[i] = 0.5 * (c->gdx[i] + 1.0); c->gdw[i] *= 0.5; }
    c->accept = 3.0;
    return c;
}

void or_destroy(or_ctx *c)
{
    if (!c) return;
    free(c->bodies); free(c->pbody); free(c->pface); free(c->pi); free(c->pj);
    free(c->nodes1d); free(c->fejer); free(c->dmat);
    free(c->nr); free(c->nau); free(c->nav); free(c->nn); free(c->nsg); free(c->nw);
    free(c->bbmin); free(c->bbmax); free(c->near);
    free(c->glx); free(c->glw); free(c->gdx); free(c->gdw);
    free(c);
}

int or_num_patches(const or_ctx *c) { return c->npatch; }
int or_num_nodes(const or_ctx *c) { return c->nnode; }

/* Node table, 17 doubles per node: r[3], a_u[3], a_v[3], n[3], sqrtG, w, u, v, patch. */
void or_node_table(const or_ctx *c, double *out)
{
    int nc = c->nc;
    for (int id = 0; id < c->nnode; ++id) {
        double *o = out + 17 * id;
        for (int d = 0; d < 3; ++d) {
            o[d] = c->nr[3 * id + d];
            o[3 + d] = c->nau[3 * id + d];
            o[6 + d] = c->nav[3 * id + d];
            o[9 + d] = c->nn[3 * id + d];
        }
        o[12] = c->nsg[id];
        o[13] = c->nw[id];
        int lu = id % nc, kv = (id / nc) % nc;
        o[14] = c->nodes1d[lu];
        o[15] = c->nodes1d[kv];
        o[16] = (double)(id / (nc * nc));
    }
}

void or_near_flags(const or_ctx *c, unsigned char *out) { memcpy(out, c->near, (size_t)c->npatch * c->npatch); }

/* Evaluate the patch map at (u,v) for tests. */
void or_patch_point(const or_ctx *c, int p, double u, double v, double *r, double *ru, double *rv)
{
    ctx_patch_map(c, p, u, v, r, ru, rv);
}

/* ------------------------------------------------------------------------- */
/* Kernels                                                                    */
/* ------------------------------------------------------------------------- */

enum { KIND_SINGLE = 0, KIND_MFIE = 1, KIND_MULLER = 2, KIND_EVEC = 3, KIND_SCALAR = 4 };

typedef struct {
    const or_ctx *c;
    int kind;      /* KIND_SINGLE: G sqrtG (single-layer, Eq. 3); KIND_MFIE: 4 tested components;
                      KIND_MULLER: 16 components (4 tested rows x 4 source currents) */
    double kbox;   /* wavenumber that sizes the adaptive boxes (the largest of the media) */
    int p;         /* source patch */
    double k;
    double tgt[3], tu[3], tv[3];
    int ncomp;
    double te[2][3];  /* KIND_EVEC: the target's test vectors sqrtG a^u, sqrtG a^v (Eqs. 17-18) */
    cplx *W;       /* ncomp x nc^2, index [comp][kv*nc + lu] */
    /* planar test map (used when p < 0): r = (a u, b v, 0) */
    double pa, pb;
} integ;

static void integ_map(const integ *ig, double u, double v, double *r, double *ru, double *rv)
{
    if (ig->p >= 0) {
        ctx_patch_map(ig->c, ig->p, u, v, r, ru, rv);
    } else {
        r[0] = ig->pa * u; r[1] = ig->pb * v; r[2] = 0.0;
        ru[0] = ig->pa; ru[1] = 0; ru[2] = 0;
        rv[0] = 0; rv[1] = ig->pb; rv[2] = 0;
    }
}

/* Cardinal functions ell_l(x) (Eq. 12 with Eq. 13) and their derivatives:
 * ell_l'(x) = sum_{n>=1} (alpha_n / N) T_n(x_l) T_n'(x),  T_n' = n U_{n-1}. */
static void cheb_cardinal_d(int n, const double *nodes, double x, double *ell, double *dell)
{
    double tx[64], dtx[64], tl[64], ux[64];
    cheb_T(n, x, tx);
    ux[0] = 1.0;
    if (n > 1) ux[1] = 2.0 * x;
    for (int j = 2; j < n; ++j) ux[j] = 2.0 * x * ux[j - 1] - ux[j - 2];
    dtx[0] = 0.0;
    for (int j = 1; j < n; ++j) dtx[j] = j * ux[j - 1];
    for (int l = 0; l < n; ++l) {
        cheb_T(n, nodes[l], tl);
        double s = tl[0] * tx[0] / n, ds = 0.0;
        for (int j = 1; j < n; ++j) {
            s += 2.0 * tl[j] * tx[j] / n;
            ds += 2.0 * tl[j] * dtx[j] / n;
        }
        ell[l] = s;
        dell[l] = ds;
    }
}

/* N-Mueller integrand at one source point r' = r_p(u,v) for target r_i (Sec. II.A,
 * Eqs. 2, 7-9 with alpha = -eps_r, beta = -1), tested with sqrt|G| a^b (Eqs. 17-18),
 * i.e. with t_u = -a_v(r_i), t_v = a_u(r_i) applied to the vector inside n x [ ].
 * Unknowns (dimensionless scaling): Jbar = eta0 J and M, both as F^a = sqrt|G| x
 * contravariant component (Eq. 11).  Kernels, R = r_i - r':
 *   K_S = G1 - eps_r G2,  grad(G1 - G2) = gD R,  grad(G1 - eps_r G2) = gE R,
 *   g_k = -(1 + j k R) exp(-j k R) / (4 pi R^3)  (grad G_k = g_k R, Eq. 4).
 * Component [row][col], rows (E-u, E-v, H-u, H-v), cols (J^u, J^v, M^u, M^v):
 *   E-row b, J^a:  j k K_S (t_b.a_a) ell - (1/(j k)) gD (t_b.R) d_a ell
 *   E-row b, M^a:  gE t_b.(R x a_a) ell
 *   H-row b, J^a: -gD t_b.(R x a_a) ell
 *   H-row b, M^a:  j k K_S (t_b.a_a) ell - (1/(j k)) gD (t_b.R) d_a ell
 * (the difference kernels carry the cancellation of the strong singularity). */
static void muller_point(integ *ig, const double *r, const double *ru, const double *rv, double u, double v,
                         double wt)
{
    const or_ctx *c = ig->c;
    double d[3] = {ig->tgt[0] - r[0], ig->tgt[1] - r[1], ig->tgt[2] - r[2]};
    double R = norm3(d);
    double k = ig->k;
    cplx k2 = c->k2, er = c->epsr;
    cplx e1 = cexp(-I * k * R), e2 = cexp(-I * k2 * R);
    cplx G1 = e1 / (4.0 * OR_PI * R), G2 = e2 / (4.0 * OR_PI * R);
    cplx g1 = -(1.0 + I * k * R) * e1 / (4.0 * OR_PI * R * R * R);
    cplx g2 = -(1.0 + I * k2 * R) * e2 / (4.0 * OR_PI * R * R * R);
    cplx KS = G1 - er * G2, gD = g1 - g2, gE = g1 - er * g2;
    double t[2][3], a[2][3];
    for (int q = 0; q < 3; ++q) {
        t[0][q] = -ig->tv[q];
        t[1][q] = ig->tu[q];
        a[0][q] = ru[q];
        a[1][q] = rv[q];
    }
    cplx cl[16], cd[16];
    for (int b = 0; b < 2; ++b) {
        double tR = dot3(t[b], d);
        for (int aa = 0; aa < 2; ++aa) {
            double ta = dot3(t[b], a[aa]);
            double cr[3];
            cross3(d, a[aa], cr);
            double tc = dot3(t[b], cr);
            cplx sl = I * k * KS * ta, sd = -(1.0 / (I * k)) * gD * tR;
            cl[(0 + b) * 4 + aa] = sl;           /* E-row b, J^a */
            cd[(0 + b) * 4 + aa] = sd;
            cl[(0 + b) * 4 + 2 + aa] = gE * tc;  /* E-row b, M^a */
            cd[(0 + b) * 4 + 2 + aa] = 0;
            cl[(2 + b) * 4 + aa] = -gD * tc;     /* H-row b, J^a */
            cd[(2 + b) * 4 + aa] = 0;
            cl[(2 + b) * 4 + 2 + aa] = sl;       /* H-row b, M^a */
            cd[(2 + b) * 4 + 2 + aa] = sd;
        }
    }
    int nc = c->nc;
    double lu[64], dlu[64], lv[64], dlv[64];
    cheb_cardinal_d(nc, c->nodes1d, u, lu, dlu);
    cheb_cardinal_d(nc, c->nodes1d, v, lv, dlv);
    for (int cmp = 0; cmp < 16; ++cmp) {
        cplx kl = cl[cmp] * wt, kd = cd[cmp] * wt;
        int src_dir = cmp & 1; /* a = u (0) or v (1): the derivative of the divergence term */
        cplx *Wc = ig->W + (size_t)cmp * nc * nc;
        for (int kb = 0; kb < nc; ++kb)
            for (int la = 0; la < nc; ++la) {
                double dl = src_dir == 0 ? dlu[la] * lv[kb] : lu[la] * dlv[kb];
                Wc[kb * nc + la] += kl * lu[la] * lv[kb] + kd * dl;
            }
    }
}

/* Accumulate one quadrature point (u,v) with weight wt. */
static void integ_point(integ *ig, double u, double v, double wt)
{
    double r[3], ru[3], rv[3];
    integ_map(ig, u, v, r, ru, rv);
    if (ig->kind == KIND_MULLER) {
        muller_point(ig, r, ru, rv, u, v, wt);
        return;
    }
    double d[3] = {ig->tgt[0] - r[0], ig->tgt[1] - r[1], ig->tgt[2] - r[2]};
    double R = norm3(d);
    cplx kv[4];
    if (ig->kind == KIND_EVEC || ig->kind == KIND_SCALAR) {
        /* G(R) t_b . a_a (vector potential part of the EFIE, tested), or G(R) alone (the
         * scalar potential of the surface divergence); no Jacobian: J dS' = F^a a_a du dv
         * and (div J) dS' = (d_u F^u + d_v F^v) du dv */
        cplx G = cexp(-I * ig->k * R) / (4.0 * OR_PI * R);
        if (ig->kind == KIND_SCALAR) {
            kv[0] = G;
        } else {
            kv[0] = G * dot3(ig->te[0], ru);
            kv[1] = G * dot3(ig->te[0], rv);
            kv[2] = G * dot3(ig->te[1], ru);
            kv[3] = G * dot3(ig->te[1], rv);
        }
    } else if (ig->kind == KIND_SINGLE) {
        double cr[3];
        cross3(ru, rv, cr);
        /* G(R) = exp(-jkR) / (4 pi R)  (Eq. 4), times the surface Jacobian */
        kv[0] = cexp(-I * ig->k * R) / (4.0 * OR_PI * R) * norm3(cr);
    } else {
        /* grad_r G = g(R) (r - r'),  g = -(1 + jkR) exp(-jkR) / (4 pi R^3) */
        cplx g = -(1.0 + I * ig->k * R) * cexp(-I * ig->k * R) / (4.0 * OR_PI * R * R * R);
        double cu[3], cv[3];
        cross3(d, ru, cu);
        cross3(d, rv, cv);
        kv[0] = g * dot3(ig->tv, cu);
        kv[1] = g * dot3(ig->tv, cv);
        kv[2] = -g * dot3(ig->tu, cu);
        kv[3] = -g * dot3(ig->tu, cv);
    }
    int nc = ig->c->nc;
    double lu[64], lv[64];
    or_cheb_cardinal(nc, ig->c->nodes1d, u, lu);
    or_cheb_cardinal(nc, ig->c->nodes1d, v, lv);
    for (int cmp = 0; cmp < ig->ncomp; ++cmp) {
        cplx kw = kv[cmp] * wt;
        cplx *Wc = ig->W + (size_t)cmp * nc * nc;
        for (int b = 0; b < nc; ++b)
            for (int a = 0; a < nc; ++a) Wc[b * nc + a] += kw * lu[a] * lv[b];
    }
}

/* Tensor Gauss-Legendre on [u0,u1] x [v0,v1]. */
static void integ_gl_box(integ *ig, double u0, double u1, double v0, double v1)
{
    const or_ctx *c = ig->c;
    double hu = u1 - u0, hv = v1 - v0;
    for (int a = 0; a < c->q; ++a)
        for (int b = 0; b < c->q; ++b)
            integ_point(ig, u0 + hu * c->glx[a], v0 + hv * c->glx[b], fabs(hu * hv) * c->glw[a] * c->glw[b]);
}

/* Adaptive quadtree box: accept when the target is at least `accept` box radii
 * away (3-D) and the box is at most 1.5/k in radius; otherwise split in four. */
static void integ_box(integ *ig, double u0, double u1, double v0, double v1, int depth)
{
    if (u1 < u0) { double t = u0; u0 = u1; u1 = t; }
    if (v1 < v0) { double t = v0; v0 = v1; v1 = t; }
    if (u1 - u0 <= 0 || v1 - v0 <= 0) return;
    double uc = 0.5 * (u0 + u1), vc = 0.5 * (v0 + v1);
    double rc[3], ru[3], rv[3];
    integ_map(ig, uc, vc, rc, ru, rv);
    double rad = 0.0;
    double us[8] = {u0, u1, u0, u1, uc, uc, u0, u1};
    double vs[8] = {v0, v0, v1, v1, v0, v1, vc, vc};
    for (int i = 0; i < 8; ++i) {
        double r[3];
        integ_map(ig, us[i], vs[i], r, ru, rv);
        double dd[3] = {r[0] - rc[0], r[1] - rc[1], r[2] - rc[2]};
        double e = norm3(dd);
        if (e > rad) rad = e;
    }
    double dt[3] = {ig->tgt[0] - rc[0], ig->tgt[1] - rc[1], ig->tgt[2] - rc[2]};
    double dist = norm3(dt);
    int ok = (depth >= 1) && (dist >= ig->c->accept * rad) && (ig->kbox * rad <= 1.5);
    if (ok || depth >= 40) {
        integ_gl_box(ig, u0, u1, v0, v1);
        return;
    }
    integ_box(ig, u0, uc, v0, vc, depth + 1);
    integ_box(ig, uc, u1, v0, vc, depth + 1);
    integ_box(ig, u0, uc, vc, v1, depth + 1);
    integ_box(ig, uc, u1, vc, v1, depth + 1);
}

/* Duffy transformation on the rectangle with corner (uc,vc) (the singular point)
 * spanning signed lengths du, dv.  Two triangles, each mapped from the unit
 * square with Jacobian |du dv| s, which removes the 1/R singularity. */
static void integ_duffy(integ *ig, double uc, double vc, double du, double dv)
{
    const or_ctx *c = ig->c;
    double A = fabs(du * dv);
    for (int a = 0; a < c->qd; ++a) {
        double s = c->gdx[a];
        for (int b = 0; b < c->qd; ++b) {
            double t = c->gdx[b];
            double wt = A * s * c->gdw[a] * c->gdw[b];
            integ_point(ig, uc + du * s, vc + dv * s * t, wt);
            integ_point(ig, uc + du * s * t, vc + dv * s, wt);
        }
    }
}

/* Rectangle with the singular point at a corner: peel off strips until the
 * physical aspect ratio (side lengths measured with |a_u|, |a_v| at the corner) is
 * at most 2, then Duffy; strips go to the adaptive quadtree. */
static void integ_corner_rect(integ *ig, double uc, double vc, double du, double dv)
{
    if (du == 0 || dv == 0) return;
    double r[3], ru[3], rv[3];
    integ_map(ig, uc, vc, r, ru, rv);
    double gu = norm3(ru), gv = norm3(rv);
    double a = fabs(du) * gu, b = fabs(dv) * gv;
    double su = du > 0 ? 1.0 : -1.0, sv = dv > 0 ? 1.0 : -1.0;
    if (b > 2.0 * a) {
        double dv1 = sv * a / gv;
        integ_corner_rect(ig, uc, vc, du, dv1);
        integ_box(ig, uc, uc + du, vc + dv1, vc + dv, 1);
        return;
    }
    if (a > 2.0 * b) {
        double du1 = su * b / gu;
        integ_corner_rect(ig, uc, vc, du1, dv);
        integ_box(ig, uc + du1, uc + du, vc, vc + dv, 1);
        return;
    }
    /* the Duffy square must resolve the kernel's oscillation: larger than 1.5/k in
     * physical size, it shrinks to that size at the corner and the rest of the
     * rectangle goes to the adaptive boxes */
    double side = fmax(a, b);
    if (ig->kbox * side > 1.5) {
        double f = 1.5 / (ig->kbox * side);
        double du1 = du * f, dv1 = dv * f;
        integ_corner_rect(ig, uc, vc, du1, dv1);
        integ_box(ig, uc + du1, uc + du, vc, vc + dv, 1);
        integ_box(ig, uc, uc + du1, vc + dv1, vc + dv, 1);
        return;
    }
    integ_duffy(ig, uc, vc, du, dv);
}

/* Integrals of kernel x cardinal function over source patch p for one target.
 * self_lu/self_kv >= 0: the target is node (self_lu, self_kv) of patch p. */
static void integ_patch(integ *ig, int self_lu, int self_kv)
{
    int nc = ig->c->nc;
    memset(ig->W, 0, sizeof(cplx) * ig->ncomp * nc * nc);
    if (self_lu >= 0) {
        double us = ig->c->nodes1d[self_lu], vs = ig->c->nodes1d[self_kv];
        integ_corner_rect(ig, us, vs, 1.0 - us, 1.0 - vs);
        integ_corner_rect(ig, us, vs, -1.0 - us, 1.0 - vs);
        integ_corner_rect(ig, us, vs, 1.0 - us, -1.0 - vs);
        integ_corner_rect(ig, us, vs, -1.0 - us, -1.0 - vs);
    } else {
        integ_box(ig, -1.0, 1.0, -1.0, 1.0, 0);
    }
}

/* Self/near MFIE integrals for target node `tn` over source patch p:
 * W[(2b+a) * nc^2 + j] = integral over [-1,1]^2 of K_ba(r_tn, r_p(u,v)) ell_j(u,v) du dv,
 * b = tested row component (u,v), a = source current component (u,v)  (Eq. 20). */
void or_near_block(const or_ctx *c, int tn, int p, cplx *W)
{
    integ ig;
    memset(&ig, 0, sizeof(ig));
    ig.c = c;
    ig.kind = KIND_MFIE;
    ig.p = p;
    ig.k = c->k;
    ig.kbox = c->k;
    ig.ncomp = 4;
    ig.W = W;
    for (int d = 0; d < 3; ++d) {
        ig.tgt[d] = c->nr[3 * tn + d];
        ig.tu[d] = c->nau[3 * tn + d];
        ig.tv[d] = c->nav[3 * tn + d];
    }
    int nc = c->nc;
    int tp = tn / (nc * nc);
    if (tp == p)
        integ_patch(&ig, tn % nc, (tn / nc) % nc);
    else
        integ_patch(&ig, -1, -1);
}

/* Single-layer weights (Eq. 3) for target node tn over patch p: W[j] = int G sqrtG ell_j. */
void or_single_layer_block(const or_ctx *c, int tn, int p, cplx *W)
{
    integ ig;
    memset(&ig, 0, sizeof(ig));
    ig.c = c;
    ig.kind = KIND_SINGLE;
    ig.p = p;
    ig.k = c->k;
    ig.kbox = c->k;
    ig.ncomp = 1;
    ig.W = W;
    for (int d = 0; d < 3; ++d) ig.tgt[d] = c->nr[3 * tn + d];
    int nc = c->nc;
    int tp = tn / (nc * nc);
    if (tp == p)
        integ_patch(&ig, tn % nc, (tn / nc) % nc);
    else
        integ_patch(&ig, -1, -1);
}

/* Test hook for the integrator alone: planar patch r = (a u, b v, 0), kernel
 * G sqrtG with wavenumber k, target tgt; self_lu >= 0 marks the target as that node.
 * Uses nc cardinal functions of the context. */
void or_planar_single_layer(const or_ctx *c, double a, double b, double k, const double *tgt, int self_lu, int self_kv, cplx *W)
{
    integ ig;
    memset(&ig, 0, sizeof(ig));
    ig.c = c;
    ig.kind = KIND_SINGLE;
    ig.p = -1;
    ig.pa = a;
    ig.pb = b;
    ig.k = k;
    ig.kbox = k;
    ig.ncomp = 1;
    ig.W = W;
    for (int d = 0; d < 3; ++d) ig.tgt[d] = tgt[d];
    integ_patch(&ig, self_lu, self_kv);
}

/* ------------------------------------------------------------------------- */
/* Matrix rows, dense matrix                                                  */
/* ------------------------------------------------------------------------- */

static void node_rows_cfie(const or_ctx *c, int i, cplx *row_u, cplx *row_v, cplx *scratch);
static void matrix_dense_cfie(const or_ctx *c, cplx *A);
static void test_vectors(const or_ctx *c, int i, double t[2][3]);

/* Both rows (u and v) of target node i of the MFIE system, length N = 2 nnode each.
 * Unknown index 2*node + a (a = 0: F^u, a = 1: F^v). */
static void node_rows(const or_ctx *c, int i, cplx *row_u, cplx *row_v, cplx *W)
{
    int nc = c->nc, nc2 = nc * nc;
    int ti = i / nc2;
    const double *ri = c->nr + 3 * i, *aui = c->nau + 3 * i, *avi = c->nav + 3 * i;
    for (int p = 0; p < c->npatch; ++p) {
        if (c->near[(size_t)ti * c->npatch + p]) {
            or_near_block(c, i, p, W);
            for (int j = 0; j < nc2; ++j) {
                int col = 2 * (p * nc2 + j);
                row_u[col] = W[0 * nc2 + j];
                row_u[col + 1] = W[1 * nc2 + j];
                row_v[col] = W[2 * nc2 + j];
                row_v[col + 1] = W[3 * nc2 + j];
            }
        } else {
            for (int j = 0; j < nc2; ++j) {
                int sn = p * nc2 + j;
                const double *rj = c->nr + 3 * sn;
                double d[3] = {ri[0] - rj[0], ri[1] - rj[1], ri[2] - rj[2]};
                double R = norm3(d);
                cplx g = -(1.0 + I * c->k * R) * cexp(-I * c->k * R) / (4.0 * OR_PI * R * R * R) * c->nw[sn];
                double cu[3], cv[3];
                cross3(d, c->nau + 3 * sn, cu);
                cross3(d, c->nav + 3 * sn, cv);
                row_u[2 * sn] = g * dot3(avi, cu);
                row_u[2 * sn + 1] = g * dot3(avi, cv);
                row_v[2 * sn] = -g * dot3(aui, cu);
                row_v[2 * sn + 1] = -g * dot3(aui, cv);
            }
        }
    }
    /* identity term from the jump relation (Eq. 5): F^b / 2 */
    row_u[2 * i] += 0.5;
    row_v[2 * i + 1] += 0.5;
}

/* Selected rows of the MFIE matrix, row-major out[nrows][N]. */
void or_matrix_rows(const or_ctx *c, int nrows, const int *rows, cplx *out)
{
    int N = 2 * c->nnode;
    int nc2 = c->nc * c->nc;
#pragma omp parallel
    {
        cplx *ru = (cplx *)malloc(sizeof(cplx) * N);
        cplx *rv = (cplx *)malloc(sizeof(cplx) * N);
        cplx *W = (cplx *)malloc(sizeof(cplx) * 4 * nc2 * (c->cfie ? 2 : 1));
#pragma omp for schedule(dynamic, 1)
        for (int t = 0; t < nrows; ++t) {
            int r = rows[t];
            if (c->cfie)
                node_rows_cfie(c, r / 2, ru, rv, W);
            else
                node_rows(c, r / 2, ru, rv, W);
            memcpy(out + (size_t)t * N, (r % 2 == 0) ? ru : rv, sizeof(cplx) * N);
        }
        free(ru);
        free(rv);
        free(W);
    }
}

/* Dense MFIE matrix, column-major A[col * N + row]. */
void or_matrix_dense(const or_ctx *c, cplx *A)
{
    int N = 2 * c->nnode;
    int nc2 = c->nc * c->nc;
    if (c->cfie) {
        matrix_dense_cfie(c, A);
        return;
    }
#pragma omp parallel
    {
        cplx *ru = (cplx *)malloc(sizeof(cplx) * N);
        cplx *rv = (cplx *)malloc(sizeof(cplx) * N);
        cplx *W = (cplx *)malloc(sizeof(cplx) * 4 * nc2);
#pragma omp for schedule(dynamic, 1)
        for (int i = 0; i < c->nnode; ++i) {
            node_rows(c, i, ru, rv, W);
            for (int col = 0; col < N; ++col) {
                A[(size_t)col * N + 2 * i] = ru[col];
                A[(size_t)col * N + 2 * i + 1] = rv[col];
            }
        }
        free(ru);
        free(rv);
        free(W);
    }
}

/* Dense single-layer matrix S[i][j] (nnode x nnode, column-major) for the sphere
 * eigenvalue check: near pairs by the integrator, far pairs by w_j sqrtG_j G. */
void or_single_layer_dense(const or_ctx *c, cplx *S)
{
    int n = c->nnode, nc2 = c->nc * c->nc;
#pragma omp parallel
    {
        cplx *W = (cplx *)malloc(sizeof(cplx) * nc2);
#pragma omp for schedule(dynamic, 1)
        for (int i = 0; i < n; ++i) {
            int ti = i / nc2;
            for (int p = 0; p < c->npatch; ++p) {
                if (c->near[(size_t)ti * c->npatch + p]) {
                    or_single_layer_block(c, i, p, W);
                    for (int j = 0; j < nc2; ++j) S[(size_t)(p * nc2 + j) * n + i] = W[j];
                } else {
                    for (int j = 0; j < nc2; ++j) {
                        int sn = p * nc2 + j;
                        double d[3] = {c->nr[3 * i] - c->nr[3 * sn], c->nr[3 * i + 1] - c->nr[3 * sn + 1], c->nr[3 * i + 2] - c->nr[3 * sn + 2]};
                        double R = norm3(d);
                        S[(size_t)sn * n + i] = cexp(-I * c->k * R) / (4.0 * OR_PI * R) * c->nw[sn] * c->nsg[sn];
                    }
                }
            }
        }
        free(W);
    }
}

/* ------------------------------------------------------------------------- */
/* PEC combined field equation (Eq. 10, both rows; combination not in the paper) */
/* ------------------------------------------------------------------------- */
/*
 * Row b of node i:  alpha E_b + (1 - alpha) M_b,  with M_b the MFIE row above and
 *   E_b = t_b . (jk S[J] - (1/(jk)) grad S[div J])  (the EFIE operator L_E of Eq. 2
 *         divided by eta0), t_b = sqrtG a^b (Eqs. 17-18): t_u = a_v x n, t_v = n x a_u;
 *   right-hand side alpha t_b . E_inc / eta0 + (1 - alpha) t_b . (n x H_inc).
 * The surface divergence of the interpolated current is its spectral derivative on the
 * source patch: (div J) dS' = (d_u F^u + d_v F^v) du dv (Eq. 11).
 * Far pairs (Nystrom / Fejer rule, grad G analytic):
 *   E_b(i; j,a) = jk w_j G_ij t_b.a_a(j) - (1/(jk)) sum_{j' on the a-line of j} w_j' g_ij' t_b.(r_i - r_j') D[l(j'), l(j)]
 * Self/near pairs: the vector part is the exact integral of G t_b.a_a against the
 * cardinal function; grad S[div J] is strongly singular, so it is taken as the tangential
 * derivative of the scalar potential Phi = S[div J] along the target patch:
 *   t_b . grad Phi (r_i) = sqrtG_i (g^{bu} d_u Phi + g^{bv} d_v Phi)(i),
 * with Phi at the target patch's nodes from the exact integrals of G against the
 * source-differentiated cardinal functions, and d_u, d_v the spectral derivatives on
 * the target patch (g^{bc}: inverse metric of a_u, a_v at the target).
 */
void or_set_cfie(or_ctx *c, double alpha)
{
    int nc = c->nc;
    c->cfie = 1;
    c->alpha = alpha;
    if (!c->dmat) c->dmat = (double *)malloc(sizeof(double) * nc * nc);
    double ell[64];
    for (int l = 0; l < nc; ++l) cheb_cardinal_d(nc, c->nodes1d, c->nodes1d[l], ell, c->dmat + l * nc);
}

/* Test vectors t_u = a_v x n, t_v = n x a_u of node i. */
static void test_vectors(const or_ctx *c, int i, double t[2][3])
{
    cross3(c->nav + 3 * i, c->nn + 3 * i, t[0]);
    cross3(c->nn + 3 * i, c->nau + 3 * i, t[1]);
}

/* The integrals of one kind for target node tn over source patch p. */
static void near_kind(const or_ctx *c, int kind, int tn, int p, cplx *W)
{
    integ ig;
    memset(&ig, 0, sizeof(ig));
    ig.c = c;
    ig.kind = kind;
    ig.p = p;
    ig.k = c->k;
    ig.kbox = c->k;
    ig.ncomp = kind == KIND_SCALAR ? 1 : 4;
    ig.W = W;
    for (int d = 0; d < 3; ++d) ig.tgt[d] = c->nr[3 * tn + d];
    test_vectors(c, tn, ig.te);
    int nc = c->nc, tp = tn / (nc * nc);
    if (tp == p)
        integ_patch(&ig, tn % nc, (tn / nc) % nc);
    else
        integ_patch(&ig, -1, -1);
}

/* CFIE entries of the rows of target nodes `tl` (local indices on patch q) against source
 * patch p, a near pair: out[(2 t + b) * 2 nc^2 + 2 j + a] for t < ntl (the identity term
 * (1 - alpha)/2 is not included).  Phi is needed at every node of the two lines of
 * each target through its patch; the integrals of each such node are computed once. */
static void cfie_near_rows(const or_ctx *c, int q, int p, int ntl, const int *tl, cplx *out)
{
    int nc = c->nc, nc2 = nc * nc, w = 2 * nc2;
    const double *D = c->dmat;
    const cplx jk = I * c->k;
    unsigned char *need = (unsigned char *)calloc(nc2, 1);
    for (int t = 0; t < ntl; ++t) {
        int li = tl[t] % nc, ki = tl[t] / nc;
        for (int l = 0; l < nc; ++l) {
            need[ki * nc + l] = 1;
            need[l * nc + li] = 1;
        }
    }
    /* Phi_a(i'; j) = sum_j' W^S(i'; j') Dsrc_a(j', j) for the needed targets i' */
    cplx *WS = (cplx *)malloc(sizeof(cplx) * nc2);
    cplx *Phi = (cplx *)calloc((size_t)nc2 * 2 * nc2, sizeof(cplx)); /* [i'][a][j] */
    for (int ip = 0; ip < nc2; ++ip) {
        if (!need[ip]) continue;
        near_kind(c, KIND_SCALAR, q * nc2 + ip, p, WS);
        cplx *Pu = Phi + (size_t)ip * 2 * nc2, *Pv = Pu + nc2;
        for (int kv = 0; kv < nc; ++kv)
            for (int lu = 0; lu < nc; ++lu) {
                cplx su = 0, sv = 0;
                for (int l2 = 0; l2 < nc; ++l2) su += WS[kv * nc + l2] * D[l2 * nc + lu];
                for (int k2 = 0; k2 < nc; ++k2) sv += WS[k2 * nc + lu] * D[k2 * nc + kv];
                Pu[kv * nc + lu] = su;
                Pv[kv * nc + lu] = sv;
            }
    }
    cplx *WV = (cplx *)malloc(sizeof(cplx) * 4 * nc2), *WM = (cplx *)malloc(sizeof(cplx) * 4 * nc2);
    for (int t = 0; t < ntl; ++t) {
        int il = tl[t], li = il % nc, ki = il / nc, tn = q * nc2 + il;
        near_kind(c, KIND_EVEC, tn, p, WV);
        or_near_block(c, tn, p, WM);
        const double *au = c->nau + 3 * tn, *av = c->nav + 3 * tn;
        double guu = dot3(au, au), guv = dot3(au, av), gvv = dot3(av, av);
        double det = guu * gvv - guv * guv, sg = c->nsg[tn];
        double gi[2][2] = {{gvv / det, -guv / det}, {-guv / det, guu / det}}; /* g^{bc} */
        for (int a = 0; a < 2; ++a)
            for (int j = 0; j < nc2; ++j) {
                /* d_u Phi_a and d_v Phi_a at the target (spectral derivative on patch q) */
                cplx du = 0, dv = 0;
                for (int l2 = 0; l2 < nc; ++l2) du += D[li * nc + l2] * Phi[((size_t)(ki * nc + l2) * 2 + a) * nc2 + j];
                for (int k2 = 0; k2 < nc; ++k2) dv += D[ki * nc + k2] * Phi[((size_t)(k2 * nc + li) * 2 + a) * nc2 + j];
                for (int b = 0; b < 2; ++b) {
                    cplx E = jk * WV[(2 * b + a) * nc2 + j] - (1.0 / jk) * sg * (gi[b][0] * du + gi[b][1] * dv);
                    cplx M = WM[(2 * b + a) * nc2 + j];
                    out[(size_t)(2 * t + b) * w + 2 * j + a] = c->alpha * E + (1.0 - c->alpha) * M;
                }
            }
    }
    free(need);
    free(WS);
    free(Phi);
    free(WV);
    free(WM);
}

/* CFIE far entries of node i's two rows against every node of source patch p
 * (row_u, row_v: full-length rows, written at p's columns). */
static void cfie_far_rows(const or_ctx *c, int i, int p, cplx *row_u, cplx *row_v, cplx *h)
{
    int nc = c->nc, nc2 = nc * nc;
    const double *D = c->dmat;
    const cplx jk = I * c->k;
    const double *ri = c->nr + 3 * i, *aui = c->nau + 3 * i, *avi = c->nav + 3 * i;
    double t[2][3];
    test_vectors(c, i, t);
    /* h[b][j'] = w_j' g(R) t_b . (r_i - r_j') */
    for (int j = 0; j < nc2; ++j) {
        int sn = p * nc2 + j;
        const double *rj = c->nr + 3 * sn;
        double d[3] = {ri[0] - rj[0], ri[1] - rj[1], ri[2] - rj[2]};
        double R = norm3(d);
        cplx g = -(1.0 + I * c->k * R) * cexp(-I * c->k * R) / (4.0 * OR_PI * R * R * R) * c->nw[sn];
        h[j] = g * dot3(t[0], d);
        h[nc2 + j] = g * dot3(t[1], d);
    }
    for (int j = 0; j < nc2; ++j) {
        int sn = p * nc2 + j, lu = j % nc, kv = j / nc;
        const double *rj = c->nr + 3 * sn, *auj = c->nau + 3 * sn, *avj = c->nav + 3 * sn;
        double d[3] = {ri[0] - rj[0], ri[1] - rj[1], ri[2] - rj[2]};
        double R = norm3(d);
        cplx ex = cexp(-I * c->k * R);
        cplx G = ex / (4.0 * OR_PI * R) * c->nw[sn];
        cplx g = -(1.0 + I * c->k * R) * ex / (4.0 * OR_PI * R * R * R) * c->nw[sn];
        double cu[3], cv[3];
        cross3(d, auj, cu);
        cross3(d, avj, cv);
        cplx M[2][2] = {{g * dot3(avi, cu), g * dot3(avi, cv)}, {-g * dot3(aui, cu), -g * dot3(aui, cv)}};
        for (int b = 0; b < 2; ++b) {
            cplx divu = 0, divv = 0;
            for (int l2 = 0; l2 < nc; ++l2) divu += h[b * nc2 + kv * nc + l2] * D[l2 * nc + lu];
            for (int k2 = 0; k2 < nc; ++k2) divv += h[b * nc2 + k2 * nc + lu] * D[k2 * nc + kv];
            cplx Eu = jk * G * dot3(t[b], auj) - (1.0 / jk) * divu;
            cplx Ev = jk * G * dot3(t[b], avj) - (1.0 / jk) * divv;
            cplx *row = b == 0 ? row_u : row_v;
            row[2 * sn] = c->alpha * Eu + (1.0 - c->alpha) * M[b][0];
            row[2 * sn + 1] = c->alpha * Ev + (1.0 - c->alpha) * M[b][1];
        }
    }
}

/* Both CFIE rows of node i (full length N). */
static void node_rows_cfie(const or_ctx *c, int i, cplx *row_u, cplx *row_v, cplx *scratch)
{
    int nc = c->nc, nc2 = nc * nc, w = 2 * nc2;
    int ti = i / nc2, il = i - ti * nc2;
    for (int p = 0; p < c->npatch; ++p) {
        if (c->near[(size_t)ti * c->npatch + p]) {
            cfie_near_rows(c, ti, p, 1, &il, scratch);
            for (int col = 0; col < w; ++col) {
                row_u[p * w + col] = scratch[col];
                row_v[p * w + col] = scratch[w + col];
            }
        } else {
            cfie_far_rows(c, i, p, row_u, row_v, scratch);
        }
    }
    row_u[2 * i] += 0.5 * (1.0 - c->alpha);
    row_v[2 * i + 1] += 0.5 * (1.0 - c->alpha);
}

/* Dense CFIE matrix, column-major, assembled by target patch so that the scalar
 * potentials of each near pair are integrated once per target node. */
static void matrix_dense_cfie(const or_ctx *c, cplx *A)
{
    int N = 2 * c->nnode, nc = c->nc, nc2 = nc * nc, w = 2 * nc2;
#pragma omp parallel
    {
        cplx *blk = (cplx *)malloc(sizeof(cplx) * (size_t)w * w);
        cplx *ru = (cplx *)malloc(sizeof(cplx) * N), *rv = (cplx *)malloc(sizeof(cplx) * N);
        cplx *h = (cplx *)malloc(sizeof(cplx) * 2 * nc2);
        int *all = (int *)malloc(sizeof(int) * nc2);
        for (int t = 0; t < nc2; ++t) all[t] = t;
#pragma omp for schedule(dynamic, 1)
        for (int q = 0; q < c->npatch; ++q) {
            for (int p = 0; p < c->npatch; ++p) {
                if (c->near[(size_t)q * c->npatch + p]) {
                    cfie_near_rows(c, q, p, nc2, all, blk);
                    for (int r = 0; r < w; ++r)
                        for (int col = 0; col < w; ++col)
                            A[(size_t)(p * w + col) * N + q * w + r] = blk[(size_t)r * w + col];
                } else {
                    for (int il = 0; il < nc2; ++il) {
                        int i = q * nc2 + il;
                        cfie_far_rows(c, i, p, ru, rv, h);
                        for (int col = p * w; col < (p + 1) * w; ++col) {
                            A[(size_t)col * N + 2 * i] = ru[col];
                            A[(size_t)col * N + 2 * i + 1] = rv[col];
                        }
                    }
                }
            }
            for (int il = 0; il < nc2; ++il) {
                int i = q * nc2 + il;
                A[(size_t)(2 * i) * N + 2 * i] += 0.5 * (1.0 - c->alpha);
                A[(size_t)(2 * i + 1) * N + 2 * i + 1] += 0.5 * (1.0 - c->alpha);
            }
        }
        free(blk);
        free(ru);
        free(rv);
        free(h);
        free(all);
    }
}

/* ------------------------------------------------------------------------- */
/* Dielectric body: N-Mueller system (Sec. II.A, Eqs. 7-9)                    */
/* ------------------------------------------------------------------------- */

/* Interior medium of relative permittivity eps_r (mu_r = 1): k2 = k sqrt(eps_r). */
void or_set_dielectric(or_ctx *c, double eps_re, double eps_im)
{
    c->dielectric = 1;
    c->epsr = eps_re + I * eps_im;
    c->k2 = c->k * csqrt(c->epsr);
    if (cimag(c->k2) > 0) c->k2 = conj(c->k2); /* decaying exp(-j k2 R) for a lossy interior */
}

static void muller_setup(const or_ctx *c, integ *ig, int tn, int p, cplx *W)
{
    memset(ig, 0, sizeof(*ig));
    ig->c = c;
    ig->kind = KIND_MULLER;
    ig->p = p;
    ig->k = c->k;
    ig->kbox = fmax(c->k, cabs(c->k2));
    ig->ncomp = 16;
    ig->W = W;
    for (int d = 0; d < 3; ++d) {
        ig->tgt[d] = c->nr[3 * tn + d];
        ig->tu[d] = c->nau[3 * tn + d];
        ig->tv[d] = c->nav[3 * tn + d];
    }
}

/* Self/near N-Mueller weights of target node tn over source patch p: the exact
 * integrals of the integrand against the Chebyshev interpolant (Eq. 20), by the
 * independent adaptive integrator.  W[(row * 4 + col) * nc^2 + j]. */
void or_muller_near_block(const or_ctx *c, int tn, int p, cplx *W)
{
    integ ig;
    muller_setup(c, &ig, tn, p, W);
    int nc = c->nc;
    if (tn / (nc * nc) == p)
        integ_patch(&ig, tn % nc, (tn / nc) % nc);
    else
        integ_patch(&ig, -1, -1);
}

/* Far N-Mueller weights: Fejer's rule on the source patch's own nodes (the Nystrom
 * rule), applied to the same integrand; the divergence terms pick up the spectral
 * derivative of the interpolant along the node's grid line. */
void or_muller_far_block(const or_ctx *c, int tn, int p, cplx *W)
{
    integ ig;
    muller_setup(c, &ig, tn, p, W);
    int nc = c->nc;
    memset(W, 0, sizeof(cplx) * 16 * nc * nc);
    for (int kv = 0; kv < nc; ++kv)
        for (int lu = 0; lu < nc; ++lu)
            integ_point(&ig, c->nodes1d[lu], c->nodes1d[kv], c->fejer[lu] * c->fejer[kv]);
}

/* The four rows (E-u, E-v, H-u, H-v) of target node i, length N = 4 nnode, unknown
 * 4 n + col with col = (Jbar^u, Jbar^v, M^u, M^v); identity terms from the jump
 * relations (Eq. 6): -(1 + eps_r)/2 on M in the E-rows, (1 + 1)/2 on J in the H-rows. */
static void node_rows_muller(const or_ctx *c, int i, cplx *rows, cplx *W)
{
    int nc = c->nc, nc2 = nc * nc, N = 4 * c->nnode;
    int ti = i / nc2;
    for (int p = 0; p < c->npatch; ++p) {
        if (c->near[(size_t)ti * c->npatch + p])
            or_muller_near_block(c, i, p, W);
        else
            or_muller_far_block(c, i, p, W);
        for (int row = 0; row < 4; ++row)
            for (int col = 0; col < 4; ++col)
                for (int j = 0; j < nc2; ++j)
                    rows[(size_t)row * N + 4 * (p * nc2 + j) + col] = W[(row * 4 + col) * nc2 + j];
    }
    cplx ide = -(1.0 + c->epsr) / 2.0;
    rows[(size_t)0 * N + 4 * i + 2] += ide;
    rows[(size_t)1 * N + 4 * i + 3] += ide;
    rows[(size_t)2 * N + 4 * i + 0] += 1.0;
    rows[(size_t)3 * N + 4 * i + 1] += 1.0;
}

/* Dense N-Mueller matrix, column-major A[col * N + row], N = 4 nnode. */
void or_matrix_dense_muller(const or_ctx *c, cplx *A)
{
    int N = 4 * c->nnode;
    int nc2 = c->nc * c->nc;
#pragma omp parallel
    {
        cplx *rows = (cplx *)malloc(sizeof(cplx) * 4 * (size_t)N);
        cplx *W = (cplx *)malloc(sizeof(cplx) * 16 * nc2);
#pragma omp for schedule(dynamic, 1)
        for (int i = 0; i < c->nnode; ++i) {
            node_rows_muller(c, i, rows, W);
            for (int col = 0; col < N; ++col)
                for (int r = 0; r < 4; ++r) A[(size_t)col * N + 4 * i + r] = rows[(size_t)r * N + col];
        }
        free(rows);
        free(W);
    }
}

/* N-Mueller right-hand sides for E = pol exp(-jk khat.r): E-row b: t_b . E_inc,
 * H-row b: t_b . (eta0 H_inc) = t_b . (khat x pol) exp(-jk khat.r); b [nrhs][4 nnode]. */
void or_rhs_muller(const or_ctx *c, int nrhs, const double *kdir, const double *pol, cplx *b)
{
    int N = 4 * c->nnode;
    for (int r = 0; r < nrhs; ++r) {
        double kh[3], h0[3];
        const double *po = pol + 3 * r;
        for (int d = 0; d < 3; ++d) kh[d] = kdir[3 * r + d];
        cross3(kh, po, h0);
        for (int i = 0; i < c->nnode; ++i) {
            cplx ph = cexp(-I * c->k * dot3(kh, c->nr + 3 * i));
            const double *au = c->nau + 3 * i, *av = c->nav + 3 * i;
            cplx *o = b + (size_t)r * N + 4 * i;
            o[0] = -dot3(av, po) * ph;
            o[1] = dot3(au, po) * ph;
            o[2] = -dot3(av, h0) * ph;
            o[3] = dot3(au, h0) * ph;
        }
    }
}

/* J (A/m) and M (V/m) at the nodes from an N-Mueller solution x[4 nnode]. */
void or_currents_muller(const or_ctx *c, const cplx *x, cplx *J, cplx *M)
{
    for (int i = 0; i < c->nnode; ++i)
        for (int d = 0; d < 3; ++d) {
            J[3 * i + d] = (x[4 * i] * c->nau[3 * i + d] + x[4 * i + 1] * c->nav[3 * i + d]) / c->nsg[i] / c->eta0;
            M[3 * i + d] = (x[4 * i + 2] * c->nau[3 * i + d] + x[4 * i + 3] * c->nav[3 * i + d]) / c->nsg[i];
        }
}

/* Far field of an N-Mueller solution: with N_J = sum_j w_j (Jbar^u a_u + Jbar^v a_v)_j
 * exp(jk rhat.r_j) and N_M likewise from M,
 *   E_far = -jk/(4 pi) [ (I - rhat rhat) N_J - rhat x N_M ],  rcs = 4 pi |E_far|^2. */
void or_farfield_muller(const or_ctx *c, const cplx *x, int nang, const double *obs, cplx *efar, double *rcs)
{
    for (int a = 0; a < nang; ++a) {
        const double *rh = obs + 3 * a;
        cplx NJ[3] = {0, 0, 0}, NM[3] = {0, 0, 0};
        for (int j = 0; j < c->nnode; ++j) {
            cplx ph = cexp(I * c->k * dot3(rh, c->nr + 3 * j)) * c->nw[j];
            for (int d = 0; d < 3; ++d) {
                NJ[d] += ph * (x[4 * j] * c->nau[3 * j + d] + x[4 * j + 1] * c->nav[3 * j + d]);
                NM[d] += ph * (x[4 * j + 2] * c->nau[3 * j + d] + x[4 * j + 3] * c->nav[3 * j + d]);
            }
        }
        cplx rn = rh[0] * NJ[0] + rh[1] * NJ[1] + rh[2] * NJ[2];
        cplx rxm[3] = {rh[1] * NM[2] - rh[2] * NM[1], rh[2] * NM[0] - rh[0] * NM[2], rh[0] * NM[1] - rh[1] * NM[0]};
        cplx pre = -I * c->k / (4.0 * OR_PI);
        double s = 0;
        for (int d = 0; d < 3; ++d) {
            cplx e = pre * (NJ[d] - rn * rh[d] - rxm[d]);
            efar[3 * a + d] = e;
            s += creal(e) * creal(e) + cimag(e) * cimag(e);
        }
        rcs[a] = 4.0 * OR_PI * s;
    }
}

/* ------------------------------------------------------------------------- */
/* Excitation and outputs                                                     */
/* ------------------------------------------------------------------------- */

/* Plane wave E = pol exp(-jk khat.r), H = (khat x pol) exp(-jk khat.r) / eta0.
 * MFIE rows: b[2i] = -a_v . H(r_i), b[2i+1] = a_u . H(r_i). b is [nrhs][N]. */
void or_rhs(const or_ctx *c, int nrhs, const double *kdir, const double *pol, cplx *b)
{
    int N = 2 * c->nnode;
    for (int r = 0; r < nrhs; ++r) {
        double kh[3], h0[3];
        for (int d = 0; d < 3; ++d) kh[d] = kdir[3 * r + d];
        cross3(kh, pol + 3 * r, h0);
        for (int i = 0; i < c->nnode; ++i) {
            cplx ph = cexp(-I * c->k * dot3(kh, c->nr + 3 * i)) / c->eta0;
            cplx hv[3] = {h0[0] * ph, h0[1] * ph, h0[2] * ph};
            const double *au = c->nau + 3 * i, *av = c->nav + 3 * i;
            cplx bu = -(av[0] * hv[0] + av[1] * hv[1] + av[2] * hv[2]);
            cplx bv = au[0] * hv[0] + au[1] * hv[1] + au[2] * hv[2];
            if (c->cfie) {
                /* alpha t_b . E_inc / eta0 + (1 - alpha) t_b . (n x H_inc) */
                double t[2][3];
                test_vectors(c, i, t);
                const double *pl = pol + 3 * r;
                bu = c->alpha * dot3(t[0], pl) * ph + (1.0 - c->alpha) * bu;
                bv = c->alpha * dot3(t[1], pl) * ph + (1.0 - c->alpha) * bv;
            }
            b[(size_t)r * N + 2 * i] = bu;
            b[(size_t)r * N + 2 * i + 1] = bv;
        }
    }
}

/* Surface current J(r_i) = (F^u a_u + F^v a_v) / sqrtG (Eq. 11) for one solution x[N]. */
void or_currents(const or_ctx *c, const cplx *x, cplx *J)
{
    for (int i = 0; i < c->nnode; ++i)
        for (int d = 0; d < 3; ++d)
            J[3 * i + d] = (x[2 * i] * c->nau[3 * i + d] + x[2 * i + 1] * c->nav[3 * i + d]) / c->nsg[i];
}

/* Far field of one solution x[N] at unit directions obs[nang][3]:
 * Nvec = sum_j w_j (F^u a_u + F^v a_v)_j exp(jk rhat.r_j);
 * E_far = -jk eta0/(4 pi) (I - rhat rhat) Nvec  (the e^{-jkr}/r factor removed);
 * rcs = 4 pi |E_far|^2 (unit incident amplitude). */
void or_farfield(const or_ctx *c, const cplx *x, int nang, const double *obs, cplx *efar, double *rcs)
{
    for (int a = 0; a < nang; ++a) {
        const double *rh = obs + 3 * a;
        cplx Nv[3] = {0, 0, 0};
        for (int j = 0; j < c->nnode; ++j) {
            cplx ph = cexp(I * c->k * dot3(rh, c->nr + 3 * j)) * c->nw[j];
            for (int d = 0; d < 3; ++d) Nv[d] += ph * (x[2 * j] * c->nau[3 * j + d] + x[2 * j + 1] * c->nav[3 * j + d]);
        }
        cplx rn = rh[0] * Nv[0] + rh[1] * Nv[1] + rh[2] * Nv[2];
        cplx pre = -I * c->k * c->eta0 / (4.0 * OR_PI);
        double s = 0;
        for (int d = 0; d < 3; ++d) {
            cplx e = pre * (Nv[d] - rn * rh[d]);
            efar[3 * a + d] = e;
            s += creal(e) * creal(e) + cimag(e) * cimag(e);
        }
        rcs[a] = 4.0 * OR_PI * s;
    }
}

/* ------------------------------------------------------------------------- */
/* Dense LU with partial pivoting and solve                                   */
/* ------------------------------------------------------------------------- */

/* Right-looking LU, column-major A (lda = n), ipiv[k] = row swapped with k.
 * Returns 0, or k+1 if the pivot of column k is exactly zero. */
int or_zgetrf(int n, cplx *A, int *ipiv)
{
    int info = 0;
    for (int k = 0; k < n; ++k) {
        int p = k;
        double best = cabs(A[(size_t)k * n + k]);
        for (int i = k + 1; i < n; ++i) {
            double v = cabs(A[(size_t)k * n + i]);
            if (v > best) { best = v; p = i; }
        }
        ipiv[k] = p;
        if (best == 0.0) { if (!info) info = k + 1; continue; }
        if (p != k)
            for (int j = 0; j < n; ++j) {
                cplx t = A[(size_t)j * n + k];
                A[(size_t)j * n + k] = A[(size_t)j * n + p];
                A[(size_t)j * n + p] = t;
            }
        cplx piv = A[(size_t)k * n + k];
        for (int i = k + 1; i < n; ++i) A[(size_t)k * n + i] /= piv;
#pragma omp parallel for schedule(static) if (n - k > 256)
        for (int j = k + 1; j < n; ++j) {
            cplx akj = A[(size_t)j * n + k];
            if (akj == 0) continue;
            cplx *colj = A + (size_t)j * n;
            const cplx *colk = A + (size_t)k * n;
            for (int i = k + 1; i < n; ++i) colj[i] -= colk[i] * akj;
        }
    }
    return info;
}

/* Solve A X = B with the factors of or_zgetrf; B is column-major n x nrhs. */
void or_zgetrs(int n, const cplx *LU, const int *ipiv, int nrhs, cplx *B)
{
    for (int r = 0; r < nrhs; ++r) {
        cplx *b = B + (size_t)r * n;
        for (int k = 0; k < n; ++k)
            if (ipiv[k] != k) { cplx t = b[k]; b[k] = b[ipiv[k]]; b[ipiv[k]] = t; }
        for (int j = 0; j < n; ++j) {
            cplx bj = b[j];
            const cplx *col = LU + (size_t)j * n;
            for (int i = j + 1; i < n; ++i) b[i] -= col[i] * bj;
        }
        for (int j = n - 1; j >= 0; --j) {
            const cplx *col = LU + (size_t)j * n;
            b[j] /= col[j];
            cplx bj = b[j];
            for (int i = 0; i < j; ++i) b[i] -= col[i] * bj;
        }
    }
}
