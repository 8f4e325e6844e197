// Node geometry (Sec. II.B, Eqs. 11, 14, 17-18) and the self/near CBIE
// quadrature (Eq. 20) for the MFIE of a PEC body.
//
// Near-field method (this library's; the paper defers its change of variables
// to its ref. [9]):
//   For target node i and source patch p, take the point (uc, vc) of p's chart
//   closest to the singularity: the node itself when i lies on p (self), else the
//   chart preimage of r_i clamped to [-1,1]^2, at parameter distance eps from the
//   true (exterior) preimage.  Split [-1,1]^2 at (uc, vc) into up to four
//   rectangles with a corner at (uc, vc).
//   * near (eps > 0): tensor rule on each rectangle; in each direction a graded
//     1-D rule: a sinh-mapped Gauss panel t = eps sinh(mu x) on [0, min(L, T0)]
//     (clusters points at the corner on the scale eps) and a plain Gauss panel on
//     [T0, L].
//   * self (eps = 0): the physically square part of each rectangle at the corner
//     is integrated in Duffy coordinates (two triangles; the Jacobian s cancels
//     the 1/R singularity of the kernel), the remaining strip with a tensor rule
//     that is plain Gauss across the strip and graded (eps = square side) along it.
//   Every piece keeps one coordinate a function of the outer index only, so the
//   Chebyshev moments beta_nm = sum K T_n(u) T_m(v) accumulate as two small
//   matrix products per chunk of rows; the nodal weights follow from the moments
//   through the discrete Chebyshev transform of Eq. 13 substituted into Eq. 12:
//   W_{lk} = sum_nm beta_nm C_nl C_mk,  C_nl = alpha_n T_n(x_l) / Nc.
#include <cstdio>

#include "hm_internal.h"

#define NEAR_THREADS 256
#define AXIS_MAX 64

// ---------------------------------------------------------------------------
// Node table: SoA [14][nnode]: r(3) a_u(3) a_v(3) n(3) sqrtG w
// ---------------------------------------------------------------------------
__global__ void k_nodes(const DevBody *__restrict__ bodies, const DevPatch *__restrict__ patches, int nc, int nnode,
                        const double *__restrict__ x1d, const double *__restrict__ w1d, double *__restrict__ out)
{
    int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= nnode) return;
    int nc2 = nc * nc;
    int p = id / nc2, loc = id - p * nc2;
    int kv = loc / nc, lu = loc - kv * nc;
    DevPatch P = patches[p];
    DevBody B = bodies[P.body];
    double r[3], ru[3], rv[3];
    patch_eval(B, P, x1d[lu], x1d[kv], r, ru, rv);
    double n[3] = {ru[1] * rv[2] - ru[2] * rv[1], ru[2] * rv[0] - ru[0] * rv[2], ru[0] * rv[1] - ru[1] * rv[0]};
    double sg = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        out[(0 + d) * nnode + id] = r[d];
        out[(3 + d) * nnode + id] = ru[d];
        out[(6 + d) * nnode + id] = rv[d];
        out[(9 + d) * nnode + id] = n[d] / sg;
    }
    out[12 * nnode + id] = sg;
    out[13 * nnode + id] = w1d[lu] * w1d[kv];
}

void launch_nodes(hm_handle_s *h, const double *d_x1d, const double *d_w1d)
{
    int T = 128;
    k_nodes<<<(h->nnode + T - 1) / T, T, 0, h->stream>>>(h->d_bodies, h->d_patches, h->nc, h->nnode, d_x1d, d_w1d,
                                                         h->d_nodes);
    HM_CHECK_LAUNCH();
    count_launch(h);
}

// Points of each patch on the grid g[ng] x g[ng] (for bounding boxes): out [P][ng*ng][3]
__global__ void k_patch_grid(const DevBody *__restrict__ bodies, const DevPatch *__restrict__ patches, int npatch,
                             const double *__restrict__ g, int ng, double *__restrict__ out)
{
    int id = blockIdx.x * blockDim.x + threadIdx.x;
    int per = ng * ng;
    if (id >= npatch * per) return;
    int p = id / per, loc = id - p * per;
    int b = loc / ng, a = loc - b * ng;
    DevPatch P = patches[p];
    double r[3], ru[3], rv[3];
    patch_eval(bodies[P.body], P, g[a], g[b], r, ru, rv);
    out[3 * (size_t)id] = r[0];
    out[3 * (size_t)id + 1] = r[1];
    out[3 * (size_t)id + 2] = r[2];
}

void launch_patch_grid(hm_handle_s *h, const double *d_g, int ng, double *d_out)
{
    int T = 128, n = h->npatch * ng * ng;
    k_patch_grid<<<(n + T - 1) / T, T, 0, h->stream>>>(h->d_bodies, h->d_patches, h->npatch, d_g, ng, d_out);
    HM_CHECK_LAUNCH();
    count_launch(h);
}

// ---------------------------------------------------------------------------
// Near-field quadrature
// ---------------------------------------------------------------------------
struct NearArgs {
    const double *nodes;
    int nnode;
    const DevBody *bodies;
    const DevPatch *patches;
    const int *pair_q, *pair_p;
    int nc;
    double k;
    int qd, qi, qo;
    double t0;
    const double *tabs;  // gd_x[qd] gd_w[qd] gi_x[qi] gi_w[qi] go_x[qo] go_w[qo] (all on [0,1])
    const double *C;     // [nc][nc]: C[n*nc + l] = alpha_n T_n(x_l) / nc
    const double *x1d;   // [nc] Chebyshev nodes
    zc *out;             // [npairs][2 nc^2][2 nc^2]
    unsigned long long *counter;
    int rmax;            // rows per chunk bound: NEAR_THREADS / min(qd, qi)
};

// MFIE kernel components at source point (u,v) for target (ri, tu = a_u(r_i), tv = a_v(r_i)):
// K[2b+a] = s_b g(R) t_b . ((r_i - r') x a_a(r')),  t_u = a_v (s=+1), t_v = a_u (s=-1),
// g(R) = -(1 + jkR) exp(-jkR) / (4 pi R^3)   (grad G of Eq. 4).
__device__ __forceinline__ void mfie_kernel(const DevBody &B, const DevPatch &P, double u, double v, const double *ri,
                                            const double *tu, const double *tv, double k, double w, zc *K)
{
    double r[3], ru[3], rv[3];
    patch_eval(B, P, u, v, r, ru, rv);
    double d0 = ri[0] - r[0], d1 = ri[1] - r[1], d2 = ri[2] - r[2];
    double R2 = d0 * d0 + d1 * d1 + d2 * d2;
    if (!(R2 > 0.0)) {
        K[0] = K[1] = K[2] = K[3] = zmake(0, 0);
        return;
    }
    double R = sqrt(R2);
    double sn, cs;
    sincos(k * R, &sn, &cs);
    double kR = k * R;
    double f = -w / (4.0 * 3.14159265358979323846 * R2 * R);
    zc g = zmake(f * (cs + kR * sn), f * (kR * cs - sn));
    double cu0 = d1 * ru[2] - d2 * ru[1], cu1 = d2 * ru[0] - d0 * ru[2], cu2 = d0 * ru[1] - d1 * ru[0];
    double cv0 = d1 * rv[2] - d2 * rv[1], cv1 = d2 * rv[0] - d0 * rv[2], cv2 = d0 * rv[1] - d1 * rv[0];
    double vu = tv[0] * cu0 + tv[1] * cu1 + tv[2] * cu2;
    double vv = tv[0] * cv0 + tv[1] * cv1 + tv[2] * cv2;
    double uu = tu[0] * cu0 + tu[1] * cu1 + tu[2] * cu2;
    double uv = tu[0] * cv0 + tu[1] * cv1 + tu[2] * cv2;
    K[0] = zscale(g, vu);
    K[1] = zscale(g, vv);
    K[2] = zscale(g, -uu);
    K[3] = zscale(g, -uv);
}

struct NearShared {
    double ri[3], tu[3], tv[3];
    int p;
    // current piece
    int type;  // 0 tensor (A = u), 1 Duffy with u = uc + du s (A = u), 2 Duffy with v = vc + dv s (A = v)
    int nA, nB;
    double uc, vc, du, dv;
    double ax[AXIS_MAX], aw[AXIS_MAX];  // tensor A axis (u)
    double bx[AXIS_MAX], bw[AXIS_MAX];  // tensor B axis (v)
    double tab[6 * AXIS_MAX];
    double C[HM_NC_MAX * HM_NC_MAX];
    double x1d[HM_NC_MAX];
    unsigned long long npts;
};

// Graded 1-D rule on [0, L] clustered at 0 for a singularity at distance eps before 0.
__device__ int graded_axis(const NearArgs &a, const NearShared &S, double eps, double L, double start, double sgn,
                           double *x, double *w)
{
    const double *gix = S.tab + a.qd * 2, *giw = gix + a.qi;
    const double *gox = giw + a.qi, *gow = gox + a.qo;
    double Lin = fmin(L, a.t0);
    double mu = asinh(Lin / eps);
    int n = 0;
    for (int i = 0; i < a.qi; ++i) {
        double sh, ch;
        double z = mu * gix[i];
        sh = sinh(z);
        ch = cosh(z);
        x[n] = start + sgn * eps * sh;
        w[n] = eps * mu * ch * giw[i];
        ++n;
    }
    if (L > a.t0) {
        for (int i = 0; i < a.qo; ++i) {
            x[n] = start + sgn * (a.t0 + (L - a.t0) * gox[i]);
            w[n] = (L - a.t0) * gow[i];
            ++n;
        }
    }
    return n;
}

// Plain Gauss on [start, start + len*sgn]
__device__ int plain_axis(const NearArgs &a, const NearShared &S, double start, double len, double sgn, double *x,
                          double *w)
{
    const double *gix = S.tab + a.qd * 2, *giw = gix + a.qi;
    for (int i = 0; i < a.qi; ++i) {
        x[i] = start + sgn * len * gix[i];
        w[i] = len * giw[i];
    }
    return a.qi;
}

// Accumulate the moments of the current piece into beta (shared, [4][nc][nc] complex).
__device__ void near_piece(const NearArgs &a, NearShared &S, const DevBody &B, const DevPatch &P, zc *Kp, double *Tb,
                           double *TA, zc *Tc, zc *beta)
{
    const int nc = a.nc, tid = threadIdx.x;
    const int nB = S.nB, nA = S.nA, type = S.type;
    const int R = max(1, NEAR_THREADS / nB);
    const double *gdx = S.tab, *gdw = S.tab + a.qd;
    for (int a0 = 0; a0 < nA; a0 += R) {
        int nr = min(R, nA - a0);
        int r = tid / nB, b = tid - r * nB;
        if (r < nr) {
            int iA = a0 + r;
            double u, v, w;
            if (type == 0) {
                u = S.ax[iA];
                v = S.bx[b];
                w = S.aw[iA] * S.bw[b];
            } else {
                double s = gdx[iA], t = gdx[b];
                w = fabs(S.du * S.dv) * s * gdw[iA] * gdw[b];
                if (type == 1) {
                    u = S.uc + S.du * s;
                    v = S.vc + S.dv * s * t;
                } else {
                    v = S.vc + S.dv * s;
                    u = S.uc + S.du * s * t;
                }
            }
            zc K[4];
            mfie_kernel(B, P, u, v, S.ri, S.tu, S.tv, a.k, w, K);
#pragma unroll
            for (int c = 0; c < 4; ++c) Kp[tid * 4 + c] = K[c];
            cheb_T(nc, type == 2 ? u : v, Tb + tid * nc);
        }
        if (tid < nr) {
            int iA = a0 + tid;
            double xa;
            if (type == 0)
                xa = S.ax[iA];
            else if (type == 1)
                xa = S.uc + S.du * gdx[iA];
            else
                xa = S.vc + S.dv * gdx[iA];
            cheb_T(nc, xa, TA + tid * nc);
        }
        __syncthreads();
        // Tc[r][c][j] = sum_b Kp[r, b][c] * Tb[r, b][j]
        for (int idx = tid; idx < nr * 4 * nc; idx += NEAR_THREADS) {
            int rr = idx / (4 * nc), rem = idx - rr * 4 * nc;
            int c = rem / nc, j = rem - c * nc;
            zc acc = zmake(0, 0);
            const zc *kp = Kp + (rr * nB) * 4 + c;
            const double *tb = Tb + (rr * nB) * nc + j;
            for (int bb = 0; bb < nB; ++bb) {
                double t = tb[bb * nc];
                zc kk = kp[bb * 4];
                acc.x = fma(kk.x, t, acc.x);
                acc.y = fma(kk.y, t, acc.y);
            }
            Tc[idx] = acc;
        }
        __syncthreads();
        // beta[c][n][m] (n: u degree, m: v degree)
        for (int idx = tid; idx < 4 * nc * nc; idx += NEAR_THREADS) {
            int c = idx / (nc * nc), rem = idx - c * nc * nc;
            int n = rem / nc, m = rem - n * nc;
            zc acc = beta[idx];
            for (int rr = 0; rr < nr; ++rr) {
                double t;
                zc tc;
                if (type != 2) {
                    t = TA[rr * nc + n];
                    tc = Tc[(rr * 4 + c) * nc + m];
                } else {
                    t = TA[rr * nc + m];
                    tc = Tc[(rr * 4 + c) * nc + n];
                }
                acc.x = fma(tc.x, t, acc.x);
                acc.y = fma(tc.y, t, acc.y);
            }
            beta[idx] = acc;
        }
        __syncthreads();
    }
    if (tid == 0) S.npts += (unsigned long long)nA * nB;
}

__global__ void __launch_bounds__(NEAR_THREADS) k_near(NearArgs a)
{
    extern __shared__ double dyn[];
    __shared__ NearShared S;
    const int nc = a.nc, nc2 = nc * nc, tid = threadIdx.x;
    const int pair = blockIdx.x / nc2, tn = blockIdx.x - pair * nc2;
    const int q = a.pair_q[pair], p = a.pair_p[pair];
    const int rmax = a.rmax;
    zc *Kp = (zc *)dyn;                                  // [256][4]
    double *Tb = (double *)(Kp + NEAR_THREADS * 4);      // [256][nc]
    double *TA = Tb + NEAR_THREADS * nc;                 // [rmax][nc]
    zc *Tc = (zc *)(TA + rmax * nc);                     // [max(rmax*4*nc, 4*nc*nc)]
    zc *beta = Tc + (rmax * 4 * nc > 4 * nc2 ? rmax * 4 * nc : 4 * nc2);  // [4][nc][nc]
    // tables
    int ntab = 2 * (a.qd + a.qi + a.qo);
    for (int i = tid; i < ntab; i += NEAR_THREADS) S.tab[i] = a.tabs[i];
    for (int i = tid; i < nc2; i += NEAR_THREADS) S.C[i] = a.C[i];
    for (int i = tid; i < nc; i += NEAR_THREADS) S.x1d[i] = a.x1d[i];
    for (int i = tid; i < 4 * nc2; i += NEAR_THREADS) beta[i] = zmake(0, 0);
    const int node = q * nc2 + tn;
    if (tid == 0) {
        for (int d = 0; d < 3; ++d) {
            S.ri[d] = a.nodes[(0 + d) * a.nnode + node];
            S.tu[d] = a.nodes[(3 + d) * a.nnode + node];
            S.tv[d] = a.nodes[(6 + d) * a.nnode + node];
        }
        S.p = p;
        S.npts = 0;
    }
    __syncthreads();
    const DevPatch P = a.patches[p];
    const DevBody B = a.bodies[P.body];
    // singular point in p's chart
    __shared__ double sh_uc, sh_vc, sh_eps, sh_gu, sh_gv;
    if (tid == 0) {
        double uc, vc, eps;
        if (q == p) {
            int kv = tn / nc, lu = tn - kv * nc;
            uc = S.x1d[lu];
            vc = S.x1d[kv];
            eps = 0.0;
        } else {
            double u0, v0;
            if (patch_chart(B, P, S.ri, &u0, &v0)) {
                uc = fmin(1.0, fmax(-1.0, u0));
                vc = fmin(1.0, fmax(-1.0, v0));
                eps = fmax(hypot(u0 - uc, v0 - vc), 1e-6);
            } else {
                uc = 0.0;
                vc = 0.0;
                eps = 1.0;
            }
        }
        double r[3], ru[3], rv[3];
        patch_eval(B, P, uc, vc, r, ru, rv);
        sh_gu = sqrt(ru[0] * ru[0] + ru[1] * ru[1] + ru[2] * ru[2]);
        sh_gv = sqrt(rv[0] * rv[0] + rv[1] * rv[1] + rv[2] * rv[2]);
        sh_uc = uc;
        sh_vc = vc;
        sh_eps = eps;
    }
    __syncthreads();
    const double uc = sh_uc, vc = sh_vc, eps = sh_eps, gu = sh_gu, gv = sh_gv;
    for (int corner = 0; corner < 4; ++corner) {
        double du = (corner & 1) ? (-1.0 - uc) : (1.0 - uc);
        double dv = (corner & 2) ? (-1.0 - vc) : (1.0 - vc);
        if (fabs(du) < 1e-14 || fabs(dv) < 1e-14) continue;
        double su = du > 0 ? 1.0 : -1.0, sv = dv > 0 ? 1.0 : -1.0;
        if (eps > 0.0) {
            if (tid == 0) {
                S.type = 0;
                S.nA = graded_axis(a, S, eps, fabs(du), uc, su, S.ax, S.aw);
                S.nB = graded_axis(a, S, eps, fabs(dv), vc, sv, S.bx, S.bw);
            }
            __syncthreads();
            near_piece(a, S, B, P, Kp, Tb, TA, Tc, beta);
            continue;
        }
        // self: Duffy on the physically square part at the corner, strip by a tensor rule
        double pa = fabs(du) * gu, pb = fabs(dv) * gv;
        double ddu = du, ddv = dv;
        int strip = 0;  // 0 none, 1 along v, 2 along u
        if (pb > pa) {
            ddv = sv * pa / gv;
            if (fabs(dv) - fabs(ddv) > 1e-14) strip = 1;
        } else {
            ddu = su * pb / gu;
            if (fabs(du) - fabs(ddu) > 1e-14) strip = 2;
        }
        for (int tri = 1; tri <= 2; ++tri) {
            if (tid == 0) {
                S.type = tri;
                S.nA = a.qd;
                S.nB = a.qd;
                S.uc = uc;
                S.vc = vc;
                S.du = ddu;
                S.dv = ddv;
            }
            __syncthreads();
            near_piece(a, S, B, P, Kp, Tb, TA, Tc, beta);
        }
        if (strip) {
            if (tid == 0) {
                S.type = 0;
                if (strip == 1) {
                    S.nA = plain_axis(a, S, uc, fabs(du), su, S.ax, S.aw);
                    S.nB = graded_axis(a, S, fabs(ddv), fabs(dv) - fabs(ddv), vc + ddv, sv, S.bx, S.bw);
                } else {
                    S.nA = graded_axis(a, S, fabs(ddu), fabs(du) - fabs(ddu), uc + ddu, su, S.ax, S.aw);
                    S.nB = plain_axis(a, S, vc, fabs(dv), sv, S.bx, S.bw);
                }
            }
            __syncthreads();
            near_piece(a, S, B, P, Kp, Tb, TA, Tc, beta);
        }
    }
    // nodal weights W_c[k][l] = sum_nm beta_c[n][m] C[n][l] C[m][k]
    zc *X = Tc;  // reuse: [4][nc(l)][nc(m)]
    for (int idx = tid; idx < 4 * nc2; idx += NEAR_THREADS) {
        int c = idx / nc2, rem = idx - c * nc2;
        int l = rem / nc, m = rem - l * nc;
        zc acc = zmake(0, 0);
        for (int n = 0; n < nc; ++n) {
            double cc = S.C[n * nc + l];
            zc bb = beta[c * nc2 + n * nc + m];
            acc.x = fma(bb.x, cc, acc.x);
            acc.y = fma(bb.y, cc, acc.y);
        }
        X[idx] = acc;
    }
    __syncthreads();
    zc *out = a.out + (size_t)pair * (2 * nc2) * (2 * nc2) + (size_t)(tn * 2) * (2 * nc2);
    for (int idx = tid; idx < 4 * nc2; idx += NEAR_THREADS) {
        int c = idx / nc2, j = idx - c * nc2;
        int kk = j / nc, l = j - kk * nc;
        zc acc = zmake(0, 0);
        for (int m = 0; m < nc; ++m) {
            double cc = S.C[m * nc + kk];
            zc xx = X[(c * nc + l) * nc + m];
            acc.x = fma(xx.x, cc, acc.x);
            acc.y = fma(xx.y, cc, acc.y);
        }
        int b = c >> 1, aa = c & 1;
        out[(size_t)b * (2 * nc2) + 2 * j + aa] = acc;
    }
    if (tid == 0) atomicAdd(a.counter, S.npts);
}

void launch_near(hm_handle_s *h, const double *d_tabs, const double *d_C)
{
    NearArgs a;
    a.nodes = h->d_nodes;
    a.nnode = h->nnode;
    a.bodies = h->d_bodies;
    a.patches = h->d_patches;
    a.pair_q = h->d_pair_q;
    a.pair_p = h->d_pair_p;
    a.nc = h->nc;
    a.k = h->prm.k0;
    a.qd = h->rule.qd;
    a.qi = h->rule.qi;
    a.qo = h->rule.qo;
    a.t0 = h->rule.t0;
    a.tabs = d_tabs;
    a.C = d_C;
    a.x1d = d_tabs + 2 * (a.qd + a.qi + a.qo);
    a.out = h->d_near;
    a.counter = h->d_counter;
    int nc = h->nc;
    int rmax = NEAR_THREADS / (a.qd < a.qi ? a.qd : a.qi);
    a.rmax = rmax;
    size_t tcn = (size_t)(rmax * 4 * nc > 4 * nc * nc ? rmax * 4 * nc : 4 * nc * nc);
    size_t smem = sizeof(zc) * NEAR_THREADS * 4 + sizeof(double) * NEAR_THREADS * nc + sizeof(double) * rmax * nc +
                  sizeof(zc) * tcn + sizeof(zc) * 4 * nc * nc;
    HM_CUDA(cudaFuncSetAttribute(k_near, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    long long nblk = (long long)h->pair_q.size() * nc * nc;
    if (nblk == 0) return;
    k_near<<<(unsigned)nblk, NEAR_THREADS, smem, h->stream>>>(a);
    HM_CHECK_LAUNCH();
    count_launch(h);
}
