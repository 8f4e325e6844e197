// N-Mueller formulation on the device (Sec. II.A, Eqs. 7-9 with alpha = -eps_r,
// beta = -1, mu_r = 1): the self/near quadrature of the 16 kernel components, the
// plane-wave right-hand side and the far field with the magnetic current.  The entry
// generators and the quadrature pieces are the host/device definitions of hm_muller.cuh.
//
// Near quadrature: one CTA per (near patch pair, target node).  The source patch's
// parameter square is split into the pieces of near_pieces (graded tensor rectangles,
// Duffy squares and strips); on each piece the points form rows along one coordinate x
// (constant within a row) with the other coordinate y varying within the row.  For each
// row the kernel values are first summed against T_m(y) (and T_m'(y) for the divergence
// terms whose derivative is along y), then multiplied by T_n(x) (or T_n'(x)) into the
// Chebyshev moments M_c[n][m] of the 16 components; the nodal weights follow from the
// moments by the map of Eq. 13, W_c[(l, k)] = sum_nm M_c[n][m] C[n][l] C[m][k], which
// serves the cardinal functions and their derivatives alike.
#include <algorithm>

#include "hm_internal.h"
#include "hm_muller.cuh"

#define NM_T 128    // threads per CTA (one quadrature point each per row chunk)
#define NM_R 8      // rows per chunk
#define NM_AX 128   // points per axis of a piece

// derivative components: (E-b, J^a) and (H-b, M^a), c = row * 4 + col; direction a = c & 1
__device__ __constant__ int nm_dcomp[8] = {0, 1, 4, 5, 10, 11, 14, 15};

struct MullerNearArgs {
    const double *nodes;
    int nnode;
    const DevBody *bodies;
    const DevPatch *patches;
    const int *pair_q, *pair_p;
    int nc;
    MullerMedia md;
    int qd, qi, qo;
    double t0;
    const double *tabs;  // gd_x gd_w gi_x gi_w go_x go_w (all on [0,1])
    const double *C;     // [nc][nc] Eq. 13 map
    const double *x1d;   // [nc]
    zc *out;             // [npairs][4 nc^2][4 nc^2]
    unsigned long long *counter;
};

// T_n(x) and T_n'(x), n < nc
__device__ __forceinline__ void cheb_TdT(int nc, double x, double *t, double *dt)
{
    double u0 = 1.0, u1 = 2.0 * x;  // U_0, U_1
    t[0] = 1.0;
    dt[0] = 0.0;
    if (nc > 1) {
        t[1] = x;
        dt[1] = 1.0;
    }
    double um2 = u0, um1 = u1;  // U_{n-2}, U_{n-1} for n = 2
    for (int n = 2; n < nc; ++n) {
        t[n] = 2.0 * x * t[n - 1] - t[n - 2];
        dt[n] = n * um1;  // T_n' = n U_{n-1}
        double un = 2.0 * x * um1 - um2;
        um2 = um1;
        um1 = un;
    }
}

__global__ void __launch_bounds__(NM_T) k_near_muller(MullerNearArgs a)
{
    extern __shared__ __align__(16) unsigned char nm_raw[];
    const int nc = a.nc, nc2 = nc * nc, tid = threadIdx.x;
    zc *Kc = (zc *)nm_raw;               // [NM_T][16]  w cl
    zc *Kd = Kc + NM_T * 16;             // [NM_T][8]   w cd (derivative components)
    zc *P = Kd + NM_T * 8;               // [NM_R][16][nc]
    zc *Pd = P + NM_R * 16 * nc;         // [NM_R][8][nc]
    zc *M = Pd + NM_R * 8 * nc;          // [16][nc][nc]
    double *Ty = (double *)(M + 16 * nc2);  // [NM_T][nc]
    double *dTy = Ty + NM_T * nc;           // [NM_T][nc]
    double *Tx = dTy + NM_T * nc;           // [NM_R][nc]
    double *dTx = Tx + NM_R * nc;           // [NM_R][nc]
    double *ax = dTx + NM_R * nc;           // [NM_AX] axis A points / weights, axis B
    double *aw = ax + NM_AX, *bx = aw + NM_AX, *bw = bx + NM_AX;
    double *tab = bw + NM_AX;               // 2 (qd + qi + qo)
    double *Cs = tab + 2 * (a.qd + a.qi + a.qo);  // [nc][nc]
    __shared__ double ri[3], tu[3], tv[3];
    __shared__ NearPiece pieces[12];
    __shared__ int s_np, s_nA, s_nB;
    __shared__ unsigned long long s_pts;

    const int pair = blockIdx.x / nc2, tn = blockIdx.x - pair * nc2;
    const int q = a.pair_q[pair], p = a.pair_p[pair];
    const int ntab = 2 * (a.qd + a.qi + a.qo);
    for (int i = tid; i < ntab; i += NM_T) tab[i] = a.tabs[i];
    for (int i = tid; i < nc2; i += NM_T) Cs[i] = a.C[i];
    for (int i = tid; i < 16 * nc2; i += NM_T) M[i] = zmake(0, 0);
    const int node = q * nc2 + tn;
    const DevPatch Pp = a.patches[p];
    const DevBody Bp = a.bodies[Pp.body];
    if (tid == 0) {
        for (int d = 0; d < 3; ++d) {
            ri[d] = a.nodes[(0 + d) * a.nnode + node];
            tu[d] = a.nodes[(3 + d) * a.nnode + node];
            tv[d] = a.nodes[(6 + d) * a.nnode + node];
        }
        double uc, vc, eps;
        if (q == p) {
            uc = a.x1d[tn % nc];
            vc = a.x1d[tn / nc];
            eps = 0.0;
        } else {
            double u0, v0;
            if (patch_chart(Bp, Pp, ri, &u0, &v0)) {
                uc = fmin(1.0, fmax(-1.0, u0));
                vc = fmin(1.0, fmax(-1.0, v0));
                eps = fmax(hypot(u0 - uc, v0 - vc), 1e-6);
            } else {
                uc = vc = 0.0;
                eps = 1.0;
            }
        }
        double r[3], ru[3], rv[3];
        patch_eval(Bp, Pp, uc, vc, r, ru, rv);
        const double gu = sqrt(ru[0] * ru[0] + ru[1] * ru[1] + ru[2] * ru[2]);
        const double gv = sqrt(rv[0] * rv[0] + rv[1] * rv[1] + rv[2] * rv[2]);
        s_np = near_pieces(uc, vc, eps, gu, gv, pieces);
        s_pts = 0;
    }
    __syncthreads();
    const double *gdx = tab, *gdw = tab + a.qd;
    const double *gix = gdw + a.qd, *giw = gix + a.qi, *gox = giw + a.qi, *gow = gox + a.qo;
    for (int ip = 0; ip < s_np; ++ip) {
        const NearPiece pc = pieces[ip];
        if (tid == 0) {
            if (pc.type == 0) {
                s_nA = near_axis_points(pc.A, gix, giw, a.qi, gox, gow, a.qo, a.t0, ax, aw);
                s_nB = near_axis_points(pc.B, gix, giw, a.qi, gox, gow, a.qo, a.t0, bx, bw);
            } else {
                s_nA = s_nB = a.qd;
            }
            s_pts += (unsigned long long)s_nA * s_nB;
        }
        __syncthreads();
        const int nA = s_nA, nB = s_nB;
        const bool xu = pc.type != 2;  // the row coordinate x is u (tensor, Duffy 1) or v (Duffy 2)
        const int R = max(1, min(NM_R, NM_T / nB));
        for (int a0 = 0; a0 < nA; a0 += R) {
            const int nr = min(R, nA - a0);
            for (int b0 = 0; b0 < nB; b0 += NM_T) {  // rows longer than the CTA: several passes
                const int nb = min(NM_T, nB - b0);
                const int rr = tid / nb, bb = tid - rr * nb;
                const bool act = nb * rr + bb < nr * nb && rr < nr;
                if (act) {
                    const int iA = a0 + rr, iB = b0 + bb;
                    double u, v, w;
                    if (pc.type == 0) {
                        u = ax[iA];
                        v = bx[iB];
                        w = aw[iA] * bw[iB];
                    } else {
                        const double s = gdx[iA], t = gdx[iB];
                        w = fabs(pc.du * pc.dv) * s * gdw[iA] * gdw[iB];
                        if (pc.type == 1) {
                            u = pc.uc + pc.du * s;
                            v = pc.vc + pc.dv * s * t;
                        } else {
                            v = pc.vc + pc.dv * s;
                            u = pc.uc + pc.du * s * t;
                        }
                    }
                    double r[3], ru[3], rv[3];
                    patch_eval(Bp, Pp, u, v, r, ru, rv);
                    zc cl[16], cd[16];
                    muller_point(ri, tu, tv, r, ru, rv, a.md, cl, cd);
                    for (int c = 0; c < 16; ++c) Kc[tid * 16 + c] = zscale(cl[c], w);
                    for (int e = 0; e < 8; ++e) Kd[tid * 8 + e] = zscale(cd[nm_dcomp[e]], w);
                    cheb_TdT(nc, xu ? v : u, Ty + tid * nc, dTy + tid * nc);
                    if (bb == 0 && b0 == 0) cheb_TdT(nc, xu ? u : v, Tx + rr * nc, dTx + rr * nc);
                }
                __syncthreads();
                // partial sums over the row's points: P[r][c][m], Pd[r][e][m]
                for (int idx = tid; idx < nr * 24 * nc; idx += NM_T) {
                    const int r2 = idx / (24 * nc), rem = idx - r2 * 24 * nc, c = rem / nc, m = rem - c * nc;
                    zc acc = b0 == 0 ? zmake(0, 0) : (c < 16 ? P[(r2 * 16 + c) * nc + m] : Pd[(r2 * 8 + c - 16) * nc + m]);
                    for (int b2 = 0; b2 < nb; ++b2) {
                        const int t = r2 * nb + b2;
                        if (c < 16) {
                            acc = zadd(acc, zscale(Kc[t * 16 + c], Ty[t * nc + m]));
                            // derivative components with the derivative along y
                            const int dirc = c & 1;  // 0: d/du, 1: d/dv
                            const bool dy = xu ? dirc == 1 : dirc == 0;
                            if (dy) {
                                int e = -1;
                                for (int q2 = 0; q2 < 8; ++q2)
                                    if (nm_dcomp[q2] == c) e = q2;
                                if (e >= 0) acc = zadd(acc, zscale(Kd[t * 8 + e], dTy[t * nc + m]));
                            }
                        } else {
                            const int e = c - 16, dirc = nm_dcomp[e] & 1;
                            const bool dx = xu ? dirc == 0 : dirc == 1;
                            if (dx) acc = zadd(acc, zscale(Kd[t * 8 + e], Ty[t * nc + m]));
                        }
                    }
                    if (c < 16)
                        P[(r2 * 16 + c) * nc + m] = acc;
                    else
                        Pd[(r2 * 8 + c - 16) * nc + m] = acc;
                }
                __syncthreads();
            }
            // moments: M_c[n][m] (n: u degree, m: v degree) += T_n(x) P + T_n'(x) Pd
            for (int idx = tid; idx < 16 * nc2; idx += NM_T) {
                const int c = idx / nc2, rem = idx - c * nc2, n = rem / nc, m = rem - n * nc;
                const int ix = xu ? n : m, iy = xu ? m : n;  // x degree, y degree
                int e = -1;
                for (int q2 = 0; q2 < 8; ++q2)
                    if (nm_dcomp[q2] == c) e = q2;
                zc acc = M[idx];
                for (int r2 = 0; r2 < nr; ++r2) {
                    acc = zadd(acc, zscale(P[(r2 * 16 + c) * nc + iy], Tx[r2 * nc + ix]));
                    if (e >= 0) acc = zadd(acc, zscale(Pd[(r2 * 8 + e) * nc + iy], dTx[r2 * nc + ix]));
                }
                M[idx] = acc;
            }
            __syncthreads();
        }
    }
    // nodal weights W_c[(l, k)] = sum_nm M_c[n][m] C[n][l] C[m][k]; P reused as X_c[l][m]
    zc *X = P;  // needs 16 nc^2 <= NM_R (16 + 8) nc: checked by the launcher
    for (int idx = tid; idx < 16 * nc2; idx += NM_T) {
        const int c = idx / nc2, rem = idx - c * nc2, l = rem / nc, m = rem - l * nc;
        zc acc = zmake(0, 0);
        for (int n = 0; n < nc; ++n) acc = zadd(acc, zscale(M[c * nc2 + n * nc + m], Cs[n * nc + l]));
        X[idx] = acc;
    }
    __syncthreads();
    const int w4 = 4 * nc2;
    zc *out = a.out + (size_t)pair * w4 * w4 + (size_t)(4 * tn) * w4;
    for (int idx = tid; idx < 16 * nc2; idx += NM_T) {
        const int c = idx / nc2, j = idx - c * nc2, kk = j / nc, l = j - kk * nc;
        zc acc = zmake(0, 0);
        for (int m = 0; m < nc; ++m) acc = zadd(acc, zscale(X[(c * nc + l) * nc + m], Cs[m * nc + kk]));
        out[(size_t)(c >> 2) * w4 + 4 * j + (c & 3)] = acc;
    }
    if (tid == 0) atomicAdd(a.counter, s_pts);
}

MullerMedia muller_media(double k0, double eps_re, double eps_im)
{
    MullerMedia md;
    md.k = k0;
    md.epsr = zmake(eps_re, eps_im);
    double mod = std::sqrt(std::sqrt(eps_re * eps_re + eps_im * eps_im));
    double arg = 0.5 * std::atan2(eps_im, eps_re);
    md.k2 = zmake(k0 * mod * std::cos(arg), k0 * mod * std::sin(arg));
    if (md.k2.y > 0) md.k2.y = -md.k2.y;
    return md;
}

void launch_near_muller(hm_handle_s *h, const double *d_tabs, const double *d_C)
{
    MullerNearArgs a;
    a.nodes = h->d_nodes;
    a.nnode = h->nnode;
    a.bodies = h->d_bodies;
    a.patches = h->d_patches;
    a.pair_q = h->d_pair_q;
    a.pair_p = h->d_pair_p;
    a.nc = h->nc;
    a.md = muller_media(h->prm.k0, h->prm.eps_r_re, h->prm.eps_r_im);
    a.qd = h->rule.qd;
    a.qi = h->rule.qi;
    a.qo = h->rule.qo;
    a.t0 = h->rule.t0;
    a.tabs = d_tabs;
    a.C = d_C;
    a.x1d = d_tabs + 2 * (a.qd + a.qi + a.qo);
    a.out = h->d_near;
    a.counter = h->d_counter;
    const int nc = h->nc, nc2 = nc * nc;
    if (a.qi + a.qo > NM_AX || a.qd > NM_AX) throw HmError{HM_ERR_ARG, "near rule too fine for the N-Mueller kernel"};
    if (16 * nc2 > NM_R * 24 * nc) throw HmError{HM_ERR_ARG, "Chebyshev order too high for the N-Mueller kernel"};
    const size_t smem = sizeof(zc) * ((size_t)NM_T * 24 + NM_R * 24 * nc + 16 * nc2) +
                        sizeof(double) * ((size_t)2 * NM_T * nc + 2 * NM_R * nc + 4 * NM_AX +
                                          2 * (a.qd + a.qi + a.qo) + nc2);
    HM_CUDA(cudaFuncSetAttribute(k_near_muller, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const long long nblk = (long long)h->pair_q.size() * nc2;
    if (nblk == 0) return;
    k_near_muller<<<(unsigned)nblk, NM_T, smem, h->stream>>>(a);
    HM_CHECK_LAUNCH();
    count_launch(h);
}

// ---------------------------------------------------------------------------
// Right-hand sides (tree order) and far field of the N-Mueller system.
// ---------------------------------------------------------------------------
__global__ void k_rhs_muller(const double *__restrict__ nodes, int nnode, const int *__restrict__ perm, double k,
                             int nrhs, const double *__restrict__ dirs, zc *__restrict__ b)
{
    const int pos = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y;
    if (pos >= nnode || r >= nrhs) return;
    const int i = perm[4 * pos] >> 2;
    zc o[4];
    muller_rhs_node(nodes, nnode, i, k, dirs + 6 * r, dirs + 6 * r + 3, o);
    const size_t N = 4 * (size_t)nnode;
    for (int c = 0; c < 4; ++c) b[r * N + 4 * pos + c] = o[c];
}

void launch_rhs_muller(hm_handle_s *h, int nrhs, const double *d_dirs, zc *d_b)
{
    dim3 g((h->nnode + 127) / 128, nrhs);
    k_rhs_muller<<<g, 128, 0, h->stream>>>(h->d_nodes, h->nnode, h->d_perm, h->prm.k0, nrhs, d_dirs, d_b);
    HM_CHECK_LAUNCH();
    count_launch(h);
}

// One CTA per (angle, rhs): radiation vectors of the electric and magnetic currents,
// E = -jk/(4 pi) [(I - r r) N_J - r x N_M], rcs = 4 pi |E|^2 (x: natural order, 4 per node).
__global__ void k_farfield_muller(const double *__restrict__ nodes, int nnode, double k, const zc *__restrict__ x,
                                  int nang, const double *__restrict__ dirs, zc *__restrict__ efar,
                                  double *__restrict__ rcs)
{
    const int an = blockIdx.x, r = blockIdx.y;
    const double *rh = dirs + 3 * an;
    const zc *xr = x + (size_t)r * 4 * nnode;
    zc NJ[3] = {zmake(0, 0), zmake(0, 0), zmake(0, 0)}, NM[3] = {zmake(0, 0), zmake(0, 0), zmake(0, 0)};
    for (int j = threadIdx.x; j < nnode; j += blockDim.x) muller_radiation_add(nodes, nnode, j, k, rh, xr + 4 * j, NJ, NM);
    __shared__ double sh[12][32];
    double v[12] = {NJ[0].x, NJ[0].y, NJ[1].x, NJ[1].y, NJ[2].x, NJ[2].y, NM[0].x, NM[0].y, NM[1].x, NM[1].y, NM[2].x, NM[2].y};
    for (int t = 0; t < 12; ++t) {
        double s = v[t];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffff, s, o);
        if ((threadIdx.x & 31) == 0) sh[t][threadIdx.x >> 5] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot[12];
        for (int t = 0; t < 12; ++t) {
            double s = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[t][w];
            tot[t] = s;
        }
        zc J3[3] = {zmake(tot[0], tot[1]), zmake(tot[2], tot[3]), zmake(tot[4], tot[5])};
        zc M3[3] = {zmake(tot[6], tot[7]), zmake(tot[8], tot[9]), zmake(tot[10], tot[11])};
        zc E[3];
        muller_far_field(rh, k, J3, M3, E);
        double s2 = 0;
        for (int d = 0; d < 3; ++d) {
            if (efar) efar[((size_t)r * nang + an) * 3 + d] = E[d];
            s2 += zabs2(E[d]);
        }
        if (rcs) rcs[(size_t)r * nang + an] = 4.0 * 3.14159265358979323846 * s2;
    }
}

void launch_farfield_muller(hm_handle_s *h, int nrhs, const zc *d_x, int nang, const double *d_dirs, zc *d_efar,
                            double *d_rcs)
{
    if (nrhs <= 0 || nang <= 0) return;
    for (int r0 = 0; r0 < nrhs; r0 += 65535) {
        const int nr = std::min(65535, nrhs - r0);
        k_farfield_muller<<<dim3(nang, nr), 256, 0, h->stream>>>(
            h->d_nodes, h->nnode, h->prm.k0, d_x + (size_t)r0 * 4 * h->nnode, nang, d_dirs,
            d_efar ? d_efar + (size_t)r0 * nang * 3 : nullptr, d_rcs ? d_rcs + (size_t)r0 * nang : nullptr);
        HM_CHECK_LAUNCH();
        count_launch(h);
    }
}
