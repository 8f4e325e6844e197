// Excitation and outputs: plane-wave right-hand sides of the MFIE rows (Eq. 22:
// b1 = -a_v . H_inc, b2 = a_u . H_inc; the paper's mu_1 row scale is dropped),
// unknown permutations between natural and tree order, far field and RCS.
#include <algorithm>

#include "hm_internal.h"

#define ETA0 376.730313668  // sqrt(mu0 / eps0), CODATA 2018

// b[r][tree unknown] for plane waves dirs[r] = (khat, pol): H = (khat x pol) exp(-jk khat.r) / eta0
__global__ void k_rhs(const double *__restrict__ nodes, int nnode, const int *__restrict__ perm, double k, int nrhs,
                      const double *__restrict__ dirs, zc *__restrict__ b)
{
    int pos = blockIdx.x * blockDim.x + threadIdx.x;
    int r = blockIdx.y;
    if (pos >= nnode || r >= nrhs) return;
    int i = perm[2 * pos] >> 1;
    const double *kh = dirs + 6 * r, *po = dirs + 6 * r + 3;
    double h0[3] = {kh[1] * po[2] - kh[2] * po[1], kh[2] * po[0] - kh[0] * po[2], kh[0] * po[1] - kh[1] * po[0]};
    double ph = -k * (kh[0] * nodes[i] + kh[1] * nodes[nnode + i] + kh[2] * nodes[2 * nnode + i]);
    double sn, cs;
    sincos(ph, &sn, &cs);
    double au[3] = {nodes[3 * nnode + i], nodes[4 * nnode + i], nodes[5 * nnode + i]};
    double av[3] = {nodes[6 * nnode + i], nodes[7 * nnode + i], nodes[8 * nnode + i]};
    double sv = -(av[0] * h0[0] + av[1] * h0[1] + av[2] * h0[2]) / ETA0;
    double su = (au[0] * h0[0] + au[1] * h0[1] + au[2] * h0[2]) / ETA0;
    size_t N = 2 * (size_t)nnode;
    b[r * N + 2 * pos] = zmake(sv * cs, sv * sn);
    b[r * N + 2 * pos + 1] = zmake(su * cs, su * sn);
}

void launch_rhs(hm_handle_s *h, int nrhs, const double *d_dirs, zc *d_b)
{
    dim3 g((h->nnode + 127) / 128, nrhs);
    k_rhs<<<g, 128, 0, h->stream>>>(h->d_nodes, h->nnode, h->d_perm, h->prm.k0, nrhs, d_dirs, d_b);
    HM_CHECK_LAUNCH();
    count_launch(h);
}

// dst[r][i] = src[r][map[i]]
__global__ void k_permute(int N, int nrhs, const zc *__restrict__ src, zc *__restrict__ dst, const int *__restrict__ map)
{
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)N * nrhs) return;
    size_t r = idx / N, i = idx % N;
    dst[idx] = src[r * N + map[i]];
}

void launch_permute(hm_handle_s *h, int nrhs, const zc *src, zc *dst, const int *map)
{
    size_t n = (size_t)h->N * nrhs;
    if (n == 0) return;
    k_permute<<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(h->N, nrhs, src, dst, map);
    HM_CHECK_LAUNCH();
    count_launch(h);
}

// One CTA per (rhs, angle): Nvec = sum_j w_j (F^u a_u + F^v a_v)_j exp(jk rhat.r_j);
// E = -jk eta0/(4 pi) (Nvec - (rhat.Nvec) rhat);  rcs = 4 pi |E|^2.
__global__ void k_farfield(const double *__restrict__ nodes, int nnode, double k, const zc *__restrict__ x, int nang,
                           const double *__restrict__ dirs, zc *__restrict__ efar, double *__restrict__ rcs)
{
    int a = blockIdx.x, r = blockIdx.y;
    const double *rh = dirs + 3 * a;
    const zc *xr = x + (size_t)r * 2 * nnode;
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int j = threadIdx.x; j < nnode; j += blockDim.x) {
        double ph = k * (rh[0] * nodes[j] + rh[1] * nodes[nnode + j] + rh[2] * nodes[2 * nnode + j]);
        double sn, cs;
        sincos(ph, &sn, &cs);
        double w = nodes[13 * nnode + j];
        zc fu = xr[2 * j], fv = xr[2 * j + 1];
        zc e = zmake(w * cs, w * sn);
        zc cu = zmul(fu, e), cv = zmul(fv, e);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            double au = nodes[(3 + d) * nnode + j], av = nodes[(6 + d) * nnode + j];
            acc[2 * d] += cu.x * au + cv.x * av;
            acc[2 * d + 1] += cu.y * au + cv.y * av;
        }
    }
    __shared__ double sh[6][32];
#pragma unroll
    for (int t = 0; t < 6; ++t) {
        double v = acc[t];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffff, v, o);
        if ((threadIdx.x & 31) == 0) sh[t][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double N[6];
        for (int t = 0; t < 6; ++t) {
            double s = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[t][w];
            N[t] = s;
        }
        zc Nv[3] = {zmake(N[0], N[1]), zmake(N[2], N[3]), zmake(N[4], N[5])};
        zc rn = zadd(zadd(zscale(Nv[0], rh[0]), zscale(Nv[1], rh[1])), zscale(Nv[2], rh[2]));
        zc pre = zmake(0.0, -k * ETA0 / (4.0 * 3.14159265358979323846));
        double s2 = 0;
        for (int d = 0; d < 3; ++d) {
            zc e = zmul(pre, zsub(Nv[d], zscale(rn, rh[d])));
            if (efar) efar[((size_t)r * nang + a) * 3 + d] = e;
            s2 += zabs2(e);
        }
        if (rcs) rcs[(size_t)r * nang + a] = 4.0 * 3.14159265358979323846 * s2;
    }
}

void launch_farfield(hm_handle_s *h, int nrhs, const zc *d_x, int nang, const double *d_dirs, zc *d_efar, double *d_rcs)
{
    if (nrhs <= 0 || nang <= 0) return;
    if (nang > 0x7fffffff / 4) throw HmError{HM_ERR_ARG, "too many observation directions"};
    // gridDim.y is limited to 65,535: right-hand sides go in chunks of at most that many
    for (int r0 = 0; r0 < nrhs; r0 += 65535) {
        const int nr = std::min(65535, nrhs - r0);
        k_farfield<<<dim3(nang, nr), 256, 0, h->stream>>>(h->d_nodes, h->nnode, h->prm.k0,
                                                          d_x + (size_t)r0 * 2 * h->nnode, nang, d_dirs,
                                                          d_efar ? d_efar + (size_t)r0 * nang * 3 : nullptr,
                                                          d_rcs ? d_rcs + (size_t)r0 * nang : nullptr);
        HM_CHECK_LAUNCH();
        count_launch(h);
    }
}
