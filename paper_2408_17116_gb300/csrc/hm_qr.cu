// Batched blocked Householder QR of the low-rank factors in a recompression
// (Sec. III: the truncation after every formatted addition of the H-LU), one
// cooperative launch per batch:
//
//   for every panel p of NB columns:
//     phase 1: one CTA per job factors panel p (unblocked Householder on the panel
//              columns) and forms the compact-WY factor T_p, H_j0..H_j0+NB-1 = I - V T V^H;
//     grid barrier;
//     phase 2: every CTA takes (job, 16-column tile) items to the right of the panel and
//              applies A <- (I - V T^H V^H) A = A - V (T^H (V^H A)) (two passes over the
//              tile's rows, V and the tile staged in shared memory);
//     grid barrier;
//   phase 3: (job, 16-column tile of Q) items form Q = H_0 ... H_{r-1} [I_r; 0] by applying
//            the panels in reverse to the tile, and (job, column) items copy R.
//
// The panel work is latency-bound (one CTA per job); the trailing updates and the
// formation of Q, which carry almost all of the flops, are spread over every SM.
// H_j = I - beta_j v_j v_j^H with v_j = x - alpha e_1, alpha = -exp(i arg x_0) |x|, as in
// the unblocked form; R[j][j] = alpha_j.
#include <cooperative_groups.h>

#include <algorithm>

#include "hm_internal.h"

namespace cg = cooperative_groups;

#define BQ_NB 16   // panel width
#define BQ_T 256   // threads per CTA
#define BQ_TW 16   // columns per update / Q tile (equal to BQ_NB: the staged tiles share a layout)

// rows staged per chunk: the shared-memory tiles stay within the 48 KB static limit
template <class C> struct BQRows;
template <> struct BQRows<cf> { static constexpr int value = 128; };
template <> struct BQRows<zc> { static constexpr int value = 48; };

template <class C>
struct BQDesc {
    C *A;          // m x K (ld m), overwritten by the reflectors below the diagonal
    int m, K, r;   // r = min(m, K)
    C *Q;          // m x r (ld m)
    C *R;          // r x K (ld r)
    typename CReal<C>::R *beta;  // r
    C *T;          // [panels][NB][NB], T[p][a][b] at a * NB + b (upper triangular)
};

template <class R>
__device__ __forceinline__ R bq_block_sum(R v, R *sh)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffff, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        R s = 0;
        for (int w = 0; w < BQ_T / 32; ++w) s += sh[w];
        sh[32] = s;
    }
    __syncthreads();
    R r = sh[32];
    __syncthreads();
    return r;
}

// v_a[i] of panel (j0, A): zero above row j0 + a, A[i, j0 + a] on and below it (the
// diagonal entry holds x_0 - alpha).
template <class C>
__device__ __forceinline__ C bq_v(const C *A, int m, int j0, int a, int i)
{
    return i < j0 + a ? cmk<C>(0, 0) : A[(size_t)(j0 + a) * m + i];
}

// Index of the job owning item `it` given the prefix array pre[0..n] (pre[n] = total).
__device__ __forceinline__ int bq_find(const int *pre, int n, int it)
{
    int lo = 0, hi = n;  // pre[lo] <= it < pre[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (pre[mid] <= it)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

// Apply (I - V W V^H) with W = T^H (trans = true) or T (trans = false) of panel (j0, nbp)
// to the columns [c0, c0 + nc) of X (rows j0 .. m, ld m).  Shared scratch: Vs, Xs
// [RC][BQ_NB] each, Ws, W2 [BQ_NB][BQ_TW], Ts [BQ_NB][BQ_NB].
template <class C, int RC>
__device__ void bq_apply(const C *A, int m, int j0, int nbp, const C *Tg, bool trans, C *X, int c0, int nc, C *Vs,
                         C *Xs, C *Ws, C *W2, C *Ts)
{
    const int tid = threadIdx.x;
    for (int e = tid; e < BQ_NB * BQ_NB; e += BQ_T) Ts[e] = Tg[e];
    for (int e = tid; e < BQ_NB * BQ_TW; e += BQ_T) Ws[e] = cmk<C>(0, 0);
    __syncthreads();
    // W = V^H X  (nbp x nc): thread (a, c) accumulates over the staged rows
    const int wa = tid / BQ_TW, wc = tid % BQ_TW;  // 16 x 16 = 256 threads
    C acc = cmk<C>(0, 0);
    for (int i0 = j0; i0 < m; i0 += RC) {
        const int nr = min(RC, m - i0);
        for (int e = tid; e < nr * BQ_NB; e += BQ_T) {
            int i = e / BQ_NB, a = e - i * BQ_NB;
            Vs[e] = a < nbp ? bq_v(A, m, j0, a, i0 + i) : cmk<C>(0, 0);
            Xs[e] = a < nc ? X[(size_t)(c0 + a) * m + i0 + i] : cmk<C>(0, 0);
        }
        __syncthreads();
        if (wa < nbp && wc < nc)
            for (int i = 0; i < nr; ++i) acc = zfmac(Vs[i * BQ_NB + wa], Xs[i * BQ_NB + wc], acc);
        __syncthreads();
    }
    Ws[wa * BQ_TW + wc] = acc;
    __syncthreads();
    // W2 = T^H W (trans) or T W
    {
        C s = cmk<C>(0, 0);
        if (wa < nbp && wc < nc) {
            if (trans) {
                for (int b = 0; b <= wa; ++b) s = zfmac(Ts[b * BQ_NB + wa], Ws[b * BQ_TW + wc], s);
            } else {
                for (int b = wa; b < nbp; ++b) s = zfma(Ts[wa * BQ_NB + b], Ws[b * BQ_TW + wc], s);
            }
        }
        W2[wa * BQ_TW + wc] = s;
    }
    __syncthreads();
    // X -= V W2
    for (int i0 = j0; i0 < m; i0 += RC) {
        const int nr = min(RC, m - i0);
        for (int e = tid; e < nr * BQ_NB; e += BQ_T) {
            int i = e / BQ_NB, a = e - i * BQ_NB;
            Vs[e] = a < nbp ? bq_v(A, m, j0, a, i0 + i) : cmk<C>(0, 0);
        }
        __syncthreads();
        for (int e = tid; e < nr * nc; e += BQ_T) {
            int c = e / nr, i = e - c * nr;
            C s = cmk<C>(0, 0);
            for (int a = 0; a < nbp; ++a) s = zfma(Vs[i * BQ_NB + a], W2[a * BQ_TW + c], s);
            C *x = X + (size_t)(c0 + c) * m + i0 + i;
            *x = zsub(*x, s);
        }
        __syncthreads();
    }
}

template <class C>
__global__ void __launch_bounds__(BQ_T) k_qr_blocked(const BQDesc<C> *__restrict__ descs, int njobs, int npanels,
                                                     const int *__restrict__ upd_pre, const int *__restrict__ q_pre,
                                                     const int *__restrict__ r_pre)
{
    typedef typename CReal<C>::R R;
    cg::grid_group grid = cg::this_grid();
    constexpr int RC = BQRows<C>::value;
    static_assert(BQ_NB == BQ_TW, "panel width and tile width share the staging layout");
    __shared__ C Vs[RC * BQ_NB], Xs[RC * BQ_NB];
    __shared__ C Ws[BQ_NB * BQ_TW], W2[BQ_NB * BQ_TW], Ts[BQ_NB * BQ_NB];
    __shared__ R sh[33];
    __shared__ C s_alpha;
    __shared__ C Sv[BQ_NB * BQ_NB];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = BQ_T / 32;
    for (int p = 0; p < npanels; ++p) {
        // phase 1: panel factorisation, one CTA per job
        for (int jb = blockIdx.x; jb < njobs; jb += gridDim.x) {
            const BQDesc<C> d = descs[jb];
            const int j0 = p * BQ_NB;
            if (j0 >= d.r) continue;
            const int nbp = min(BQ_NB, d.r - j0), m = d.m;
            C *A = d.A;
            for (int jj = 0; jj < nbp; ++jj) {
                const int j = j0 + jj;
                C *x = A + (size_t)j * m;
                R nrm2 = 0;
                for (int i = j + tid; i < m; i += BQ_T) nrm2 += zabs2(x[i]);
                nrm2 = bq_block_sum(nrm2, sh);
                if (tid == 0) {
                    R nrm = sqrt(nrm2);
                    C x0 = x[j];
                    R a0 = sqrt(zabs2(x0));
                    C ph = a0 > 0 ? zscale(x0, (R)1 / a0) : cmk<C>(1, 0);
                    C alpha = zscale(ph, -nrm);
                    s_alpha = alpha;
                    x[j] = zsub(x0, alpha);
                    R vhv = 2 * (nrm2 + nrm * a0);
                    d.beta[j] = vhv > 0 ? 2 / vhv : 0;
                    d.R[(size_t)j * d.r + j] = alpha;
                }
                __syncthreads();
                const R beta = d.beta[j];
                // the reflector on the panel's remaining columns
                for (int c = j + 1 + warp; c < j0 + nbp; c += nw) {
                    C *a = A + (size_t)c * m;
                    C s = cmk<C>(0, 0);
                    for (int i = j + lane; i < m; i += 32) s = zfmac(x[i], a[i], s);
                    for (int o = 16; o > 0; o >>= 1) {
                        s.x += __shfl_xor_sync(0xffffffff, s.x, o);
                        s.y += __shfl_xor_sync(0xffffffff, s.y, o);
                    }
                    s = zscale(s, beta);
                    for (int i = j + lane; i < m; i += 32) a[i] = zsub(a[i], zmul(x[i], s));
                }
                __syncthreads();
            }
            // T: T[a][a] = beta_a, T[0:a, a] = -beta_a T[0:a, 0:a] (V[:, 0:a]^H v_a)
            for (int e = warp; e < nbp * nbp; e += nw) {
                const int a = e / nbp, b = e - a * nbp;
                if (a >= b) continue;
                C s = cmk<C>(0, 0);
                for (int i = j0 + b + lane; i < m; i += 32) s = zfmac(bq_v(A, m, j0, a, i), bq_v(A, m, j0, b, i), s);
                for (int o = 16; o > 0; o >>= 1) {
                    s.x += __shfl_xor_sync(0xffffffff, s.x, o);
                    s.y += __shfl_xor_sync(0xffffffff, s.y, o);
                }
                if (lane == 0) Sv[a * BQ_NB + b] = s;
            }
            __syncthreads();
            if (tid == 0) {
                C *T = d.T + (size_t)p * BQ_NB * BQ_NB;
                for (int e = 0; e < BQ_NB * BQ_NB; ++e) T[e] = cmk<C>(0, 0);
                for (int b = 0; b < nbp; ++b) {
                    const R bb = d.beta[j0 + b];
                    for (int a = 0; a < b; ++a) {
                        C s = cmk<C>(0, 0);
                        for (int l = a; l < b; ++l) s = zfma(T[a * BQ_NB + l], Sv[l * BQ_NB + b], s);
                        T[a * BQ_NB + b] = zscale(s, -bb);
                    }
                    T[b * BQ_NB + b] = cmk<C>(bb, 0);
                }
            }
            __syncthreads();
        }
        grid.sync();
        // phase 2: trailing update of every job, (job, tile) items over the grid
        const int *pre = upd_pre + (size_t)p * (njobs + 1);
        for (int it = blockIdx.x; it < pre[njobs]; it += gridDim.x) {
            const int jb = bq_find(pre, njobs, it);
            const BQDesc<C> d = descs[jb];
            const int j0 = p * BQ_NB, nbp = min(BQ_NB, d.r - j0);
            const int c0 = j0 + nbp + (it - pre[jb]) * BQ_TW;
            const int nc = min(BQ_TW, d.K - c0);
            bq_apply<C, RC>(d.A, d.m, j0, nbp, d.T + (size_t)p * BQ_NB * BQ_NB, true, d.A, c0, nc, Vs, Xs, Ws, W2, Ts);
        }
        grid.sync();
    }
    // phase 3: explicit Q = H_0 ... H_{r-1} [I; 0] per 16-column tile, panels in reverse
    for (int it = blockIdx.x; it < q_pre[njobs]; it += gridDim.x) {
        const int jb = bq_find(q_pre, njobs, it);
        const BQDesc<C> d = descs[jb];
        const int q0 = (it - q_pre[jb]) * BQ_TW, nc = min(BQ_TW, d.r - q0), m = d.m;
        for (int e = tid; e < m * nc; e += BQ_T) {
            int c = e / m, i = e - c * m;
            d.Q[(size_t)(q0 + c) * m + i] = cmk<C>(i == q0 + c ? 1 : 0, 0);
        }
        __syncthreads();
        // panels starting below the tile's last row leave it unchanged
        const int plast = min((d.r - 1) / BQ_NB, (q0 + nc - 1) / BQ_NB);
        for (int pp = plast; pp >= 0; --pp) {
            const int j0 = pp * BQ_NB, nbp = min(BQ_NB, d.r - j0);
            bq_apply<C, RC>(d.A, m, j0, nbp, d.T + (size_t)pp * BQ_NB * BQ_NB, false, d.Q, q0, nc, Vs, Xs, Ws, W2, Ts);
        }
    }
    // R: the upper triangle of the factored A (the diagonal was written in phase 1)
    for (int it = blockIdx.x; it < r_pre[njobs]; it += gridDim.x) {
        const int jb = bq_find(r_pre, njobs, it);
        const BQDesc<C> d = descs[jb];
        const int c = it - r_pre[jb];
        for (int i = tid; i < d.r; i += BQ_T) {
            if (i == c) continue;
            d.R[(size_t)c * d.r + i] = i < c ? d.A[(size_t)c * d.m + i] : cmk<C>(0, 0);
        }
    }
}

template <class C>
void batched_qr(hm_handle_s *h, const std::vector<QRJob<C>> &jobs)
{
    typedef typename CReal<C>::R R;
    const int nj = (int)jobs.size();
    if (nj == 0) return;
    int npanels = 0;
    size_t nbeta = 0, nT = 0;
    for (auto &J : jobs) {
        const int r = std::min(J.m, J.K);
        const int np = (r + BQ_NB - 1) / BQ_NB;
        npanels = std::max(npanels, np);
        nbeta += r;
        nT += (size_t)np * BQ_NB * BQ_NB;
    }
    // device descriptors, workspace and item prefixes
    std::vector<BQDesc<C>> dd(nj);
    std::vector<int> upd((size_t)npanels * (nj + 1), 0), qp(nj + 1, 0), rp(nj + 1, 0);
    R *beta = (R *)dalloc(h, sizeof(R) * std::max<size_t>(nbeta, 1));
    C *T = (C *)dalloc(h, sizeof(C) * std::max<size_t>(nT, 1));
    size_t ob = 0, ot = 0;
    for (int j = 0; j < nj; ++j) {
        const QRJob<C> &J = jobs[j];
        const int r = std::min(J.m, J.K), np = (r + BQ_NB - 1) / BQ_NB;
        dd[j] = BQDesc<C>{J.A, J.m, J.K, r, J.Q, J.R, beta + ob, T + ot};
        ob += r;
        ot += (size_t)np * BQ_NB * BQ_NB;
        for (int p = 0; p < npanels; ++p) {
            int tiles = 0;
            if (p < np) {
                const int cstart = p * BQ_NB + std::min(BQ_NB, r - p * BQ_NB);
                tiles = std::max(0, (J.K - cstart + BQ_TW - 1) / BQ_TW);
            }
            upd[(size_t)p * (nj + 1) + j + 1] = upd[(size_t)p * (nj + 1) + j] + tiles;
        }
        qp[j + 1] = qp[j] + (r + BQ_TW - 1) / BQ_TW;
        rp[j + 1] = rp[j] + J.K;
    }
    const size_t bytes = sizeof(BQDesc<C>) * nj + sizeof(int) * (upd.size() + qp.size() + rp.size());
    char *buf = (char *)dalloc(h, bytes);
    BQDesc<C> *d_desc = (BQDesc<C> *)buf;
    int *d_upd = (int *)(buf + sizeof(BQDesc<C>) * nj);
    int *d_qp = d_upd + upd.size(), *d_rp = d_qp + qp.size();
    std::vector<char> hb(bytes);
    memcpy(hb.data(), dd.data(), sizeof(BQDesc<C>) * nj);
    memcpy(hb.data() + sizeof(BQDesc<C>) * nj, upd.data(), sizeof(int) * upd.size());
    memcpy(hb.data() + sizeof(BQDesc<C>) * nj + sizeof(int) * upd.size(), qp.data(), sizeof(int) * qp.size());
    memcpy(hb.data() + sizeof(BQDesc<C>) * nj + sizeof(int) * (upd.size() + qp.size()), rp.data(),
           sizeof(int) * rp.size());
    HM_CUDA(cudaMemcpyAsync(buf, hb.data(), bytes, cudaMemcpyHostToDevice, h->stream));
    // one CTA per SM slot the kernel can hold (cooperative launch: all CTAs resident)
    static int grid_cache[2] = {0, 0};
    int &grid = grid_cache[sizeof(R) == 8 ? 1 : 0];
    if (!grid) {
        int per_sm = 0, nsm = 0, dev = 0;
        HM_CUDA(cudaGetDevice(&dev));
        HM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        HM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_qr_blocked<C>, BQ_T, 0));
        grid = std::max(1, std::min(per_sm, 2) * nsm);
    }
    int g = grid;
    int npan = npanels;
    int njv = nj;
    void *kargs[] = {(void *)&d_desc, (void *)&njv, (void *)&npan, (void *)&d_upd, (void *)&d_qp, (void *)&d_rp};
    HM_CUDA(cudaLaunchCooperativeKernel((const void *)k_qr_blocked<C>, dim3(g), dim3(BQ_T), kargs, 0, h->stream));
    count_launch(h);
    dfree(h, buf);
    dfree(h, beta);
    dfree(h, T);
}

template void batched_qr<zc>(hm_handle_s *, const std::vector<QRJob<zc>> &);
template void batched_qr<cf>(hm_handle_s *, const std::vector<QRJob<cf>> &);
