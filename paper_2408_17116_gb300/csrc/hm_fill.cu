// Matrix fill of the H-matrix (Sec. III): the entry rule of Eq. 20 (far entries by
// the Nystrom/Fejer rule, self/near entries from the precomputed near store,
// identity term 1/2 from the jump relation, Eq. 5), dense inadmissible leaves,
// and partial-pivot ACA of admissible leaves (Sec. III, ref. [22]).
#include "hm_internal.h"
#include "hm_muller.cuh"

struct EntryCtx {
    const double *nodes;  // SoA [14][nnode]
    int nnode, nc2, P;
    const int *nearidx;   // [P][P]
    const zc *near;       // [npairs][dof nc2][dof nc2]
    const int *perm;      // tree unknown -> natural unknown
    double k;
    int dof;              // unknowns per node: 2 (MFIE) or 4 (N-Mueller)
    int nc;
    MullerMedia md;       // N-Mueller: the interior medium
    const double *d1;     // N-Mueller: [nc][nc] derivatives of the cardinal functions at the nodes
    const int *patch_body;  // independent bodies: body of each patch (entries between bodies are zero)
};

// The four entries A[2ni + b, 2nj + a] of node pair (ni, nj) (natural node indices),
// out[2b + a].  Far: w_j g(R) s_b t_b . ((r_i - r_j) x a_a(r_j)); near: stored weight.
__device__ __forceinline__ void node_pair(const EntryCtx &E, int ni, int nj, zc *out)
{
    int pi = ni / E.nc2, pj = nj / E.nc2;
    int np = E.nearidx[(size_t)pi * E.P + pj];
    if (np >= 0) {
        int w = 2 * E.nc2;
        const zc *blk = E.near + (size_t)np * w * w;
        int ti = ni - pi * E.nc2, sj = nj - pj * E.nc2;
        const zc *r0 = blk + (size_t)(2 * ti) * w + 2 * sj;
        out[0] = r0[0];
        out[1] = r0[1];
        out[2] = r0[w];
        out[3] = r0[w + 1];
    } else {
        const double *X = E.nodes;
        int n = E.nnode;
        double d0 = X[ni] - X[nj], d1 = X[n + ni] - X[n + nj], d2 = X[2 * n + ni] - X[2 * n + nj];
        double R2 = d0 * d0 + d1 * d1 + d2 * d2;
        double R = sqrt(R2);
        double sn, cs;
        sincos(E.k * R, &sn, &cs);
        double kR = E.k * R;
        double f = -X[13 * n + nj] / (4.0 * 3.14159265358979323846 * R2 * R);
        zc g = zmake(f * (cs + kR * sn), f * (kR * cs - sn));
        double au0 = X[3 * n + nj], au1 = X[4 * n + nj], au2 = X[5 * n + nj];
        double av0 = X[6 * n + nj], av1 = X[7 * n + nj], av2 = X[8 * n + nj];
        double cu0 = d1 * au2 - d2 * au1, cu1 = d2 * au0 - d0 * au2, cu2 = d0 * au1 - d1 * au0;
        double cv0 = d1 * av2 - d2 * av1, cv1 = d2 * av0 - d0 * av2, cv2 = d0 * av1 - d1 * av0;
        double tu0 = X[3 * n + ni], tu1 = X[4 * n + ni], tu2 = X[5 * n + ni];
        double tv0 = X[6 * n + ni], tv1 = X[7 * n + ni], tv2 = X[8 * n + ni];
        out[0] = zscale(g, tv0 * cu0 + tv1 * cu1 + tv2 * cu2);
        out[1] = zscale(g, tv0 * cv0 + tv1 * cv1 + tv2 * cv2);
        out[2] = zscale(g, -(tu0 * cu0 + tu1 * cu1 + tu2 * cu2));
        out[3] = zscale(g, -(tu0 * cv0 + tu1 * cv1 + tu2 * cv2));
    }
    if (ni == nj) {
        out[0].x += 0.5;
        out[3].x += 0.5;
    }
}

// The 16 entries of node pair (ni, nj) of the N-Mueller system, out[row * 4 + col]: rows
// E-u, E-v, H-u, H-v, columns eta0 J^u, eta0 J^v, M^u, M^v (Eqs. 7-9); near pairs from the
// near store, far pairs by the Nystrom rule (hm_muller.cuh); identity terms of the jump
// relations (Eq. 6) -(1 + eps_r)/2 on M in the E-rows and 1 on J in the H-rows.
__device__ __forceinline__ void node_pair_muller(const EntryCtx &E, int ni, int nj, zc *out)
{
    int pi = ni / E.nc2, pj = nj / E.nc2;
    int np = E.nearidx[(size_t)pi * E.P + pj];
    if (np >= 0) {
        const int w = 4 * E.nc2;
        const zc *blk = E.near + (size_t)np * w * w;
        const int ti = ni - pi * E.nc2, sj = nj - pj * E.nc2;
        for (int r = 0; r < 4; ++r)
            for (int c = 0; c < 4; ++c) out[r * 4 + c] = blk[(size_t)(4 * ti + r) * w + 4 * sj + c];
    } else {
        muller_far_pair(E.nodes, E.nnode, E.nc, E.d1, E.md, ni, nj, out);
    }
    if (ni == nj) {
        const double hr = -0.5 * (1.0 + E.md.epsr.x), hi = -0.5 * E.md.epsr.y;
        out[0 * 4 + 2] = zadd(out[0 * 4 + 2], zmake(hr, hi));
        out[1 * 4 + 3] = zadd(out[1 * 4 + 3], zmake(hr, hi));
        out[2 * 4 + 0].x += 1.0;
        out[3 * 4 + 1].x += 1.0;
    }
}

// dof x dof entries of node pair (ni, nj), out[b * dof + a]
__device__ __forceinline__ void pair_entries(const EntryCtx &E, int ni, int nj, zc *out)
{
    if (E.patch_body && E.patch_body[ni / E.nc2] != E.patch_body[nj / E.nc2]) {
        for (int e = 0; e < E.dof * E.dof; ++e) out[e] = zmake(0, 0);
        return;
    }
    if (E.dof == 4)
        node_pair_muller(E, ni, nj, out);
    else
        node_pair(E, ni, nj, out);
}

static EntryCtx entry_ctx(hm_handle_s *h)
{
    EntryCtx E;
    E.dof = h->dof;
    E.nc = h->nc;
    E.md = muller_media(h->prm.k0, h->prm.eps_r_re, h->prm.eps_r_im);
    E.d1 = h->d_d1;
    E.nodes = h->d_nodes;
    E.nnode = h->nnode;
    E.nc2 = h->nc * h->nc;
    E.P = h->npatch;
    E.nearidx = h->d_nearidx;
    E.near = h->d_near;
    E.perm = h->d_perm;
    E.k = h->prm.k0;
    E.patch_body = h->d_patch_body;
    return E;
}

// ---------------------------------------------------------------------------
// Dense leaves: one thread per node pair (2 x 2 entries), 16 x 16 node tiles
// ---------------------------------------------------------------------------
__global__ void k_dense_fill(EntryCtx E, const DenseDesc *__restrict__ descs, const int4 *__restrict__ tiles)
{
    int4 t = tiles[blockIdx.x];
    DenseDesc d = descs[t.x];
    const int D = E.dof;
    int rn = t.y * 16 + threadIdx.x;  // node row within block
    int cn = t.z * 16 + threadIdx.y;  // node col within block
    if (D * rn >= d.nr || D * cn >= d.ncol) return;
    int ni = E.perm[d.r0 + D * rn] / D;
    int nj = E.perm[d.c0 + D * cn] / D;
    zc e[16];
    pair_entries(E, ni, nj, e);
    size_t ld = d.nr;
    zc *c0 = d.D + (size_t)(D * cn) * ld + D * rn;
    for (int b = 0; b < D; ++b)
        for (int a = 0; a < D; ++a) c0[(size_t)a * ld + b] = e[b * D + a];
}

void launch_dense_fill(hm_handle_s *h, const std::vector<DenseDesc> &descs)
{
    if (descs.empty()) return;
    std::vector<int4> tiles;
    for (size_t i = 0; i < descs.size(); ++i) {
        int tr = (descs[i].nr / h->dof + 15) / 16, tc = (descs[i].ncol / h->dof + 15) / 16;
        for (int a = 0; a < tr; ++a)
            for (int b = 0; b < tc; ++b) tiles.push_back(make_int4((int)i, a, b, 0));
    }
    DenseDesc *d_desc = (DenseDesc *)dalloc(h, sizeof(DenseDesc) * descs.size());
    int4 *d_tiles = (int4 *)dalloc(h, sizeof(int4) * tiles.size());
    HM_CUDA(cudaMemcpyAsync(d_desc, descs.data(), sizeof(DenseDesc) * descs.size(), cudaMemcpyHostToDevice, h->stream));
    HM_CUDA(cudaMemcpyAsync(d_tiles, tiles.data(), sizeof(int4) * tiles.size(), cudaMemcpyHostToDevice, h->stream));
    // grid-stride over tiles in chunks (gridDim.x limit is large; one launch)
    k_dense_fill<<<(unsigned)tiles.size(), dim3(16, 16), 0, h->stream>>>(entry_ctx(h), d_desc, d_tiles);
    HM_CHECK_LAUNCH();
    count_launch(h);
    HM_CUDA(cudaStreamSynchronize(h->stream));  // host vectors above go out of scope
    dfree(h, d_desc);
    dfree(h, d_tiles);
}

// ---------------------------------------------------------------------------
// Entries at arbitrary (row, col) natural indices (inspection / sampled parity)
// ---------------------------------------------------------------------------
__global__ void k_entries(EntryCtx E, int n, const int *__restrict__ rows, const int *__restrict__ cols, zc *out)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int r = rows[i], c = cols[i];
    const int D = E.dof;
    zc e[16];
    pair_entries(E, r / D, c / D, e);
    out[i] = e[D * (r % D) + (c % D)];
}

void launch_entries(hm_handle_s *h, int n, const int *d_rows, const int *d_cols, zc *d_out)
{
    if (n <= 0) return;
    k_entries<<<(n + 127) / 128, 128, 0, h->stream>>>(entry_ctx(h), n, d_rows, d_cols, d_out);
    HM_CHECK_LAUNCH();
    count_launch(h);
}

// ---------------------------------------------------------------------------
// ACA with partial pivoting, one CTA per admissible block.
// A ~ sum_l u_l v_l^T is stored as U W^H with W = conj(V) (so A ~ U W^H).
//   1. residual row r = A(i,:) - sum_l U(i,l) v_l
//   2. j = argmax |r_j| (ties to the lowest index); an all-zero row is skipped
//   3. v_k = r / r_j;  u_k = A(:,j) - sum_l v_l(j) u_l
//   4. |S_k|^2 = |S_{k-1}|^2 + 2 Re sum_{l<k} (u_l^H u_k)(v_l^H v_k) + |u_k|^2 |v_k|^2
//   5. stop when |u_k| |v_k| <= tol |S_k|; next row i = argmax over unused rows |u_k(i)|
// ---------------------------------------------------------------------------
#define ACA_THREADS 256
#define ACA_WARPS (ACA_THREADS / 32)
#define ACA_MAXROWS 65536

__device__ __forceinline__ void argmax_merge(double &v, int &i, double v2, int i2)
{
    if (v2 > v || (v2 == v && i2 < i)) {
        v = v2;
        i = i2;
    }
}

// block-wide argmax (value, index); returns through shared memory to all threads
__device__ void block_argmax(double v, int i, double *sv, int *si, double &ov, int &oi)
{
    for (int o = 16; o > 0; o >>= 1) {
        double v2 = __shfl_down_sync(0xffffffff, v, o);
        int i2 = __shfl_down_sync(0xffffffff, i, o);
        argmax_merge(v, i, v2, i2);
    }
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        sv[w] = v;
        si[w] = i;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double bv = sv[0];
        int bi = si[0];
        for (int k = 1; k < ACA_WARPS; ++k) argmax_merge(bv, bi, sv[k], si[k]);
        sv[ACA_WARPS] = bv;
        si[ACA_WARPS] = bi;
    }
    __syncthreads();
    ov = sv[ACA_WARPS];
    oi = si[ACA_WARPS];
    __syncthreads();
}

__device__ double block_sum(double v, double *sv)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffff, v, o);
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) sv[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0;
        for (int k = 0; k < ACA_WARPS; ++k) s += sv[k];
        sv[ACA_WARPS] = s;
    }
    __syncthreads();
    double r = sv[ACA_WARPS];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(ACA_THREADS) k_aca(EntryCtx E, const LRDesc *__restrict__ descs, double tol,
                                                      int *__restrict__ rank_out, int *__restrict__ flag_out)
{
    extern __shared__ zc sh[];
    const LRDesc d = descs[blockIdx.x];
    const int nr = d.nr, ncl = d.ncol, kmax = d.kmax, tid = threadIdx.x;
    zc *Urow = sh;          // [kmax]
    zc *Vrow = sh + kmax;   // [kmax]
    unsigned *used = (unsigned *)(Vrow + kmax);  // bitmask [nr/32 + 1]
    __shared__ double sv[ACA_WARPS + 1];
    __shared__ int si[ACA_WARPS + 1];
    __shared__ double cross_acc;
    const int nwords = (nr + 31) / 32;
    for (int i = tid; i < nwords; i += ACA_THREADS) used[i] = 0u;
    zc *U = d.U, *W = d.V;
    double S2 = 0.0;
    int k = 0, i = 0, flag = 0;
    __syncthreads();
    while (true) {
        if (k >= kmax) {
            flag = 1;
            break;
        }
        // pivot row cache
        for (int l = tid; l < k; l += ACA_THREADS) Urow[l] = U[(size_t)l * nr + i];
        __syncthreads();
        const int D = E.dof;
        const int ni = E.perm[d.r0 + i] / D, bi = (d.r0 + i) % D;
        // 1. residual row into W[:,k]
        double bv = -1.0;
        int bj = 0x7fffffff;
        for (int jj = tid; D * jj < ncl; jj += ACA_THREADS) {
            int nj = E.perm[d.c0 + D * jj] / D;
            zc e[16];
            pair_entries(E, ni, nj, e);
            for (int a = 0; a < D; ++a) {
                int j = D * jj + a;
                zc r = e[D * bi + a];
                for (int l = 0; l < k; ++l) r = zsub(r, zmul(Urow[l], zconj(W[(size_t)l * ncl + j])));
                W[(size_t)k * ncl + j] = r;
                double m = zabs2(r);
                argmax_merge(bv, bj, m, j);
            }
        }
        double mv;
        int jk;
        block_argmax(bv, bj, sv, si, mv, jk);
        if (!(mv > 1e-300)) {
            // zero residual row: mark used, move to the lowest unused row
            if (tid == 0) used[i >> 5] |= 1u << (i & 31);
            __syncthreads();
            int nexti = -1;
            for (int w = 0; w < nwords && nexti < 0; ++w) {
                unsigned m = ~used[w];
                if (w == nwords - 1 && (nr & 31)) m &= (1u << (nr & 31)) - 1u;
                if (m) nexti = w * 32 + __ffs(m) - 1;
            }
            __syncthreads();
            if (nexti < 0) break;
            i = nexti;
            continue;
        }
        const zc piv = W[(size_t)k * ncl + jk];
        __syncthreads();
        // 2. v_k = r / piv, stored as conj
        double nv2 = 0.0;
        for (int j = tid; j < ncl; j += ACA_THREADS) {
            zc v = zdiv(W[(size_t)k * ncl + j], piv);
            W[(size_t)k * ncl + j] = zconj(v);
            nv2 += zabs2(v);
        }
        for (int l = tid; l < k; l += ACA_THREADS) Vrow[l] = zconj(W[(size_t)l * ncl + jk]);
        if (tid == 0) used[i >> 5] |= 1u << (i & 31);
        __syncthreads();
        nv2 = block_sum(nv2, sv);
        // 3. residual column into U[:,k]
        const int nj = E.perm[d.c0 + jk] / D, aj = (d.c0 + jk) % D;
        double nu2 = 0.0;
        bv = -1.0;
        bj = 0x7fffffff;
        for (int ii = tid; D * ii < nr; ii += ACA_THREADS) {
            int nii = E.perm[d.r0 + D * ii] / D;
            zc e[16];
            pair_entries(E, nii, nj, e);
            for (int b = 0; b < D; ++b) {
                int row = D * ii + b;
                zc c = e[D * b + aj];
                for (int l = 0; l < k; ++l) c = zsub(c, zmul(U[(size_t)l * nr + row], Vrow[l]));
                U[(size_t)k * nr + row] = c;
                double m = zabs2(c);
                nu2 += m;
                if (!((used[row >> 5] >> (row & 31)) & 1u)) argmax_merge(bv, bj, m, row);
            }
        }
        __syncthreads();
        nu2 = block_sum(nu2, sv);
        int inext;
        double mu;
        block_argmax(bv, bj, sv, si, mu, inext);
        // 4. norm update: cross terms (u_l^H u_k)(v_l^H v_k), v_l^H v_k = sum_j W_l[j] conj(W_k[j])
        if (tid == 0) cross_acc = 0.0;
        __syncthreads();
        {
            int w = tid >> 5, lane = tid & 31;
            double part = 0.0;
            for (int l = w; l < k; l += ACA_WARPS) {
                zc a = zmake(0, 0), b = zmake(0, 0);
                for (int r = lane; r < nr; r += 32) a = zfmac(U[(size_t)l * nr + r], U[(size_t)k * nr + r], a);
                for (int j = lane; j < ncl; j += 32) b = zfmac(W[(size_t)k * ncl + j], W[(size_t)l * ncl + j], b);
                for (int o = 16; o > 0; o >>= 1) {
                    a.x += __shfl_down_sync(0xffffffff, a.x, o);
                    a.y += __shfl_down_sync(0xffffffff, a.y, o);
                    b.x += __shfl_down_sync(0xffffffff, b.x, o);
                    b.y += __shfl_down_sync(0xffffffff, b.y, o);
                }
                if (lane == 0) part += zmul(a, b).x;
            }
            if (lane == 0 && part != 0.0) atomicAdd(&cross_acc, part);
        }
        __syncthreads();
        S2 += 2.0 * cross_acc + nu2 * nv2;
        ++k;
        if (nu2 * nv2 <= tol * tol * S2) break;
        if (inext < 0 || inext >= nr || !(mu >= 0.0)) {
            // all rows used
            break;
        }
        i = inext;
        __syncthreads();
    }
    if (tid == 0) {
        rank_out[blockIdx.x] = k;
        flag_out[blockIdx.x] = flag;
    }
}

void launch_aca(hm_handle_s *h, const std::vector<LRDesc> &descs, int *d_rank, int *d_flag)
{
    if (descs.empty()) return;
    int kmax = 0, nrmax = 0;
    for (auto &d : descs) {
        kmax = std::max(kmax, d.kmax);
        nrmax = std::max(nrmax, d.nr);
    }
    if (nrmax > ACA_MAXROWS) throw HmError{HM_ERR_ARG, "ACA block too large"};
    size_t smem = sizeof(zc) * 2 * kmax + sizeof(unsigned) * ((nrmax + 31) / 32 + 1);
    HM_CUDA(cudaFuncSetAttribute(k_aca, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    LRDesc *d_desc = (LRDesc *)dalloc(h, sizeof(LRDesc) * descs.size());
    HM_CUDA(cudaMemcpyAsync(d_desc, descs.data(), sizeof(LRDesc) * descs.size(), cudaMemcpyHostToDevice, h->stream));
    k_aca<<<(unsigned)descs.size(), ACA_THREADS, smem, h->stream>>>(entry_ctx(h), d_desc, h->tol, d_rank, d_flag);
    HM_CHECK_LAUNCH();
    count_launch(h);
    HM_CUDA(cudaStreamSynchronize(h->stream));
    dfree(h, d_desc);
}
