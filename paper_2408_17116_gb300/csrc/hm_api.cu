// C ABI of libhm (declared in include/hm.h).  Every entry point converts internal
// errors to an hm_status and stores the message for hm_last_error.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>

#include "hm_internal.h"

#define HM_VERSION "hm-cbie-gb300 0.2 (MFIE; FP64 H-LU or FP32 H-LU + FP64 refinement)"
#define HM_DEFAULT_RANK_CAP 160

void *dalloc(hm_handle_s *h, size_t bytes)
{
    if (h->fault == HM_FAULT_ALLOC) {  // host-side injection: this allocation reports failure
        h->fault = HM_FAULT_NONE;
        throw HmError{HM_ERR_OOM, "device allocation failed (injected)"};
    }
    void *p = nullptr;
    cudaError_t e = cudaMallocAsync(&p, std::max<size_t>(bytes, 16), h->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw HmError{HM_ERR_OOM, std::string("device allocation of ") + std::to_string(bytes) + " bytes failed"};
    }
    return p;
}

void dfree(hm_handle_s *h, void *p)
{
    if (p) cudaFreeAsync(p, h->stream);
}

void pool_fork(hm_handle_s *h, int n)
{
    n = std::min(n, HM_POOL_STREAMS);
    while ((int)h->pool.size() < n) {
        cudaStream_t s;
        cudaEvent_t e;
        HM_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        HM_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        h->pool.push_back(s);
        h->pool_ev.push_back(e);
    }
    cudaEvent_t e = h->pool_ev[0];
    HM_CUDA(cudaEventRecord(e, h->stream));
    for (int i = 0; i < n; ++i) HM_CUDA(cudaStreamWaitEvent(h->pool[i], e, 0));
}

void pool_join(hm_handle_s *h, int n)
{
    n = std::min(n, HM_POOL_STREAMS);
    for (int i = 0; i < n; ++i) {
        HM_CUDA(cudaEventRecord(h->pool_ev[i], h->pool[i]));
        HM_CUDA(cudaStreamWaitEvent(h->stream, h->pool_ev[i], 0));
    }
}

namespace {

struct Timer {
    cudaEvent_t a, b;
    cudaStream_t s;
    Timer(cudaStream_t st) : s(st)
    {
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        cudaEventRecord(a, s);
    }
    double stop()
    {
        cudaEventRecord(b, s);
        cudaEventSynchronize(b);
        float ms = 0;
        cudaEventElapsedTime(&ms, a, b);
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        return ms * 1e-3;
    }
};

template <class F>
hm_status guard(hm_handle h, F &&f)
{
    if (!h) return HM_ERR_ARG;
    try {
        f();
        h->err.clear();
        return HM_OK;
    } catch (const HmError &e) {
        h->err = e.msg;
        return e.st;
    } catch (const std::bad_alloc &) {
        h->err = "host allocation failed";
        return HM_ERR_OOM;
    } catch (...) {
        h->err = "unknown error";
        return HM_ERR_CUDA;
    }
}

void free_plans(hm_handle_s *h)
{
    tile_free(h, h->tmat64);
    tile_free(h, h->tmatcopy);
    tile_free(h, h->tfac64);
    tile_free(h, h->tfac32);
    h->tmat64 = h->tmatcopy = h->tfac64 = nullptr;
    h->tfac32 = nullptr;
}

void free_matrix(hm_handle_s *h)
{
    free_plans(h);
    for (Block *b : h->blocks) {
        if (b->D) dfree(h, b->D);
        if (b->U) dfree(h, b->U);
        if (b->V) dfree(h, b->V);
        if (b->piv) dfree(h, b->piv);
        for (zc *q : b->pu) dfree(h, q);
        for (zc *q : b->pv) dfree(h, q);
        b->pu.clear();
        b->pv.clear();
        b->pk.clear();
        b->pend_k = 0;
        b->D = b->U = b->V = nullptr;
        b->piv = nullptr;
        b->k = 0;
    }
    free_tree(h, h->copy_blocks);
    h->copy_root = nullptr;
    free_tree(h, h->blocks32);
    h->root32 = nullptr;
}

void free_all(hm_handle_s *h)
{
    free_matrix(h);
    for (Block *b : h->blocks) delete b;
    h->blocks.clear();
    h->leaves.clear();
    h->root = nullptr;
    void *ptrs[] = {h->d_bodies, h->d_patches, h->d_nodes, h->d_pair_q, h->d_pair_p, h->d_nearidx,
                    h->d_near,   h->d_perm,    h->d_iperm, h->d_d1,     h->d_patch_body};
    for (void *p : ptrs) dfree(h, p);
    h->d_patch_body = nullptr;
    h->d_bodies = nullptr;
    h->d_patches = nullptr;
    h->d_nodes = nullptr;
    h->d_pair_q = h->d_pair_p = h->d_nearidx = nullptr;
    h->d_near = nullptr;
    h->d_perm = h->d_iperm = nullptr;
    h->d_d1 = nullptr;
    for (auto &w : h->tc_ws) dfree(h, w.p);
    h->tc_ws.clear();
}

void collect_leaves(Block *b, std::vector<Block *> &out)
{
    if (b->type == B_HIER) {
        for (int i = 0; i < 4; ++i) collect_leaves(b->ch[i], out);
    } else {
        b->leaf_id = (int)out.size();
        out.push_back(b);
    }
}

void rebuild_leaves(hm_handle_s *h)
{
    h->leaves.clear();
    collect_leaves(h->root, h->leaves);
}

void storage(hm_handle_s *h, Block *root_unused, double &words, int &maxk, double &meank, int &ndense, int &nlr)
{
    (void)root_unused;
    words = 0;
    maxk = 0;
    ndense = nlr = 0;
    double ks = 0;
    for (Block *b : h->leaves) {
        if (b->type == B_DENSE && !b->D) continue;  // merged into a dense block of the factor
        if (b->type == B_DENSE) {
            words += (double)b->nr * b->nc;
            ++ndense;
        } else {
            words += (double)b->k * (b->nr + b->nc);
            maxk = std::max(maxk, b->k);
            ks += b->k;
            ++nlr;
        }
    }
    meank = nlr ? ks / nlr : 0.0;
}

}  // namespace

// Geometric features of an admissible block (t, s) read by the rank model:
// log2 of both sizes, both cluster diameters and their separation in wavelengths,
// the separation ratio of Eq. 21, nodes per direction and the ACA tolerance.
void rank_features(hm_handle_s *h, const Block *b, float *f)
{
    const Cluster &ct = h->clusters[b->t], &cs = h->clusters[b->s];
    double dt = 0, ds = 0, g2 = 0;
    for (int d = 0; d < 3; ++d) {
        dt += (ct.bmax[d] - ct.bmin[d]) * (ct.bmax[d] - ct.bmin[d]);
        ds += (cs.bmax[d] - cs.bmin[d]) * (cs.bmax[d] - cs.bmin[d]);
        double g = std::max(0.0, std::max(ct.bmin[d] - cs.bmax[d], cs.bmin[d] - ct.bmax[d]));
        g2 += g * g;
    }
    dt = std::sqrt(dt);
    ds = std::sqrt(ds);
    double dist = std::sqrt(g2);
    const double lam = h->prm.k0 > 0 ? 2.0 * 3.14159265358979323846 / h->prm.k0 : 1.0;
    f[0] = (float)(std::log2((double)b->nr) / 10.0);
    f[1] = (float)(std::log2((double)b->nc) / 10.0);
    f[2] = (float)(dt / lam / 8.0);
    f[3] = (float)(ds / lam / 8.0);
    f[4] = (float)(dist / lam / 8.0);
    f[5] = (float)(std::max(dt, ds) / std::max(dist, 1e-300) / 4.0);
    f[6] = (float)(h->nc / 10.0);
    f[7] = (float)(-std::log10(h->tol) / 10.0);
}

// Cluster level from which the factor stores dense blocks.  factor_leaf > 0: the first
// level whose clusters hold at most factor_leaf unknowns.  factor_leaf = 0: the coarsest
// level of clusters of at most `cap` unknowns (4,096 for the complex64 factor, 1,280 for
// the complex128 one) whose non-low-rank blocks store at least 35 % of their dense size in
// H-format, else the level of 640-unknown clusters.  -1 when factor_leaf is negative.
// (Measured on GB300 at 19,200 unknowns, where the near blocks store 47 % of their dense
// size: the factor with dense 2,400-unknown blocks takes 3.4 s, with dense 600-unknown
// blocks and low-rank blocks above them 13 s, recompressions dominating the latter.)
template <class Z>
static int dense_level(hm_handle_s *h, BlockT<Z> *root, bool c64)
{
    if (h->prm.factor_leaf < 0) return -1;
    auto level_of = [&](int bd) {
        int lev = 0;
        while (h->dof * ((h->nnode + (1 << lev) - 1) >> lev) > bd && (1 << lev) < h->nnode) ++lev;
        return lev;
    };
    if (h->prm.factor_leaf > 0) return level_of(h->prm.factor_leaf);
    if (h->prm.independent) return HM_MERGE_BODIES;  // each body's diagonal block, dense
    // A dense block factors at the rate of large products (tensor cores for complex64, the
    // FP64 pipe at its peak for complex128) while the formatted arithmetic below it runs
    // small, latency-bound kernels: merge from the coarsest level whose dense storage fits
    // in 40 % of the free device memory.  Without tensor cores the dense blocks are kept to
    // clusters of at most 24,576 unknowns (a dense FP64 LU of that size takes seconds).
    size_t fr = 0, tot = 0;
    HM_CUDA(cudaMemGetInfo(&fr, &tot));
    const int Lm = dense_level_by_memory<Z>(h, root, 0.4 * (double)fr / (c64 ? sizeof(cf) : sizeof(zc)));
    if (Lm >= 0) {
        if (c64 && !h->prm.simt_gemm) return Lm;
        return std::max(Lm, level_of(24576));
    }
    const int cap = c64 ? 4096 : 1280;
    const int L = dense_level_by_storage<Z>(h, root, cap, 0.35);
    return L >= 0 ? L : level_of(640);
}

// The first diagonal dense leaf of a block tree (the top-left leaf).
template <class Z>
static BlockT<Z> *first_diagonal_leaf(BlockT<Z> *b)
{
    while (b->type == B_HIER) b = b->ch[0];
    return b;
}

extern "C" {

const char *hm_version(void) { return HM_VERSION; }

hm_status hm_create(hm_handle *out, void *stream)
{
    if (!out) return HM_ERR_ARG;
    *out = nullptr;
    hm_handle_s *h = new (std::nothrow) hm_handle_s();
    if (!h) return HM_ERR_OOM;
    h->stream = (cudaStream_t)stream;
    if (cudaGetDevice(&h->device) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return HM_ERR_CUDA;
    }
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, h->device) == cudaSuccess) {
        uint64_t thr = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    if (cudaMalloc(&h->d_counter, sizeof(unsigned long long) * 4) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return HM_ERR_OOM;
    }
    cudaMemset(h->d_counter, 0, sizeof(unsigned long long) * 4);
    *out = h;
    return HM_OK;
}

hm_status hm_build_geometry(hm_handle h, const hm_body *bodies, int nbodies, int nodes_per_dir, const hm_params *p)
{
    return guard(h, [&] {
        if (!bodies || nbodies <= 0 || !p) throw HmError{HM_ERR_ARG, "null bodies or params"};
        if (nodes_per_dir < 2 || nodes_per_dir > HM_NC_MAX) throw HmError{HM_ERR_ARG, "nodes_per_dir out of range 2..16"};
        if (p->formulation == HM_PEC_CFIE)
            throw HmError{HM_ERR_ARG, "formulation HM_PEC_CFIE is not built in this library"};
        if (p->formulation != HM_PEC_MFIE && p->formulation != HM_DIEL_MULLER)
            throw HmError{HM_ERR_ARG, "unknown formulation"};
        if (p->formulation == HM_DIEL_MULLER) {
            if (!(p->eps_r_re > 0.0) || !(p->eps_r_im <= 0.0) || !std::isfinite(p->eps_r_re) ||
                !std::isfinite(p->eps_r_im))
                throw HmError{HM_ERR_ARG, "eps_r needs a positive real part and Im <= 0 (exp(j w t))"};
            if (!(p->mu_r == 0.0 || p->mu_r == 1.0)) throw HmError{HM_ERR_ARG, "only mu_r = 1 is supported"};
            if (nodes_per_dir > 12) throw HmError{HM_ERR_ARG, "N-Mueller: nodes_per_dir at most 12"};
            if (!(p->k0 > 0.0)) throw HmError{HM_ERR_ARG, "N-Mueller: k0 must be positive"};
        }
        if (!(p->trunc_tol >= 0.0) || p->quad_order < 0 || (p->quad_order > 0 && (p->quad_order < 4 || p->quad_order > 36)))
            throw HmError{HM_ERR_ARG, "trunc_tol must be >= 0 and quad_order 0 or 4..36"};
        if (p->precision != HM_FP64 && p->precision != HM_FP32_REFINED) throw HmError{HM_ERR_ARG, "unsupported precision"};
        if (!(p->factor_tol >= 0.0) || !(p->refine_tol >= 0.0) || p->refine_max_iter < 0)
            throw HmError{HM_ERR_ARG, "invalid refinement parameter"};
        if (!(p->k0 >= 0.0) || !std::isfinite(p->k0) || p->leaf < 2 || !(p->eta > 0.0) || !(p->aca_tol > 0.0) || !(p->near_delta >= 0.0))
            throw HmError{HM_ERR_ARG, "invalid parameter value"};
        long long P = 0;
        for (int b = 0; b < nbodies; ++b) {
            if (bodies[b].family != 0 || bodies[b].m < 1 || bodies[b].m > 256) throw HmError{HM_ERR_ARG, "bad body"};
            for (int d = 0; d < 3; ++d)
                if (!(bodies[b].semi_axes[d] > 0.0) || !std::isfinite(bodies[b].semi_axes[d]))
                    throw HmError{HM_ERR_ARG, "semi-axes must be positive and finite"};
            for (int d = 0; d < 3; ++d)
                if (!std::isfinite(bodies[b].center[d])) throw HmError{HM_ERR_ARG, "body centre is not finite"};
            for (int d = 0; d < 9; ++d)
                if (!std::isfinite(bodies[b].rot[d])) throw HmError{HM_ERR_ARG, "body rotation is not finite"};
            P += 6LL * bodies[b].m * bodies[b].m;
        }
        if (P * nodes_per_dir * nodes_per_dir * 2 > (1LL << 30)) throw HmError{HM_ERR_ARG, "problem too large"};
        cudaStreamSynchronize(h->stream);
        free_all(h);
        h->prm = *p;
        h->tol = p->aca_tol;
        h->trunc_tol = p->trunc_tol > 0.0 ? p->trunc_tol : p->aca_tol;
        h->factor_tol = p->factor_tol > 0.0 ? p->factor_tol : 1e-4;
        if (p->quad_order > 0) {
            h->rule.qd = h->rule.qi = p->quad_order;
            h->rule.qo = (2 * p->quad_order + 2) / 3;
        } else {
            h->rule = NearRule{24, 24, 16, 0.5};
        }
        if (h->prm.refine_tol <= 0.0) h->prm.refine_tol = 1e-10;
        if (h->prm.refine_max_iter <= 0) h->prm.refine_max_iter = 30;
        h->nc = nodes_per_dir;
        h->nbodies = nbodies;
        h->bodies.clear();
        h->patches.clear();
        for (int b = 0; b < nbodies; ++b) {
            DevBody B{};
            const hm_body &hb = bodies[b];
            for (int a = 0; a < 3; ++a) {
                B.c[a] = hb.center[a];
                for (int d = 0; d < 3; ++d) {
                    B.M[3 * a + d] = hb.rot[3 * a + d] * hb.semi_axes[d];
                    B.Minv[3 * a + d] = hb.rot[3 * d + a] / hb.semi_axes[a];
                }
            }
            B.m = hb.m;
            h->bodies.push_back(B);
            for (int f = 0; f < 6; ++f)
                for (int i = 0; i < hb.m; ++i)
                    for (int j = 0; j < hb.m; ++j) h->patches.push_back(DevPatch{b, f, i, j});
        }
        h->npatch = (int)h->patches.size();
        h->nnode = h->npatch * h->nc * h->nc;
        h->dof = h->prm.formulation == HM_DIEL_MULLER ? 4 : 2;
        h->N = h->dof * h->nnode;
        if (h->prm.formulation == HM_DIEL_MULLER && p->quad_order == 0) {
            // the rule must resolve the interior wavelength: twice the points above a
            // contrast of 3 in the wavenumber
            const double kr = std::sqrt(std::hypot(p->eps_r_re, p->eps_r_im));
            if (kr > 3.0) h->rule = NearRule{48, 48, 32, 0.5};
        }
        Timer t(h->stream);
        plan_geometry(h);
        h->t_geom = t.stop();
        h->state = 1;
    });
}

hm_status hm_fill(hm_handle h)
{
    return guard(h, [&] {
        if (h->state < 1) throw HmError{HM_ERR_STATE, "hm_fill before hm_build_geometry"};
        if (h->state > 1) {
            free_matrix(h);
            rebuild_block_tree(h);  // the adaptive ACA split below changes the tree
        }
        const int nc = h->nc, w = h->dof * nc * nc;
        h->tr_batches = h->tr_jobs = h->tr_maxk = h->tr_work = h->tr_seconds = 0;
        h->kqr_s = h->kqr_flops = h->kqr_n = h->kcore_s = h->kcore_flops = h->kcore_n = 0;
        h->trunc_log.clear();
        // near-field quadrature (A3)
        {
            Timer t(h->stream);
            if (!h->d_near) h->d_near = (zc *)dalloc(h, sizeof(zc) * (size_t)h->pair_q.size() * w * w);
            NearRule R = h->rule;
            std::vector<double> tab;
            auto add_gl = [&](int q) {
                std::vector<double> x(q), wt(q);
                gauss_legendre_host(q, x.data(), wt.data());
                std::vector<int> o(q);
                for (int i = 0; i < q; ++i) o[i] = i;
                std::sort(o.begin(), o.end(), [&](int a, int b) { return x[a] < x[b]; });
                for (int i = 0; i < q; ++i) tab.push_back(0.5 * (x[o[i]] + 1.0));
                for (int i = 0; i < q; ++i) tab.push_back(0.5 * wt[o[i]]);
            };
            add_gl(R.qd);
            add_gl(R.qi);
            add_gl(R.qo);
            std::vector<double> x1d(nc);
            cheb_nodes_host(nc, x1d.data());
            for (int l = 0; l < nc; ++l) tab.push_back(x1d[l]);
            // C[n][l] = alpha_n T_n(x_l) / nc  (Eq. 13)
            std::vector<double> C(nc * nc);
            for (int n = 0; n < nc; ++n)
                for (int l = 0; l < nc; ++l) {
                    double th = 3.14159265358979323846 * (2 * l + 1) / (2.0 * nc);
                    C[n * nc + l] = (n == 0 ? 1.0 : 2.0) * std::cos(n * th) / nc;
                }
            double *d_tab = (double *)dalloc(h, sizeof(double) * (tab.size() + C.size()));
            HM_CUDA(cudaMemcpyAsync(d_tab, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice, h->stream));
            HM_CUDA(cudaMemcpyAsync(d_tab + tab.size(), C.data(), sizeof(double) * C.size(), cudaMemcpyHostToDevice,
                                    h->stream));
            HM_CUDA(cudaMemsetAsync(h->d_counter, 0, sizeof(unsigned long long), h->stream));
            if (h->dof == 4) {
                // derivatives of the cardinal functions at the nodes (the divergence terms of
                // the far entries): d1[l' nc + l] = ell_l'(x_l') = sum_n C[n][l] T_n'(x_l')
                std::vector<double> x1(nc), d1((size_t)nc * nc), U(nc + 1);
                cheb_nodes_host(nc, x1.data());
                for (int lp = 0; lp < nc; ++lp) {
                    U[0] = 1.0;
                    U[1] = 2.0 * x1[lp];
                    for (int j = 2; j < nc; ++j) U[j] = 2.0 * x1[lp] * U[j - 1] - U[j - 2];
                    for (int l = 0; l < nc; ++l) {
                        double s = 0.0;
                        for (int n = 1; n < nc; ++n) s += C[n * nc + l] * n * U[n - 1];  // T_n' = n U_{n-1}
                        d1[lp * nc + l] = s;
                    }
                }
                if (!h->d_d1) h->d_d1 = (double *)dalloc(h, sizeof(double) * nc * nc);
                HM_CUDA(cudaMemcpyAsync(h->d_d1, d1.data(), sizeof(double) * d1.size(), cudaMemcpyHostToDevice,
                                        h->stream));
                HM_CUDA(cudaStreamSynchronize(h->stream));
                launch_near_muller(h, d_tab, d_tab + tab.size());
            } else {
                launch_near(h, d_tab, d_tab + tab.size());
            }
            dfree(h, d_tab);
            h->t_near = t.stop();
            HM_CUDA(cudaMemcpy(&h->near_points, h->d_counter, sizeof(unsigned long long), cudaMemcpyDeviceToHost));
        }
        // ACA of admissible leaves (A5).  A block whose ACA reaches its rank bound is split
        // into its four (still admissible) children and retried; at the leaf level it is
        // stored dense.  Dense blocks therefore only occur on the leaf level.
        // With a rank model: a block whose predicted rank is at least 1.25 times its bound
        // is split (or, on the leaf level, stored dense) without the doomed ACA attempt;
        // otherwise the predicted rank sizes the block's buffers and orders the launch
        // (largest predicted first), and a block whose ACA stops at a predicted bound below
        // its real bound is re-run with the real bound (plain adaptive ACA).
        {
            Timer t(h->stream);
            std::vector<Block *> pending;
            for (Block *b : h->leaves)
                if (b->type == B_LR && !b->zero) pending.push_back(b);
            int cap = h->prm.aca_max_rank > 0 ? h->prm.aca_max_rank : HM_DEFAULT_RANK_CAP;
            h->aca_nonconv = 0;
            h->aca_reruns = 0;
            h->aca_skipped = 0;
            h->aca_prealloc = 0;
            h->rank_feat.clear();
            h->rank_target.clear();
            double pred_err = 0;
            int npred = 0;
            std::vector<int> rerun_bound;  // per pending block: 0 = first attempt, else the bound to use
            rerun_bound.assign(pending.size(), 0);
            while (!pending.empty()) {
                const size_t np = pending.size();
                std::vector<int> bound(np), kmaxv(np);
                std::vector<float> feat((size_t)HM_RANK_NFEAT * np), pred(np, -1.0f);
                for (size_t i = 0; i < np; ++i) {
                    Block *b = pending[i];
                    bound[i] = std::max(1, std::min(cap, (int)((long long)b->nr * b->nc / (b->nr + b->nc))));
                    rank_features(h, b, &feat[HM_RANK_NFEAT * i]);
                }
                if (h->rank_model) mlp_predict_host(h->rank_model, (int)np, feat.data(), pred.data());
                std::vector<size_t> order(np);
                for (size_t i = 0; i < np; ++i) {
                    order[i] = i;
                    int km = bound[i];
                    if (h->rank_model && !rerun_bound[i]) {
                        double pk = std::exp((double)pred[i]) - 1.0;
                        km = pk >= 1.25 * bound[i] ? 0  // predicted to fail: no attempt
                                                   : std::min(bound[i], std::max(4, (int)std::ceil(1.25 * pk + 4.0)));
                    } else if (rerun_bound[i]) {
                        km = rerun_bound[i];
                    }
                    kmaxv[i] = km;
                }
                if (h->rank_model)
                    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return kmaxv[a] > kmaxv[b]; });
                std::vector<Block *> sorted(np);
                std::vector<int> sb(np), sk(np), sr(np);
                std::vector<float> sp(np);
                std::vector<float> sf((size_t)HM_RANK_NFEAT * np);
                for (size_t i = 0; i < np; ++i) {
                    sorted[i] = pending[order[i]];
                    sb[i] = bound[order[i]];
                    sk[i] = kmaxv[order[i]];
                    sr[i] = rerun_bound[order[i]];
                    sp[i] = pred[order[i]];
                    std::copy(&feat[HM_RANK_NFEAT * order[i]], &feat[HM_RANK_NFEAT * (order[i] + 1)],
                              &sf[HM_RANK_NFEAT * i]);
                }
                pending.swap(sorted);
                std::vector<LRDesc> descs;
                std::vector<int> slot(np, -1);
                for (size_t i = 0; i < np; ++i) {
                    Block *b = pending[i];
                    int kmax = sk[i];
                    if (kmax == 0) {
                        ++h->aca_skipped;
                        continue;
                    }
                    b->U = (zc *)dalloc(h, sizeof(zc) * (size_t)b->nr * kmax);
                    b->V = (zc *)dalloc(h, sizeof(zc) * (size_t)b->nc * kmax);
                    h->aca_prealloc += (double)kmax * (b->nr + b->nc);
                    slot[i] = (int)descs.size();
                    descs.push_back(LRDesc{b->r0, b->nr, b->c0, b->nc, b->U, b->V, kmax});
                }
                const size_t nd = descs.size();
                std::vector<int> rf(2 * nd);
                if (nd) {
                    int *d_rf = (int *)dalloc(h, sizeof(int) * 2 * nd);
                    launch_aca(h, descs, d_rf, d_rf + nd);
                    HM_CUDA(cudaMemcpyAsync(rf.data(), d_rf, sizeof(int) * rf.size(), cudaMemcpyDeviceToHost,
                                            h->stream));
                    HM_CUDA(cudaStreamSynchronize(h->stream));
                    dfree(h, d_rf);
                }
                std::vector<Block *> next;
                std::vector<int> next_rerun;
                for (size_t i = 0; i < pending.size(); ++i) {
                    Block *b = pending[i];
                    const bool skipped = slot[i] < 0;
                    const bool hit = skipped || rf[nd + slot[i]] != 0;
                    const int rank_i = skipped ? 0 : rf[slot[i]];
                    if (!skipped && (!hit || sk[i] == sb[i])) {
                        // training sample, log(1 + rank): the rank ACA reached, or twice the bound
                        // for a block that reached its bound (its rank is only known to exceed it)
                        h->rank_feat.insert(h->rank_feat.end(), &sf[HM_RANK_NFEAT * i], &sf[HM_RANK_NFEAT * (i + 1)]);
                        h->rank_target.push_back((float)std::log(1.0 + (hit ? 2.0 * sb[i] : rank_i)));
                        if (h->rank_model) {
                            pred_err += std::fabs((double)sp[i] - h->rank_target.back());
                            ++npred;
                        }
                    }
                    if (!hit) {
                        b->k = rank_i;
                        continue;
                    }
                    if (!skipped && sk[i] < sb[i]) {
                        // the prediction was too low: plain adaptive ACA with the real bound
                        dfree(h, b->U);
                        dfree(h, b->V);
                        b->U = b->V = nullptr;
                        ++h->aca_reruns;
                        next.push_back(b);
                        next_rerun.push_back(sb[i]);
                        continue;
                    }
                    if (!skipped) ++h->aca_nonconv;
                    dfree(h, b->U);
                    dfree(h, b->V);
                    b->U = b->V = nullptr;
                    b->k = 0;
                    const Cluster &ct = h->clusters[b->t], &cs = h->clusters[b->s];
                    if (ct.child[0] >= 0 && cs.child[0] >= 0) {
                        b->type = B_HIER;
                        for (int a = 0; a < 2; ++a)
                            for (int c = 0; c < 2; ++c) {
                                Block *ch = new Block();
                                h->blocks.push_back(ch);
                                const Cluster &t2 = h->clusters[ct.child[a]], &s2 = h->clusters[cs.child[c]];
                                ch->t = ct.child[a];
                                ch->s = cs.child[c];
                                ch->r0 = h->dof * t2.off;
                                ch->nr = h->dof * t2.cnt;
                                ch->c0 = h->dof * s2.off;
                                ch->nc = h->dof * s2.cnt;
                                ch->type = B_LR;
                                b->ch[2 * a + c] = ch;
                                next.push_back(ch);
                                next_rerun.push_back(0);
                            }
                    } else {
                        b->type = B_DENSE;
                    }
                }
                pending.swap(next);
                rerun_bound.swap(next_rerun);
            }
            h->rank_pred_err = npred ? pred_err / npred : 0.0;
            rebuild_leaves(h);
            h->t_aca = t.stop();
        }
        // QR + SVD recompression of every low-rank leaf (A6).  In HM_FP32_REFINED mode the
        // FP64 H-matrix only serves the refinement residual: it keeps the ACA factors, and
        // the complex64 copy is recompressed to factor_tol when hm_factor starts.
        h->t_trunc = 0;
        if (h->prm.precision != HM_FP32_REFINED) {
            Timer t(h->stream);
            std::vector<Block *> keep;
            std::vector<int> ranks;
            for (Block *b : h->leaves)
                if (b->type == B_LR && b->k > 0) {
                    keep.push_back(b);
                    ranks.push_back(b->k);
                }
            batched_truncate(h, keep, ranks, h->trunc_tol);
            h->t_trunc = t.stop();
        }
        // dense leaves (A4)
        {
            Timer t(h->stream);
            std::vector<DenseDesc> dd;
            for (Block *b : h->leaves)
                if (b->type == B_DENSE) {
                    b->D = (zc *)dalloc(h, sizeof(zc) * (size_t)b->nr * b->nc);
                    dd.push_back(DenseDesc{b->r0, b->nr, b->c0, b->nc, b->D});
                }
            launch_dense_fill(h, dd);
            h->t_dense = t.stop();
        }
        h->state = 2;
    });
}

hm_status hm_factor(hm_handle h)
{
    return guard(h, [&] {
        if (h->state != 2) throw HmError{HM_ERR_STATE, "hm_factor requires a filled, unfactored matrix"};
        const bool zero_pivot = h->fault == HM_FAULT_ZERO_PIVOT;
        if (zero_pivot) h->fault = HM_FAULT_NONE;
        h->flops_factor = 0;
        h->tr_batches = h->tr_jobs = h->tr_maxk = h->tr_work = h->tr_seconds = 0;
        h->kqr_s = h->kqr_flops = h->kqr_n = h->kcore_s = h->kcore_flops = h->kcore_n = 0;
        h->trunc_log.clear();
        gemm_timing_collect(h);
        h->kgemm_s = h->kgemm_flops = h->kgemm_n = 0;
        h->ktc_s = h->ktc_flops = h->ktc_n = 0;
        phase_collect(h);
        h->phase_s[PH_LU_PANEL] = h->phase_s[PH_LU_U12] = h->phase_s[PH_TILE_BUILD] = 0;
        if (h->prm.precision == HM_FP32_REFINED) {
            // the FP64 H-matrix stays unfactored: it is the refinement operator
            Timer t(h->stream);
            tile_free(h, h->tfac32);
            h->tfac32 = nullptr;
            free_tree(h, h->blocks32);
            h->dirty32.clear();
            // with tensor-core products the dense level does not depend on the ranks: the copy
            // is made with its dense blocks already merged (one batched expansion), and only
            // the low-rank leaves that stay are recompressed
            const bool merge_first = !h->prm.simt_gemm && h->prm.factor_leaf >= 0;
            int lev = -1;
            if (merge_first) lev = dense_level<zc>(h, h->root, true);
            if (lev != -1)
                h->root32 = clone_tree_merged(h, h->root, lev, h->blocks32);
            else
                h->root32 = clone_tree<cf>(h, h->root, h->blocks32);
            // the factor only needs factor_tol: recompress the copied low-rank leaves
            std::vector<Block32 *> lr;
            std::vector<int> ranks;
            for (Block32 *b : h->blocks32)
                if (b->type == B_LR && b->k > 0) {
                    lr.push_back(b);
                    ranks.push_back(b->k);
                }
            batched_truncate<cf>(h, lr, ranks, h->factor_tol);
            if (!merge_first) {
                lev = dense_level<cf>(h, h->root32, true);
                if (lev != -1) coarsen_tree<cf>(h, h->root32, lev);
            }
            h->dense_lev = lev;
            if (zero_pivot) {  // host-side injection: the first column of the first leaf is zero
                Block32 *d = first_diagonal_leaf(h->root32);
                HM_CUDA(cudaMemsetAsync(d->D, 0, sizeof(cf) * d->nr, h->stream));
            }
            hlu_factor<cf>(h, h->root32, h->factor_tol);
            tile_free(h, h->tfac32);
            h->tfac32 = tile_build<cf>(h, h->root32, true);
            if (!h->tmat64) h->tmat64 = tile_build<zc>(h, h->root, false);
            h->t_factor = t.stop();
            tc_check(h);
            gemm_timing_collect(h);
            h->state = 3;
            return;
        }
        if (h->prm.keep_matrix) {
            tile_free(h, h->tmatcopy);
            h->tmatcopy = nullptr;
            free_tree(h, h->copy_blocks);
            h->copy_root = clone_tree<zc>(h, h->root, h->copy_blocks);
        }
        Timer t(h->stream);
        h->dirty64.clear();
        const int lev = dense_level<zc>(h, h->root, false);
        if (lev != -1) {
            coarsen_tree<zc>(h, h->root, lev);
            rebuild_leaves(h);
        }
        h->dense_lev = lev;
        if (zero_pivot) {  // host-side injection: the first column of the first leaf is zero
            Block *d = first_diagonal_leaf(h->root);
            HM_CUDA(cudaMemsetAsync(d->D, 0, sizeof(zc) * d->nr, h->stream));
        }
        tile_free(h, h->tmat64);  // the tree now holds the factors
        h->tmat64 = nullptr;
        hlu_factor<zc>(h, h->root, h->trunc_tol);
        tile_free(h, h->tfac64);
        h->tfac64 = tile_build<zc>(h, h->root, true);
        h->t_factor = t.stop();
        gemm_timing_collect(h);
        h->state = 3;
    });
}

// Per-column squared 2-norms of X (rows x cols, ld = rows): out[c] = sum_i |X[i,c]|^2.
__global__ void k_colnorm2(const zc *__restrict__ X, int rows, double *__restrict__ out)
{
    const zc *x = X + (size_t)blockIdx.x * rows;
    double s = 0;
    for (int i = threadIdx.x; i < rows; i += blockDim.x) s += zabs2(x[i]);
    __shared__ double sh[32];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffff, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
        out[blockIdx.x] = t;
    }
}

// x += d (n complex values)
__global__ void k_axpy1(const zc *__restrict__ d, zc *__restrict__ x, size_t n)
{
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = zadd(x[i], d[i]);
}

// Number of non-finite real or imaginary parts among n complex values, added to *cnt.
__global__ void k_nonfinite(const zc *__restrict__ x, size_t n, int *cnt)
{
    int bad = 0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        bad += !(isfinite(x[i].x) && isfinite(x[i].y));
    for (int o = 16; o > 0; o >>= 1) bad += __shfl_down_sync(0xffffffff, bad, o);
    if ((threadIdx.x & 31) == 0 && bad) atomicAdd(cnt, bad);
}

// Throws HM_ERR_NUMERIC when x (n complex values, device) holds a NaN or an infinity.
static void check_finite(hm_handle_s *h, const zc *x, size_t n, const char *what)
{
    int *d_cnt = (int *)dalloc(h, sizeof(int));
    HM_CUDA(cudaMemsetAsync(d_cnt, 0, sizeof(int), h->stream));
    unsigned g = (unsigned)std::min<size_t>((n + 255) / 256, 1024);
    k_nonfinite<<<std::max(g, 1u), 256, 0, h->stream>>>(x, n, d_cnt);
    HM_CHECK_LAUNCH();
    count_launch(h);
    int cnt = 0;
    HM_CUDA(cudaMemcpyAsync(&cnt, d_cnt, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    HM_CUDA(cudaStreamSynchronize(h->stream));
    dfree(h, d_cnt);
    if (cnt) throw HmError{HM_ERR_NUMERIC, std::string(what) + ": " + std::to_string(cnt) + " non-finite values"};
}

static std::vector<double> colnorm2(hm_handle_s *h, const zc *X, int nrhs, double *d_tmp)
{
    k_colnorm2<<<nrhs, 256, 0, h->stream>>>(X, h->N, d_tmp);
    HM_CHECK_LAUNCH();
    count_launch(h);
    std::vector<double> out(nrhs);
    HM_CUDA(cudaMemcpyAsync(out.data(), d_tmp, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, h->stream));
    HM_CUDA(cudaStreamSynchronize(h->stream));
    return out;
}

// FP64 iterative refinement preconditioned by the FP32 H-LU factor (tree order):
//   x_0 = 0, r_0 = b;  d = M^-1 r (FP32 H-solve);  x += d;  r = b - A x (FP64 H-matrix)
// until max_c |r_c| / |b_c| <= refine_tol.  Returns false when the step limit is hit.
static bool refine_solve(hm_handle_s *h, int nrhs, const zc *b, zc *x)
{
    const size_t n = (size_t)h->N * nrhs;
    zc *r = (zc *)dalloc(h, sizeof(zc) * n);
    cf *r32 = (cf *)dalloc(h, sizeof(cf) * n);
    zc *d = (zc *)dalloc(h, sizeof(zc) * n);
    double *d_nrm = (double *)dalloc(h, sizeof(double) * nrhs);
    HM_CUDA(cudaMemsetAsync(x, 0, sizeof(zc) * n, h->stream));
    HM_CUDA(cudaMemcpyAsync(r, b, sizeof(zc) * n, cudaMemcpyDeviceToDevice, h->stream));
    std::vector<double> bn = colnorm2(h, b, nrhs, d_nrm);
    bool ok = false;
    int it = 0;
    double worst = 1.0;
    for (it = 1; it <= h->prm.refine_max_iter; ++it) {
        convert_vec(h, r, r32, n);
        {
            PhaseScope ps(h, PH_SOLVE_SWEEP);
            tile_solve<cf>(h, h->tfac32, r32, nrhs);
        }
        convert_vec(h, r32, d, n);
        k_axpy1<<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(d, x, n);
        HM_CHECK_LAUNCH();
        count_launch(h);
        HM_CUDA(cudaMemcpyAsync(r, b, sizeof(zc) * n, cudaMemcpyDeviceToDevice, h->stream));
        {
            PhaseScope ps(h, PH_SOLVE_MATVEC);
            tile_matvec<zc>(h, h->tmat64, x, r, nrhs, zmake(-1, 0));
        }
        std::vector<double> rn = colnorm2(h, r, nrhs, d_nrm);
        worst = 0;
        bool finite = true;
        for (int c = 0; c < nrhs; ++c) {
            double q = bn[c] > 0 ? std::sqrt(rn[c] / bn[c]) : 0.0;
            finite = finite && std::isfinite(q) && std::isfinite(bn[c]);
            worst = std::max(worst, q);
        }
        if (!finite) {  // a NaN or an infinity: further steps cannot recover; the scan reports it
            worst = std::numeric_limits<double>::infinity();
            break;
        }
        if (worst <= h->prm.refine_tol) {
            ok = true;
            break;
        }
    }
    h->refine_iters = std::min(it, h->prm.refine_max_iter);
    h->refine_res = worst;
    dfree(h, r);
    dfree(h, r32);
    dfree(h, d);
    dfree(h, d_nrm);
    return ok;
}

static void solve_dev(hm_handle_s *h, int nrhs, const double *inc, const double *pol, zc *x_dev)
{
    if (h->state != 3) throw HmError{HM_ERR_STATE, "hm_solve requires hm_factor"};
    if (nrhs <= 0 || !inc || !pol || !x_dev) throw HmError{HM_ERR_ARG, "bad solve arguments"};
    std::vector<double> dirs(6 * (size_t)nrhs);
    for (int r = 0; r < nrhs; ++r)
        for (int d = 0; d < 3; ++d) {
            dirs[6 * r + d] = inc[3 * r + d];
            dirs[6 * r + 3 + d] = pol[3 * r + d];
        }
    phase_collect(h);
    h->phase_s[PH_SOLVE_SWEEP] = h->phase_s[PH_SOLVE_MATVEC] = 0;
    Timer t(h->stream);
    double *d_dirs = (double *)dalloc(h, sizeof(double) * dirs.size());
    HM_CUDA(cudaMemcpyAsync(d_dirs, dirs.data(), sizeof(double) * dirs.size(), cudaMemcpyHostToDevice, h->stream));
    zc *b = (zc *)dalloc(h, sizeof(zc) * (size_t)h->N * nrhs);
    if (h->dof == 4)
        launch_rhs_muller(h, nrhs, d_dirs, b);
    else
        launch_rhs(h, nrhs, d_dirs, b);
    if (h->fault == HM_FAULT_NAN_RHS) {  // host-side injection: one right-hand-side entry is NaN
        h->fault = HM_FAULT_NONE;
        const zc nan = zmake(std::numeric_limits<double>::quiet_NaN(), 0.0);
        HM_CUDA(cudaMemcpyAsync(b, &nan, sizeof(zc), cudaMemcpyHostToDevice, h->stream));
        HM_CUDA(cudaStreamSynchronize(h->stream));
    }
    bool converged = true;
    if (h->prm.precision == HM_FP32_REFINED) {
        zc *x = (zc *)dalloc(h, sizeof(zc) * (size_t)h->N * nrhs);
        converged = refine_solve(h, nrhs, b, x);
        launch_permute(h, nrhs, x, x_dev, h->d_iperm);
        dfree(h, x);
    } else {
        {
            PhaseScope ps(h, PH_SOLVE_SWEEP);
            tile_solve<zc>(h, h->tfac64, b, nrhs);
        }
        launch_permute(h, nrhs, b, x_dev, h->d_iperm);
        h->refine_iters = 0;
        h->refine_res = 0;
    }
    dfree(h, b);
    dfree(h, d_dirs);
    h->t_solve = t.stop();  // also keeps the host vector alive until the copy is done
    check_finite(h, x_dev, (size_t)h->N * nrhs, "hm_solve output");
    if (!converged)
        throw HmError{HM_ERR_NOT_CONVERGED, "iterative refinement did not reach refine_tol (residual " +
                                                std::to_string(h->refine_res) + ")"};
}

hm_status hm_solve(hm_handle h, int nrhs, const double *inc_dirs, const double *pols, void *x_dev)
{
    return guard(h, [&] { solve_dev(h, nrhs, inc_dirs, pols, (zc *)x_dev); });
}

hm_status hm_solve_host(hm_handle h, int nrhs, const double *inc_dirs, const double *pols, void *x_host)
{
    return guard(h, [&] {
        if (!x_host) throw HmError{HM_ERR_ARG, "null x_host"};
        zc *x = (zc *)dalloc(h, sizeof(zc) * (size_t)h->N * std::max(nrhs, 1));
        solve_dev(h, nrhs, inc_dirs, pols, x);
        HM_CUDA(cudaMemcpyAsync(x_host, x, sizeof(zc) * (size_t)h->N * nrhs, cudaMemcpyDeviceToHost, h->stream));
        dfree(h, x);
        HM_CUDA(cudaStreamSynchronize(h->stream));
    });
}

hm_status hm_farfield(hm_handle h, int nrhs, const void *x_dev, int nang, const double *obs, void *efar_dev,
                      double *rcs_host)
{
    return guard(h, [&] {
        if (h->state < 1) throw HmError{HM_ERR_STATE, "hm_farfield before hm_build_geometry"};
        if (nrhs <= 0 || nang <= 0 || !x_dev || !obs) throw HmError{HM_ERR_ARG, "bad farfield arguments"};
        double *d_obs = (double *)dalloc(h, sizeof(double) * 3 * nang);
        HM_CUDA(cudaMemcpyAsync(d_obs, obs, sizeof(double) * 3 * nang, cudaMemcpyHostToDevice, h->stream));
        double *d_rcs = rcs_host ? (double *)dalloc(h, sizeof(double) * (size_t)nrhs * nang) : nullptr;
        if (h->dof == 4)
            launch_farfield_muller(h, nrhs, (const zc *)x_dev, nang, d_obs, (zc *)efar_dev, d_rcs);
        else
            launch_farfield(h, nrhs, (const zc *)x_dev, nang, d_obs, (zc *)efar_dev, d_rcs);
        if (rcs_host)
            HM_CUDA(cudaMemcpyAsync(rcs_host, d_rcs, sizeof(double) * (size_t)nrhs * nang, cudaMemcpyDeviceToHost,
                                    h->stream));
        dfree(h, d_obs);
        if (d_rcs) dfree(h, d_rcs);
        HM_CUDA(cudaStreamSynchronize(h->stream));  // obs is only read during the call
    });
}

hm_status hm_matvec(hm_handle h, int nrhs, const void *x_dev, void *y_dev)
{
    return guard(h, [&] {
        TileOp<zc> **plan = nullptr;
        Block *A = nullptr;
        if (h->state == 2 || (h->state == 3 && h->prm.precision == HM_FP32_REFINED)) {
            A = h->root;
            plan = &h->tmat64;
        } else if (h->state == 3 && h->copy_root) {
            A = h->copy_root;
            plan = &h->tmatcopy;
        } else {
            throw HmError{HM_ERR_STATE, "hm_matvec needs a filled matrix (or keep_matrix before hm_factor)"};
        }
        if (nrhs <= 0 || !x_dev || !y_dev) throw HmError{HM_ERR_ARG, "bad matvec arguments"};
        if (!*plan) *plan = tile_build<zc>(h, A, false);
        size_t n = (size_t)h->N * nrhs;
        zc *xt = (zc *)dalloc(h, sizeof(zc) * n), *yt = (zc *)dalloc(h, sizeof(zc) * n);
        launch_permute(h, nrhs, (const zc *)x_dev, xt, h->d_perm);
        HM_CUDA(cudaMemsetAsync(yt, 0, sizeof(zc) * n, h->stream));
        tile_matvec<zc>(h, *plan, xt, yt, nrhs, zmake(1, 0));
        launch_permute(h, nrhs, yt, (zc *)y_dev, h->d_iperm);
        dfree(h, xt);
        dfree(h, yt);
    });
}

hm_status hm_query(hm_handle h, int what, double *out)
{
    return guard(h, [&] {
        if (!out) throw HmError{HM_ERR_ARG, "null out"};
        HM_CUDA(cudaStreamSynchronize(h->stream));
        double words;
        int maxk, nd, nl;
        double meank;
        storage(h, h->root, words, maxk, meank, nd, nl);
        switch (what) {
        case HM_Q_N: *out = h->N; break;
        case HM_Q_NNODE: *out = h->nnode; break;
        case HM_Q_NPATCH: *out = h->npatch; break;
        case HM_Q_NEAR_PAIRS: *out = (double)h->pair_q.size(); break;
        case HM_Q_DENSE_BLOCKS: *out = nd; break;
        case HM_Q_LR_BLOCKS: *out = nl; break;
        case HM_Q_CR: *out = h->N ? 1.0 - words / ((double)h->N * h->N) : 0.0; break;
        case HM_Q_MAX_RANK: *out = maxk; break;
        case HM_Q_T_GEOMETRY: *out = h->t_geom; break;
        case HM_Q_T_NEAR: *out = h->t_near; break;
        case HM_Q_T_DENSE: *out = h->t_dense; break;
        case HM_Q_T_ACA: *out = h->t_aca; break;
        case HM_Q_T_RECOMPRESS: *out = h->t_trunc; break;
        case HM_Q_T_FACTOR: *out = h->t_factor; break;
        case HM_Q_T_SOLVE: *out = h->t_solve; break;
        case HM_Q_FLOPS_FACTOR: *out = h->flops_factor; break;
        case HM_Q_STORAGE: *out = words; break;
        case HM_Q_ACA_NONCONV: *out = h->aca_nonconv; break;
        case HM_Q_LAUNCHES: *out = (double)h->launches; break;
        case HM_Q_NEAR_QPOINTS: *out = (double)h->near_points; break;
        case HM_Q_MEAN_RANK: *out = meank; break;
        case HM_Q_STORAGE_FACTOR: *out = words; break;
        case HM_Q_REFINE_ITERS: *out = h->refine_iters; break;
        case HM_Q_ACA_PREALLOC: *out = h->aca_prealloc; break;
        case HM_Q_ACA_RERUNS: *out = h->aca_reruns; break;
        case HM_Q_RANK_PRED_ERR: *out = h->rank_pred_err; break;
        case HM_Q_TRUNC_BATCHES: *out = h->tr_batches; break;
        case HM_Q_TRUNC_JOBS: *out = h->tr_jobs; break;
        case HM_Q_TRUNC_MAXK: *out = h->tr_maxk; break;
        case HM_Q_TRUNC_WORK: *out = h->tr_work; break;
        case HM_Q_T_TRUNC: *out = h->tr_seconds; break;
        case HM_Q_ACA_SKIPPED: *out = h->aca_skipped; break;
        case HM_Q_KQR_SECONDS: *out = h->kqr_s; break;
        case HM_Q_KQR_FLOPS: *out = h->kqr_flops; break;
        case HM_Q_KQR_LAUNCHES: *out = h->kqr_n; break;
        case HM_Q_KCORE_SECONDS: *out = h->kcore_s; break;
        case HM_Q_KCORE_FLOPS: *out = h->kcore_flops; break;
        case HM_Q_KCORE_LAUNCHES: *out = h->kcore_n; break;
        case HM_Q_REFINE_RES: *out = h->refine_res; break;
        case HM_Q_DENSE_LEVEL: *out = h->dense_lev; break;
        case HM_Q_KGEMM_SECONDS: gemm_timing_collect(h); *out = h->kgemm_s; break;
        case HM_Q_KGEMM_FLOPS: gemm_timing_collect(h); *out = h->kgemm_flops; break;
        case HM_Q_KGEMM_LAUNCHES: gemm_timing_collect(h); *out = h->kgemm_n; break;
        case HM_Q_KTC_SECONDS: gemm_timing_collect(h); *out = h->ktc_s; break;
        case HM_Q_KTC_FLOPS: gemm_timing_collect(h); *out = h->ktc_flops; break;
        case HM_Q_KTC_LAUNCHES: gemm_timing_collect(h); *out = h->ktc_n; break;
        case HM_Q_T_LU_PANEL: phase_collect(h); *out = h->phase_s[PH_LU_PANEL]; break;
        case HM_Q_T_LU_U12: phase_collect(h); *out = h->phase_s[PH_LU_U12]; break;
        case HM_Q_T_TILE_BUILD: phase_collect(h); *out = h->phase_s[PH_TILE_BUILD]; break;
        case HM_Q_T_SOLVE_SWEEP: phase_collect(h); *out = h->phase_s[PH_SOLVE_SWEEP]; break;
        case HM_Q_T_SOLVE_MATVEC: phase_collect(h); *out = h->phase_s[PH_SOLVE_MATVEC]; break;
        case HM_Q_STORAGE32: {
            // the blocks reachable from the factor's root (a coarsened tree detaches the
            // blocks it merged)
            double w32 = 0;
            std::vector<Block32 *> st;
            if (h->root32) st.push_back(h->root32);
            while (!st.empty()) {
                Block32 *b = st.back();
                st.pop_back();
                if (b->type == B_HIER)
                    for (int i = 0; i < 4; ++i) st.push_back(b->ch[i]);
                else if (b->type == B_DENSE)
                    w32 += (double)b->nr * b->nc;
                else
                    w32 += (double)b->k * (b->nr + b->nc);
            }
            *out = w32;
            break;
        }
        default: throw HmError{HM_ERR_ARG, "unknown query key"};
        }
    });
}

const char *hm_last_error(hm_handle h) { return h ? h->err.c_str() : "null handle"; }

hm_status hm_get_trunc_log_host(hm_handle h, int *nbatches, double *out)
{
    return guard(h, [&] {
        if (!nbatches) throw HmError{HM_ERR_ARG, "null count"};
        *nbatches = (int)(h->trunc_log.size() / 7);
        if (out) std::copy(h->trunc_log.begin(), h->trunc_log.end(), out);
    });
}

hm_status hm_cgemm(hm_handle h, char opA, char opB, int m, int n, int k, const float *alpha, const void *A, int lda,
                   const void *B, int ldb, const float *beta, void *C, int ldc, int path)
{
    return guard(h, [&] {
        if ((opA != 'N' && opA != 'C') || (opB != 'N' && opB != 'C') || !alpha || !beta)
            throw HmError{HM_ERR_ARG, "hm_cgemm: op must be 'N' or 'C'; alpha, beta non-null"};
        if (m < 0 || n < 0 || k < 0 || path < 0 || path > 5) throw HmError{HM_ERR_ARG, "hm_cgemm: bad size or path"};
        if (m == 0 || n == 0) return;
        const int rowsA = opA == 'N' ? m : k, rowsB = opB == 'N' ? k : n;
        if (!C || ldc < std::max(1, m) || (k > 0 && (!A || !B || lda < std::max(1, rowsA) || ldb < std::max(1, rowsB))))
            throw HmError{HM_ERR_ARG, "hm_cgemm: null pointer or leading dimension too small"};
        if (path >= 2 && (m < 64 || n < 64 || k < 16))
            throw HmError{HM_ERR_ARG, "hm_cgemm: the tensor-core path needs m, n >= 64 and k >= 16"};
        const cf al = cmk<cf>(alpha[0], alpha[1]), be = cmk<cf>(beta[0], beta[1]);
        const int saved = h->prm.simt_gemm;
        try {
            if (path >= 2) {
                static const int variant[4] = {0, 2, 4, 1};  // path 2: autotuned; 3, 4, 5: forced
                tc_gemm(h, opA, opB, m, n, k, al, (const cf *)A, lda, (const cf *)B, ldb, be, (cf *)C, ldc,
                        variant[path - 2]);
            } else {
                if (path == 1) h->prm.simt_gemm = 1;
                zgemm<cf>(h, opA, opB, m, n, k, al, (const cf *)A, lda, (const cf *)B, ldb, be, (cf *)C, ldc);
            }
        } catch (...) {
            h->prm.simt_gemm = saved;
            throw;
        }
        h->prm.simt_gemm = saved;
        HM_CUDA(cudaStreamSynchronize(h->stream));
        tc_check(h);
    });
}

hm_status hm_tc_tuning(int *stages, float *ms)
{
    if (!stages || !ms) return HM_ERR_ARG;
    tc_tune_record(stages, ms);
    return HM_OK;
}

hm_status hm_inject_fault(hm_handle h, int what)
{
    return guard(h, [&] {
        if (what < HM_FAULT_NONE || what > HM_FAULT_ALLOC) throw HmError{HM_ERR_ARG, "unknown fault"};
        h->fault = what;
    });
}

hm_status hm_rank_samples(hm_handle h, int *n, float *feat_host, float *target_host)
{
    return guard(h, [&] {
        if (!n) throw HmError{HM_ERR_ARG, "null count"};
        if (h->state < 2) throw HmError{HM_ERR_STATE, "rank samples exist after hm_fill"};
        *n = (int)h->rank_target.size();
        if (feat_host) std::copy(h->rank_feat.begin(), h->rank_feat.end(), feat_host);
        if (target_host) std::copy(h->rank_target.begin(), h->rank_target.end(), target_host);
    });
}

hm_status hm_set_rank_model(hm_handle h, hm_mlp m)
{
    return guard(h, [&] {
        if (m && mlp_nin(m) != HM_RANK_NFEAT) throw HmError{HM_ERR_ARG, "rank model must have 8 inputs"};
        h->rank_model = m;
    });
}

void hm_destroy(hm_handle h)
{
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    try {
        free_all(h);
    } catch (...) {
    }
    cudaStreamSynchronize(h->stream);
    if (h->d_counter) cudaFree(h->d_counter);
    for (cudaEvent_t e : h->ev)
        if (e) cudaEventDestroy(e);
    for (const GemmTiming &t : h->gemm_pending) {
        cudaEventDestroy(t.e0);
        cudaEventDestroy(t.e1);
    }
    for (const PhaseMark &m : h->phase_pending) {
        cudaEventDestroy(m.e0);
        cudaEventDestroy(m.e1);
    }
    for (cudaEvent_t e : h->gemm_free) cudaEventDestroy(e);
    if (h->d_tc_err) cudaFree(h->d_tc_err);
    for (cudaStream_t ps : h->pool) cudaStreamDestroy(ps);
    for (cudaEvent_t pe : h->pool_ev) cudaEventDestroy(pe);
    delete h;
}

hm_status hm_get_nodes_host(hm_handle h, double *out)
{
    return guard(h, [&] {
        if (h->state < 1 || !out) throw HmError{HM_ERR_STATE, "no geometry"};
        for (int i = 0; i < h->nnode; ++i)
            for (int c = 0; c < 14; ++c) out[14 * (size_t)i + c] = h->h_nodes[(size_t)c * h->nnode + i];
    });
}

hm_status hm_get_near_pairs_host(hm_handle h, int *out)
{
    return guard(h, [&] {
        if (h->state < 1 || !out) throw HmError{HM_ERR_STATE, "no geometry"};
        for (size_t i = 0; i < h->pair_q.size(); ++i) {
            out[2 * i] = h->pair_q[i];
            out[2 * i + 1] = h->pair_p[i];
        }
    });
}

hm_status hm_get_near_block_host(hm_handle h, int tn, int p, void *out)
{
    return guard(h, [&] {
        if (h->state < 2 || !out) throw HmError{HM_ERR_STATE, "near store not filled"};
        const int D = h->dof, nc2 = h->nc * h->nc, w = D * nc2;
        if (tn < 0 || tn >= h->nnode || p < 0 || p >= h->npatch) throw HmError{HM_ERR_ARG, "index out of range"};
        int q = tn / nc2, idx = -1;
        for (size_t i = 0; i < h->pair_q.size(); ++i)
            if (h->pair_q[i] == q && h->pair_p[i] == p) idx = (int)i;
        if (idx < 0) throw HmError{HM_ERR_ARG, "not a near pair"};
        std::vector<zc> rows(D * (size_t)w);
        HM_CUDA(cudaMemcpyAsync(rows.data(), h->d_near + ((size_t)idx * w + D * (tn - q * nc2)) * w,
                                sizeof(zc) * D * w, cudaMemcpyDeviceToHost, h->stream));
        HM_CUDA(cudaStreamSynchronize(h->stream));
        zc *o = (zc *)out;
        for (int b = 0; b < D; ++b)
            for (int a = 0; a < D; ++a)
                for (int j = 0; j < nc2; ++j) o[(D * b + a) * nc2 + j] = rows[(size_t)b * w + D * j + a];
    });
}

hm_status hm_entries_host(hm_handle h, int n, const int *rows, const int *cols, void *out)
{
    return guard(h, [&] {
        if (h->state < 2) throw HmError{HM_ERR_STATE, "matrix not filled"};
        if (n <= 0) return;
        if (!rows || !cols || !out) throw HmError{HM_ERR_ARG, "null pointer"};
        for (int i = 0; i < n; ++i)
            if (rows[i] < 0 || rows[i] >= h->N || cols[i] < 0 || cols[i] >= h->N) throw HmError{HM_ERR_ARG, "index out of range"};
        int *d_rc = (int *)dalloc(h, sizeof(int) * 2 * n);
        zc *d_o = (zc *)dalloc(h, sizeof(zc) * n);
        HM_CUDA(cudaMemcpyAsync(d_rc, rows, sizeof(int) * n, cudaMemcpyHostToDevice, h->stream));
        HM_CUDA(cudaMemcpyAsync(d_rc + n, cols, sizeof(int) * n, cudaMemcpyHostToDevice, h->stream));
        launch_entries(h, n, d_rc, d_rc + n, d_o);
        HM_CUDA(cudaMemcpyAsync(out, d_o, sizeof(zc) * n, cudaMemcpyDeviceToHost, h->stream));
        HM_CUDA(cudaStreamSynchronize(h->stream));
        dfree(h, d_rc);
        dfree(h, d_o);
    });
}

hm_status hm_get_perm_host(hm_handle h, int *perm)
{
    return guard(h, [&] {
        if (h->state < 1 || !perm) throw HmError{HM_ERR_STATE, "no geometry"};
        HM_CUDA(cudaMemcpyAsync(perm, h->d_perm, sizeof(int) * h->N, cudaMemcpyDeviceToHost, h->stream));
        HM_CUDA(cudaStreamSynchronize(h->stream));
    });
}

hm_status hm_get_blocks_host(hm_handle h, int *nblocks, int *out)
{
    return guard(h, [&] {
        if (h->state < 1 || !nblocks) throw HmError{HM_ERR_STATE, "no geometry"};
        *nblocks = (int)h->leaves.size();
        if (!out) return;
        for (size_t i = 0; i < h->leaves.size(); ++i) {
            Block *b = h->leaves[i];
            int *o = out + 6 * i;
            o[0] = b->type == B_DENSE ? 0 : 1;
            o[1] = b->r0;
            o[2] = b->nr;
            o[3] = b->c0;
            o[4] = b->nc;
            o[5] = b->type == B_LR ? b->k : 0;
        }
    });
}

hm_status hm_get_block_dense_host(hm_handle h, int bi, void *out)
{
    return guard(h, [&] {
        if (h->state != 2) throw HmError{HM_ERR_STATE, "blocks are inspectable between hm_fill and hm_factor"};
        if (bi < 0 || bi >= (int)h->leaves.size() || !out) throw HmError{HM_ERR_ARG, "bad block index"};
        Block *b = h->leaves[bi];
        size_t n = (size_t)b->nr * b->nc;
        zc *d = (zc *)dalloc(h, sizeof(zc) * n);
        if (b->type == B_DENSE)
            HM_CUDA(cudaMemcpyAsync(d, b->D, sizeof(zc) * n, cudaMemcpyDeviceToDevice, h->stream));
        else
            zgemm(h, 'N', 'C', b->nr, b->nc, b->k, zmake(1, 0), b->U, b->nr, b->V, b->nc, zmake(0, 0), d, b->nr);
        HM_CUDA(cudaMemcpyAsync(out, d, sizeof(zc) * n, cudaMemcpyDeviceToHost, h->stream));
        HM_CUDA(cudaStreamSynchronize(h->stream));
        dfree(h, d);
    });
}

}  // extern "C"
