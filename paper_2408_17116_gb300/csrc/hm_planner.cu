// Host planner: quadrature rules, node geometry launch, near patch pairs, cluster
// tree and block cluster tree (Sec. III: recursive geometric partition, bounding
// boxes, admissibility of Eq. 21, leaf size n_leaf; Sec. III.B: the u and v
// unknowns of a node stay together, interleaved).
#include <algorithm>
#include <cmath>
#include <numeric>

#include "hm_internal.h"

static const double PI = 3.14159265358979323846;

void cheb_nodes_host(int n, double *x)
{
    for (int l = 0; l < n; ++l) x[l] = std::cos(PI * (2 * l + 1) / (2.0 * n));
}

// Fejer's first rule as the integrals of the Chebyshev cardinal functions
// (Eq. 13 in Eq. 12): w_l = sum_{n even} (alpha_n / N) T_n(x_l) * 2 / (1 - n^2).
void fejer_weights_host(int n, double *w)
{
    for (int l = 0; l < n; ++l) {
        double th = PI * (2 * l + 1) / (2.0 * n);
        double s = 2.0 / n;  // n = 0 term: alpha_0 = 1, integral of T_0 = 2
        for (int j = 2; j < n; j += 2) s += (2.0 / n) * std::cos(j * th) * 2.0 / (1.0 - (double)j * j);
        w[l] = s;
    }
}

// Gauss-Legendre on [-1, 1]: Newton iteration on P_q from Tricomi-type initial guesses.
void gauss_legendre_host(int q, double *x, double *w)
{
    for (int i = 0; i < q; ++i) {
        double t = PI * (4 * i + 3) / (4.0 * q + 2);
        double z = std::cos(t + 1.0 / (8.0 * q * q * std::tan(t)));
        double pd = 1.0;
        for (int it = 0; it < 60; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= q; ++k) {
                double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            if (q == 1) p0 = 1.0, p1 = z;
            pd = q * (p0 - z * p1) / (1.0 - z * z);
            double dz = p1 / pd;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= q; ++k) {
            double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        if (q == 1) p0 = 1.0, p1 = z;
        pd = q * (p0 - z * p1) / (1.0 - z * z);
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * pd * pd);
    }
}

static double bbox_dist(const double *amin, const double *amax, const double *bmin, const double *bmax)
{
    double s = 0;
    for (int d = 0; d < 3; ++d) {
        double g = std::max(0.0, std::max(amin[d] - bmax[d], bmin[d] - amax[d]));
        s += g * g;
    }
    return std::sqrt(s);
}
static double bbox_diam(const double *mn, const double *mx)
{
    double s = 0;
    for (int d = 0; d < 3; ++d) s += (mx[d] - mn[d]) * (mx[d] - mn[d]);
    return std::sqrt(s);
}

static void build_clusters(hm_handle_s *h, int off, int cnt, int level, int depth, int &idx_out)
{
    Cluster c;
    c.off = off;
    c.cnt = cnt;
    c.level = level;
    c.child[0] = c.child[1] = -1;
    const double *X = h->h_nodes.data();
    int n = h->nnode;
    for (int d = 0; d < 3; ++d) {
        c.bmin[d] = 1e300;
        c.bmax[d] = -1e300;
    }
    for (int i = off; i < off + cnt; ++i) {
        int nd = h->perm_node[i];
        for (int d = 0; d < 3; ++d) {
            c.bmin[d] = std::min(c.bmin[d], X[d * n + nd]);
            c.bmax[d] = std::max(c.bmax[d], X[d * n + nd]);
        }
    }
    const bool indep = h->prm.independent && !h->node_body.empty();
    if (indep) {
        c.b0 = h->node_body[h->perm_node[off]];
        c.b1 = h->node_body[h->perm_node[off + cnt - 1]];
    }
    int me = (int)h->clusters.size();
    h->clusters.push_back(c);
    idx_out = me;
    if (indep && c.b0 != c.b1) {
        // several bodies (contiguous in tree order): split at the body boundary nearest the
        // middle, so that every cluster below holds one body
        int best = -1;
        for (int i = off + 1; i < off + cnt; ++i)
            if (h->node_body[h->perm_node[i]] != h->node_body[h->perm_node[i - 1]] &&
                (best < 0 || std::abs(2 * (i - off) - cnt) < std::abs(2 * (best - off) - cnt)))
                best = i;
        int c0, c1;
        build_clusters(h, off, best - off, level + 1, depth, c0);
        build_clusters(h, best, off + cnt - best, level + 1, depth, c1);
        h->clusters[me].child[0] = c0;
        h->clusters[me].child[1] = c1;
        h->clusters[c0].body_root = h->clusters[c0].b0 == h->clusters[c0].b1;
        h->clusters[c1].body_root = h->clusters[c1].b0 == h->clusters[c1].b1;
        return;
    }
    // one body: geometric bisection; independent bodies stop at n_leaf unknowns per cluster,
    // otherwise at the common leaf depth
    if (indep ? (h->dof * cnt <= h->prm.leaf || cnt < 2) : (level >= depth || cnt < 2)) return;
    int ax = 0;
    double ext = -1;
    for (int d = 0; d < 3; ++d)
        if (c.bmax[d] - c.bmin[d] > ext) {
            ext = c.bmax[d] - c.bmin[d];
            ax = d;
        }
    auto beg = h->perm_node.begin() + off, end = beg + cnt;
    std::sort(beg, end, [&](int a, int b) {
        double xa = X[ax * n + a], xb = X[ax * n + b];
        return xa < xb || (xa == xb && a < b);
    });
    int half = cnt / 2;
    int c0, c1;
    build_clusters(h, off, half, level + 1, depth, c0);
    build_clusters(h, off + half, cnt - half, level + 1, depth, c1);
    h->clusters[me].child[0] = c0;
    h->clusters[me].child[1] = c1;
}

static Block *build_blocks(hm_handle_s *h, int t, int s)
{
    const Cluster &ct = h->clusters[t], &cs = h->clusters[s];
    Block *b = new Block();
    h->blocks.push_back(b);
    b->t = t;
    b->s = s;
    b->r0 = h->dof * ct.off;
    b->nr = h->dof * ct.cnt;
    b->c0 = h->dof * cs.off;
    b->nc = h->dof * cs.cnt;
    if (h->prm.independent && (ct.b1 < cs.b0 || cs.b1 < ct.b0)) {
        // independent bodies: no body in common, an identically zero block
        b->type = B_LR;
        b->zero = true;
        b->k = 0;
        b->leaf_id = (int)h->leaves.size();
        h->leaves.push_back(b);
        return b;
    }
    double dist = bbox_dist(ct.bmin, ct.bmax, cs.bmin, cs.bmax);
    double dm = std::min(bbox_diam(ct.bmin, ct.bmax), bbox_diam(cs.bmin, cs.bmax));
    bool adm = dist > 0.0 && dm <= h->prm.eta * dist;
    if (adm) {
        b->type = B_LR;
        b->leaf_id = (int)h->leaves.size();
        h->leaves.push_back(b);
    } else if (ct.child[0] < 0 || cs.child[0] < 0) {
        b->type = B_DENSE;
        b->leaf_id = (int)h->leaves.size();
        h->leaves.push_back(b);
    } else {
        b->type = B_HIER;
        b->ch[0] = build_blocks(h, ct.child[0], cs.child[0]);
        b->ch[1] = build_blocks(h, ct.child[0], cs.child[1]);
        b->ch[2] = build_blocks(h, ct.child[1], cs.child[0]);
        b->ch[3] = build_blocks(h, ct.child[1], cs.child[1]);
    }
    return b;
}

void plan_geometry(hm_handle_s *h)
{
    const int nc = h->nc, nc2 = nc * nc, P = h->npatch;
    // bodies and patches to the device
    h->d_bodies = (DevBody *)dalloc(h, sizeof(DevBody) * h->bodies.size());
    h->d_patches = (DevPatch *)dalloc(h, sizeof(DevPatch) * h->patches.size());
    HM_CUDA(cudaMemcpyAsync(h->d_bodies, h->bodies.data(), sizeof(DevBody) * h->bodies.size(), cudaMemcpyHostToDevice,
                            h->stream));
    HM_CUDA(cudaMemcpyAsync(h->d_patches, h->patches.data(), sizeof(DevPatch) * h->patches.size(),
                            cudaMemcpyHostToDevice, h->stream));
    // node geometry (A1)
    std::vector<double> x1d(nc), w1d(nc);
    cheb_nodes_host(nc, x1d.data());
    fejer_weights_host(nc, w1d.data());
    double *d_1d = (double *)dalloc(h, sizeof(double) * 2 * nc);
    HM_CUDA(cudaMemcpyAsync(d_1d, x1d.data(), sizeof(double) * nc, cudaMemcpyHostToDevice, h->stream));
    HM_CUDA(cudaMemcpyAsync(d_1d + nc, w1d.data(), sizeof(double) * nc, cudaMemcpyHostToDevice, h->stream));
    h->d_nodes = (double *)dalloc(h, sizeof(double) * 14 * (size_t)h->nnode);
    launch_nodes(h, d_1d, d_1d + nc);
    h->h_nodes.resize(14 * (size_t)h->nnode);
    HM_CUDA(cudaMemcpyAsync(h->h_nodes.data(), h->d_nodes, sizeof(double) * 14 * (size_t)h->nnode,
                            cudaMemcpyDeviceToHost, h->stream));
    // patch boxes over the grid {-1, nodes, +1}^2
    int ng = nc + 2;
    std::vector<double> g(ng);
    g[0] = -1.0;
    for (int l = 0; l < nc; ++l) g[l + 1] = x1d[l];
    g[ng - 1] = 1.0;
    double *d_g = (double *)dalloc(h, sizeof(double) * ng);
    double *d_pts = (double *)dalloc(h, sizeof(double) * 3 * (size_t)P * ng * ng);
    HM_CUDA(cudaMemcpyAsync(d_g, g.data(), sizeof(double) * ng, cudaMemcpyHostToDevice, h->stream));
    launch_patch_grid(h, d_g, ng, d_pts);
    std::vector<double> pts(3 * (size_t)P * ng * ng);
    HM_CUDA(cudaMemcpyAsync(pts.data(), d_pts, sizeof(double) * pts.size(), cudaMemcpyDeviceToHost, h->stream));
    HM_CUDA(cudaStreamSynchronize(h->stream));
    dfree(h, d_1d);
    dfree(h, d_g);
    dfree(h, d_pts);
    std::vector<double> bmin(3 * P, 1e300), bmax(3 * P, -1e300), diam(P);
    for (int p = 0; p < P; ++p) {
        for (int i = 0; i < ng * ng; ++i)
            for (int d = 0; d < 3; ++d) {
                double v = pts[3 * ((size_t)p * ng * ng + i) + d];
                bmin[3 * p + d] = std::min(bmin[3 * p + d], v);
                bmax[3 * p + d] = std::max(bmax[3 * p + d], v);
            }
        diam[p] = bbox_diam(&bmin[3 * p], &bmax[3 * p]);
    }
    // near patch pairs (Eq. 20 self/near split)
    h->pair_q.clear();
    h->pair_p.clear();
    std::vector<int> nearidx((size_t)P * P, -1);
    for (int q = 0; q < P; ++q)
        for (int p = 0; p < P; ++p) {
            bool nr = (q == p) || bbox_dist(&bmin[3 * q], &bmax[3 * q], &bmin[3 * p], &bmax[3 * p]) <
                                      h->prm.near_delta * std::max(diam[q], diam[p]);
            if (h->prm.independent && h->patches[q].body != h->patches[p].body) nr = false;
            if (nr) {
                nearidx[(size_t)q * P + p] = (int)h->pair_q.size();
                h->pair_q.push_back(q);
                h->pair_p.push_back(p);
            }
        }
    int npairs = (int)h->pair_q.size();
    h->d_nearidx = (int *)dalloc(h, sizeof(int) * (size_t)P * P);
    h->d_pair_q = (int *)dalloc(h, sizeof(int) * npairs);
    h->d_pair_p = (int *)dalloc(h, sizeof(int) * npairs);
    HM_CUDA(cudaMemcpyAsync(h->d_nearidx, nearidx.data(), sizeof(int) * nearidx.size(), cudaMemcpyHostToDevice, h->stream));
    HM_CUDA(cudaMemcpyAsync(h->d_pair_q, h->pair_q.data(), sizeof(int) * npairs, cudaMemcpyHostToDevice, h->stream));
    HM_CUDA(cudaMemcpyAsync(h->d_pair_p, h->pair_p.data(), sizeof(int) * npairs, cudaMemcpyHostToDevice, h->stream));
    h->node_body.clear();
    if (h->prm.independent) {
        h->node_body.resize(h->nnode);
        for (int nd = 0; nd < h->nnode; ++nd) h->node_body[nd] = h->patches[nd / nc2].body;
        std::vector<int> pb(P);
        for (int p = 0; p < P; ++p) pb[p] = h->patches[p].body;
        h->d_patch_body = (int *)dalloc(h, sizeof(int) * P);
        HM_CUDA(cudaMemcpyAsync(h->d_patch_body, pb.data(), sizeof(int) * P, cudaMemcpyHostToDevice, h->stream));
        HM_CUDA(cudaStreamSynchronize(h->stream));  // pb is a host temporary
    }
    build_cluster_tree(h);
    std::vector<int> perm(h->N), iperm(h->N);
    for (int pos = 0; pos < h->nnode; ++pos)
        for (int c = 0; c < h->dof; ++c) {
            perm[h->dof * pos + c] = h->dof * h->perm_node[pos] + c;
            iperm[h->dof * h->perm_node[pos] + c] = h->dof * pos + c;
        }
    h->d_perm = (int *)dalloc(h, sizeof(int) * h->N);
    h->d_iperm = (int *)dalloc(h, sizeof(int) * h->N);
    HM_CUDA(cudaMemcpyAsync(h->d_perm, perm.data(), sizeof(int) * h->N, cudaMemcpyHostToDevice, h->stream));
    HM_CUDA(cudaMemcpyAsync(h->d_iperm, iperm.data(), sizeof(int) * h->N, cudaMemcpyHostToDevice, h->stream));
    // block cluster tree
    rebuild_block_tree(h);
    HM_CUDA(cudaStreamSynchronize(h->stream));
}

// Cluster tree over the host node table: balanced median bisection along the widest
// bounding-box axis to a common leaf depth (the first depth whose clusters hold at
// most n_leaf unknowns, dof per node).
void build_cluster_tree(hm_handle_s *h)
{
    int depth = 0;
    while (h->dof * ((h->nnode + (1 << depth) - 1) >> depth) > h->prm.leaf && (1 << depth) < h->nnode) ++depth;
    h->perm_node.resize(h->nnode);
    std::iota(h->perm_node.begin(), h->perm_node.end(), 0);
    h->clusters.clear();
    int root;
    build_clusters(h, 0, h->nnode, 0, depth, root);
    h->clusters[root].body_root = h->prm.independent && h->clusters[root].b0 == h->clusters[root].b1;
}

static hm_status plan_host(const double *xyz, const int *node_body, int nnode, int dof, int leaf, double eta,
                           int *nblocks, int *blocks, int *perm_node)
{
    if (!xyz || nnode <= 0 || (dof != 2 && dof != 4) || leaf < dof || !(eta > 0.0) || !nblocks) return HM_ERR_ARG;
    if (node_body)
        for (int i = 1; i < nnode; ++i)
            if (node_body[i] < node_body[i - 1] || node_body[0] < 0) return HM_ERR_ARG;
    try {
        hm_handle_s h;  // host-only planning: no stream, no device memory
        h.nnode = nnode;
        h.dof = dof;
        h.N = dof * nnode;
        h.prm.leaf = leaf;
        h.prm.eta = eta;
        h.prm.independent = node_body ? 1 : 0;
        if (node_body) h.node_body.assign(node_body, node_body + nnode);
        h.h_nodes.assign(14 * (size_t)nnode, 0.0);
        for (int i = 0; i < nnode; ++i)
            for (int d = 0; d < 3; ++d) h.h_nodes[(size_t)d * nnode + i] = xyz[3 * (size_t)i + d];
        build_cluster_tree(&h);
        rebuild_block_tree(&h);
        *nblocks = (int)h.leaves.size();
        if (blocks)
            for (size_t i = 0; i < h.leaves.size(); ++i) {
                const Block *b = h.leaves[i];
                int *o = blocks + 5 * i;
                o[0] = b->type == B_DENSE ? 0 : (b->zero ? 2 : 1);
                o[1] = b->r0;
                o[2] = b->nr;
                o[3] = b->c0;
                o[4] = b->nc;
            }
        if (perm_node) std::copy(h.perm_node.begin(), h.perm_node.end(), perm_node);
        for (Block *b : h.blocks) delete b;
        h.blocks.clear();
        return HM_OK;
    } catch (...) {
        return HM_ERR_OOM;
    }
}

extern "C" hm_status hm_plan_host(const double *xyz, int nnode, int dof, int leaf, double eta, int *nblocks,
                                  int *blocks, int *perm_node)
{
    return plan_host(xyz, nullptr, nnode, dof, leaf, eta, nblocks, blocks, perm_node);
}

extern "C" hm_status hm_plan_bodies_host(const double *xyz, const int *node_body, int nnode, int dof, int leaf,
                                         double eta, int *nblocks, int *blocks, int *perm_node)
{
    if (!node_body) return HM_ERR_ARG;
    return plan_host(xyz, node_body, nnode, dof, leaf, eta, nblocks, blocks, perm_node);
}

void rebuild_block_tree(hm_handle_s *h)
{
    for (Block *b : h->blocks) delete b;
    h->blocks.clear();
    h->leaves.clear();
    h->root = build_blocks(h, 0, 0);
}
