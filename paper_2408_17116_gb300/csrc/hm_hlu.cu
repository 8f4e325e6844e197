// H-LU factorisation and H-solve (Sec. III and III.A: block LU of Eq. 23 applied
// recursively, forward substitution Eqs. 24, 26, 27, back substitution Eqs. 25,
// 28), on the "entire matrix" block cluster tree (Sec. III.B).
//
// Recursion on a diagonal block A = [[A11, A12], [A21, A22]]:
//   A11 = P1^T L11 U11                       (recursive; partial pivoting inside dense leaves)
//   U12 = L11^-1 P1 A12,  L21 = A21 U11^-1   (H-triangular solves)
//   S   = A22 - L21 U12                      (formatted multiply-add with truncation)
//   S   = P2^T L22 U22                       (recursive)
// so that A x = b is solved by y1 = L11^-1 P1 b1, y2 = L22^-1 P2 (b2 - L21 y1),
// x2 = U22^-1 y2, x1 = U11^-1 (y1 - U12 x2).  Low-rank blocks are U V^H; every
// low-rank sum is recompressed (QR + SVD) to the ACA tolerance.
#include <algorithm>

#include "hm_internal.h"

static const zc ONE = {1.0, 0.0};
static const zc ZERO = {0.0, 0.0};
static const zc MONE = {-1.0, 0.0};

static inline MV rows_of(MV X, int r0, int nr) { return MV{X.p + r0, nr, X.cols, X.ld}; }
void flush(hm_handle_s *h, Block *b);

static zc *zalloc(hm_handle_s *h, size_t n) { return (zc *)dalloc(h, sizeof(zc) * std::max<size_t>(n, 1)); }

static void zzero(hm_handle_s *h, MV X)
{
    if (X.rows <= 0 || X.cols <= 0) return;
    if (X.ld == X.rows) {
        HM_CUDA(cudaMemsetAsync(X.p, 0, sizeof(zc) * (size_t)X.rows * X.cols, h->stream));
    } else {
        for (int j = 0; j < X.cols; ++j)
            HM_CUDA(cudaMemsetAsync(X.p + (size_t)j * X.ld, 0, sizeof(zc) * X.rows, h->stream));
    }
}

// Y += alpha op(A) X,  op = N (X rows = A.nc) or C (X rows = A.nr)
void hmatvec(hm_handle_s *h, Block *A, MV X, MV Y, zc alpha, bool ct)
{
    if (X.cols <= 0) return;
    if (A->pend_k) flush(h, A);
    switch (A->type) {
    case B_DENSE:
        if (!ct)
            zgemm(h, 'N', 'N', A->nr, X.cols, A->nc, alpha, A->D, A->nr, X.p, X.ld, ONE, Y.p, Y.ld);
        else
            zgemm(h, 'C', 'N', A->nc, X.cols, A->nr, alpha, A->D, A->nr, X.p, X.ld, ONE, Y.p, Y.ld);
        break;
    case B_LR: {
        if (A->k == 0) return;
        zc *t = zalloc(h, (size_t)A->k * X.cols);
        if (!ct) {
            zgemm(h, 'C', 'N', A->k, X.cols, A->nc, ONE, A->V, A->nc, X.p, X.ld, ZERO, t, A->k);
            zgemm(h, 'N', 'N', A->nr, X.cols, A->k, alpha, A->U, A->nr, t, A->k, ONE, Y.p, Y.ld);
        } else {
            zgemm(h, 'C', 'N', A->k, X.cols, A->nr, ONE, A->U, A->nr, X.p, X.ld, ZERO, t, A->k);
            zgemm(h, 'N', 'N', A->nc, X.cols, A->k, alpha, A->V, A->nc, t, A->k, ONE, Y.p, Y.ld);
        }
        dfree(h, t);
        break;
    }
    case B_HIER:
        for (int c = 0; c < 4; ++c) {
            Block *b = A->ch[c];
            int ro = b->r0 - A->r0, co = b->c0 - A->c0;
            if (!ct)
                hmatvec(h, b, rows_of(X, co, b->nc), rows_of(Y, ro, b->nr), alpha, false);
            else
                hmatvec(h, b, rows_of(X, ro, b->nr), rows_of(Y, co, b->nc), alpha, true);
        }
        break;
    }
}


static void collect_pending(Block *b, std::vector<Block *> &out)
{
    if (b->type == B_HIER) {
        for (int i = 0; i < 4; ++i) collect_pending(b->ch[i], out);
    } else if (b->type == B_LR && b->pend_k > 0) {
        out.push_back(b);
    }
}

// Recompress, in one batch, every low-rank block of b's subtree that has pending
// updates: [U | Up_1 | ...] [V | Vp_1 | ...]^H -> truncated U' V'^H.
void flush(hm_handle_s *h, Block *b)
{
    std::vector<Block *> list;
    collect_pending(b, list);
    if (list.empty()) return;
    std::vector<int> ranks;
    for (Block *c : list) {
        int K = c->k + c->pend_k;
        zc *Us = zalloc(h, (size_t)c->nr * K), *Vs = zalloc(h, (size_t)c->nc * K);
        int off = 0;
        if (c->k) {
            zcopy2d(h, MV{Us, c->nr, c->k, c->nr}, MV{c->U, c->nr, c->k, c->nr});
            zcopy2d(h, MV{Vs, c->nc, c->k, c->nc}, MV{c->V, c->nc, c->k, c->nc});
            off = c->k;
        }
        for (size_t i = 0; i < c->pu.size(); ++i) {
            zcopy2d(h, MV{Us + (size_t)off * c->nr, c->nr, c->pk[i], c->nr}, MV{c->pu[i], c->nr, c->pk[i], c->nr});
            zcopy2d(h, MV{Vs + (size_t)off * c->nc, c->nc, c->pk[i], c->nc}, MV{c->pv[i], c->nc, c->pk[i], c->nc});
            off += c->pk[i];
            dfree(h, c->pu[i]);
            dfree(h, c->pv[i]);
        }
        c->pu.clear();
        c->pv.clear();
        c->pk.clear();
        c->pend_k = 0;
        if (c->U) dfree(h, c->U);
        if (c->V) dfree(h, c->V);
        c->U = Us;
        c->V = Vs;
        c->k = K;
        ranks.push_back(K);
    }
    batched_truncate(h, list, ranks, h->tol);
}

// C += alpha U V^H  (U: C.nr x k, V: C.nc x k)
static void add_lr(hm_handle_s *h, Block *C, MV U, MV V, zc alpha)
{
    int k = U.cols;
    if (k <= 0) return;
    switch (C->type) {
    case B_DENSE:
        zgemm(h, 'N', 'C', C->nr, C->nc, k, alpha, U.p, U.ld, V.p, V.ld, ONE, C->D, C->nr);
        break;
    case B_LR: {
        // append (alpha U) V^H to the pending updates; recompressed at the next flush
        zc *Up = zalloc(h, (size_t)C->nr * k), *Vp = zalloc(h, (size_t)C->nc * k);
        zcopy2d(h, MV{Up, C->nr, k, C->nr}, U);
        zcopy2d(h, MV{Vp, C->nc, k, C->nc}, V);
        if (alpha.x != 1.0 || alpha.y != 0.0)  // zgemm with k = 0 computes C = alpha C
            zgemm(h, 'N', 'N', C->nr, k, 0, ZERO, nullptr, 1, nullptr, 1, alpha, Up, C->nr);
        C->pu.push_back(Up);
        C->pv.push_back(Vp);
        C->pk.push_back(k);
        C->pend_k += k;
        if (C->k + C->pend_k > std::max(256, std::min(C->nr, C->nc))) flush(h, C);
        break;
    }
    case B_HIER:
        for (int c = 0; c < 4; ++c) {
            Block *b = C->ch[c];
            add_lr(h, b, rows_of(U, b->r0 - C->r0, b->nr), rows_of(V, b->c0 - C->c0, b->nc), alpha);
        }
        break;
    }
}

// P += alpha A B into a dense view P (A.nr x B.nc)
static void mul_dense(hm_handle_s *h, MV P, Block *A, Block *B, zc alpha)
{
    if (A->type == B_LR) {
        if (A->k == 0) return;
        zc *Y = zalloc(h, (size_t)B->nc * A->k);
        zzero(h, MV{Y, B->nc, A->k, B->nc});
        hmatvec(h, B, MV{A->V, A->nc, A->k, A->nc}, MV{Y, B->nc, A->k, B->nc}, ONE, true);
        zgemm(h, 'N', 'C', A->nr, B->nc, A->k, alpha, A->U, A->nr, Y, B->nc, ONE, P.p, P.ld);
        dfree(h, Y);
    } else if (B->type == B_LR) {
        if (B->k == 0) return;
        zc *X = zalloc(h, (size_t)A->nr * B->k);
        zzero(h, MV{X, A->nr, B->k, A->nr});
        hmatvec(h, A, MV{B->U, B->nr, B->k, B->nr}, MV{X, A->nr, B->k, A->nr}, ONE, false);
        zgemm(h, 'N', 'C', A->nr, B->nc, B->k, alpha, X, A->nr, B->V, B->nc, ONE, P.p, P.ld);
        dfree(h, X);
    } else if (A->type == B_DENSE && B->type == B_DENSE) {
        zgemm(h, 'N', 'N', A->nr, B->nc, A->nc, alpha, A->D, A->nr, B->D, B->nr, ONE, P.p, P.ld);
    } else if (A->type == B_HIER && B->type == B_HIER) {
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j)
                for (int l = 0; l < 2; ++l) {
                    Block *a = A->ch[2 * i + l], *b = B->ch[2 * l + j];
                    MV Pij{P.p + (size_t)(b->c0 - B->c0) * P.ld + (a->r0 - A->r0), a->nr, b->nc, P.ld};
                    mul_dense(h, Pij, a, b, alpha);
                }
    } else {
        throw HmError{HM_ERR_STATE, "mul_dense: mixed dense/hierarchical operands"};
    }
}

__global__ void k_identity(zc *I, int n)
{
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)n * n) return;
    I[idx] = zmake((idx % n) == (idx / n) ? 1.0 : 0.0, 0.0);
}

__global__ void k_ctrans(const zc *A, int lda, int m, int n, zc *B)  // B (n x m) = A^H
{
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)m * n) return;
    int i = (int)(idx % m), j = (int)(idx / m);
    B[(size_t)i * n + j] = zconj(A[(size_t)j * lda + i]);
}

// C += alpha A B  (formatted)
static void addmul(hm_handle_s *h, Block *C, Block *A, Block *B, zc alpha)
{
    if (A->pend_k) flush(h, A);
    if (B->pend_k) flush(h, B);
    if (A->type == B_LR) {
        if (A->k == 0) return;
        zc *Y = zalloc(h, (size_t)B->nc * A->k);  // Y = B^H V_A
        zzero(h, MV{Y, B->nc, A->k, B->nc});
        hmatvec(h, B, MV{A->V, A->nc, A->k, A->nc}, MV{Y, B->nc, A->k, B->nc}, ONE, true);
        add_lr(h, C, MV{A->U, A->nr, A->k, A->nr}, MV{Y, B->nc, A->k, B->nc}, alpha);
        dfree(h, Y);
        return;
    }
    if (B->type == B_LR) {
        if (B->k == 0) return;
        zc *X = zalloc(h, (size_t)A->nr * B->k);  // X = A U_B
        zzero(h, MV{X, A->nr, B->k, A->nr});
        hmatvec(h, A, MV{B->U, B->nr, B->k, B->nr}, MV{X, A->nr, B->k, A->nr}, ONE, false);
        add_lr(h, C, MV{X, A->nr, B->k, A->nr}, MV{B->V, B->nc, B->k, B->nc}, alpha);
        dfree(h, X);
        return;
    }
    if (C->type == B_HIER && A->type == B_HIER && B->type == B_HIER) {
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j)
                for (int l = 0; l < 2; ++l) addmul(h, C->ch[2 * i + j], A->ch[2 * i + l], B->ch[2 * l + j], alpha);
        return;
    }
    if (C->type == B_DENSE) {
        mul_dense(h, MV{C->D, C->nr, C->nc, C->nr}, A, B, alpha);
        return;
    }
    if (C->type == B_LR) {
        if (A->type == B_DENSE && B->type == B_DENSE) {
            // A B = A (B^H)^H: exact low-rank form of rank A.nc
            zc *Bh = zalloc(h, (size_t)B->nc * B->nr);
            size_t n = (size_t)B->nr * B->nc;
            k_ctrans<<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(B->D, B->nr, B->nr, B->nc, Bh);
            HM_CHECK_LAUNCH();
            count_launch(h);
            add_lr(h, C, MV{A->D, A->nr, A->nc, A->nr}, MV{Bh, B->nc, B->nr, B->nc}, alpha);
            dfree(h, Bh);
            return;
        }
        if (A->type == B_HIER && B->type == B_HIER) {
            // hierarchical product into a low-rank block: products of the 2 x 2 children into
            // temporary low-rank blocks, agglomerated and recompressed into C
            Block T[4];
            for (int i = 0; i < 2; ++i)
                for (int j = 0; j < 2; ++j) {
                    Block &t = T[2 * i + j];
                    t.type = B_LR;
                    t.r0 = A->ch[2 * i]->r0;
                    t.nr = A->ch[2 * i]->nr;
                    t.c0 = B->ch[j]->c0;
                    t.nc = B->ch[j]->nc;
                    t.k = 0;
                }
            for (int i = 0; i < 2; ++i)
                for (int j = 0; j < 2; ++j)
                    for (int l = 0; l < 2; ++l) addmul(h, &T[2 * i + j], A->ch[2 * i + l], B->ch[2 * l + j], ONE);
            {
                // recompress the four temporaries in one batch
                Block Hh;
                Hh.type = B_HIER;
                for (int t = 0; t < 4; ++t) Hh.ch[t] = &T[t];
                flush(h, &Hh);
            }
            int K = T[0].k + T[1].k + T[2].k + T[3].k;
            if (K > 0) {
                zc *Ua = zalloc(h, (size_t)C->nr * K), *Va = zalloc(h, (size_t)C->nc * K);
                zzero(h, MV{Ua, C->nr, K, C->nr});
                zzero(h, MV{Va, C->nc, K, C->nc});
                int off = 0;
                for (int t = 0; t < 4; ++t) {
                    if (!T[t].k) continue;
                    zcopy2d(h, MV{Ua + (size_t)off * C->nr + (T[t].r0 - C->r0), T[t].nr, T[t].k, C->nr},
                            MV{T[t].U, T[t].nr, T[t].k, T[t].nr});
                    zcopy2d(h, MV{Va + (size_t)off * C->nc + (T[t].c0 - C->c0), T[t].nc, T[t].k, C->nc},
                            MV{T[t].V, T[t].nc, T[t].k, T[t].nc});
                    off += T[t].k;
                }
                add_lr(h, C, MV{Ua, C->nr, K, C->nr}, MV{Va, C->nc, K, C->nc}, alpha);
                dfree(h, Ua);
                dfree(h, Va);
            }
            for (int t = 0; t < 4; ++t) {
                if (T[t].U) dfree(h, T[t].U);
                if (T[t].V) dfree(h, T[t].V);
            }
            return;
        }
        // a dense operand at a hierarchical level (a block stored dense after ACA hit its
        // rank bound): dense product, then [U | P][V | I]
        zc *P = zalloc(h, (size_t)C->nr * C->nc);
        zzero(h, MV{P, C->nr, C->nc, C->nr});
        mul_dense(h, MV{P, C->nr, C->nc, C->nr}, A, B, ONE);
        zc *I = zalloc(h, (size_t)C->nc * C->nc);
        size_t n = (size_t)C->nc * C->nc;
        k_identity<<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(I, C->nc);
        HM_CHECK_LAUNCH();
        count_launch(h);
        add_lr(h, C, MV{P, C->nr, C->nc, C->nr}, MV{I, C->nc, C->nc, C->nc}, alpha);
        dfree(h, P);
        dfree(h, I);
        return;
    }
    throw HmError{HM_ERR_STATE, "addmul: unsupported block formats"};
}

// X <- L^-1 P X for a factored diagonal block L (rows of X = L.nr)
static void trsm_L_mv(hm_handle_s *h, Block *L, MV X)
{
    if (X.cols <= 0) return;
    if (L->type == B_DENSE) {
        zlaswp(h, X, L->piv, L->nr);
        ztrsm_lln(h, L->D, L->nr, L->nr, X);
        return;
    }
    Block *L11 = L->ch[0], *L21 = L->ch[2], *L22 = L->ch[3];
    MV X1 = rows_of(X, 0, L11->nr), X2 = rows_of(X, L11->nr, L22->nr);
    trsm_L_mv(h, L11, X1);
    hmatvec(h, L21, X1, X2, MONE, false);
    trsm_L_mv(h, L22, X2);
}

// X <- U^-1 X
static void trsm_U_mv(hm_handle_s *h, Block *U, MV X)
{
    if (X.cols <= 0) return;
    if (U->type == B_DENSE) {
        ztrsm_lun(h, U->D, U->nr, U->nr, X);
        return;
    }
    Block *U11 = U->ch[0], *U12 = U->ch[1], *U22 = U->ch[3];
    MV X1 = rows_of(X, 0, U11->nr), X2 = rows_of(X, U11->nr, U22->nr);
    trsm_U_mv(h, U22, X2);
    hmatvec(h, U12, X2, X1, MONE, false);
    trsm_U_mv(h, U11, X1);
}

// X <- U^-H X
static void trsm_UH_mv(hm_handle_s *h, Block *U, MV X)
{
    if (X.cols <= 0) return;
    if (U->type == B_DENSE) {
        ztrsm_luh(h, U->D, U->nr, U->nr, X);
        return;
    }
    Block *U11 = U->ch[0], *U12 = U->ch[1], *U22 = U->ch[3];
    MV X1 = rows_of(X, 0, U11->nr), X2 = rows_of(X, U11->nr, U22->nr);
    trsm_UH_mv(h, U11, X1);
    hmatvec(h, U12, X1, X2, MONE, true);
    trsm_UH_mv(h, U22, X2);
}

static void trsm_UH_mv(hm_handle_s *h, Block *U, MV X);

// B <- L^-1 P B  (B has the row cluster of L)
static void trsm_L_block(hm_handle_s *h, Block *L, Block *B)
{
    flush(h, B);
    if (B->type == B_LR) {
        trsm_L_mv(h, L, MV{B->U, B->nr, B->k, B->nr});
        return;
    }
    if (B->type == B_DENSE) {
        trsm_L_mv(h, L, MV{B->D, B->nr, B->nc, B->nr});
        return;
    }
    if (L->type != B_HIER) throw HmError{HM_ERR_STATE, "trsm_L_block: hierarchical B under a dense L"};
    for (int j = 0; j < 2; ++j) {
        trsm_L_block(h, L->ch[0], B->ch[j]);
        addmul(h, B->ch[2 + j], L->ch[2], B->ch[j], MONE);
        trsm_L_block(h, L->ch[3], B->ch[2 + j]);
    }
}

// B <- B U^-1  (B has the column cluster of U)
static void trsm_U_right_block(hm_handle_s *h, Block *U, Block *B)
{
    flush(h, B);
    if (B->type == B_LR) {
        trsm_UH_mv(h, U, MV{B->V, B->nc, B->k, B->nc});
        return;
    }
    if (B->type == B_DENSE) {
        if (U->type == B_DENSE) {
            ztrsm_run(h, U->D, U->nr, U->nr, MV{B->D, B->nr, B->nc, B->nr});
            return;
        }
        // B U^-1 = (U^-H B^H)^H
        zc *Bh = zalloc(h, (size_t)B->nc * B->nr);
        size_t n = (size_t)B->nr * B->nc;
        k_ctrans<<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(B->D, B->nr, B->nr, B->nc, Bh);
        HM_CHECK_LAUNCH();
        trsm_UH_mv(h, U, MV{Bh, B->nc, B->nr, B->nc});
        k_ctrans<<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(Bh, B->nc, B->nc, B->nr, B->D);
        HM_CHECK_LAUNCH();
        count_launch(h, 2);
        dfree(h, Bh);
        return;
    }
    if (U->type != B_HIER) throw HmError{HM_ERR_STATE, "trsm_U_right_block: hierarchical B under a dense U"};
    for (int i = 0; i < 2; ++i) {
        trsm_U_right_block(h, U->ch[0], B->ch[2 * i]);
        addmul(h, B->ch[2 * i + 1], B->ch[2 * i], U->ch[1], MONE);
        trsm_U_right_block(h, U->ch[3], B->ch[2 * i + 1]);
    }
}

static void hlu_rec(hm_handle_s *h, Block *A, int *d_info)
{
    flush(h, A);
    if (A->type == B_DENSE) {
        if (!A->piv) A->piv = (int *)dalloc(h, sizeof(int) * A->nr);
        zgetrf(h, A->nr, A->D, A->nr, A->piv, d_info);
        return;
    }
    if (A->type != B_HIER) throw HmError{HM_ERR_STATE, "H-LU: low-rank diagonal block"};
    hlu_rec(h, A->ch[0], d_info);
    trsm_L_block(h, A->ch[0], A->ch[1]);
    trsm_U_right_block(h, A->ch[0], A->ch[2]);
    addmul(h, A->ch[3], A->ch[2], A->ch[1], MONE);
    hlu_rec(h, A->ch[3], d_info);
}

// Invariant: operands of addmul / hmatvec are free of pending updates (every
// triangular solve and every diagonal step flushes its target subtree first), so
// only low-rank leaves are checked there.
void hlu_factor(hm_handle_s *h)
{
    int *d_info = (int *)dalloc(h, sizeof(int));
    HM_CUDA(cudaMemsetAsync(d_info, 0, sizeof(int), h->stream));
    hlu_rec(h, h->root, d_info);
    flush(h, h->root);
    int info = 0;
    HM_CUDA(cudaMemcpyAsync(&info, d_info, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    HM_CUDA(cudaStreamSynchronize(h->stream));
    dfree(h, d_info);
    if (info) throw HmError{HM_ERR_SINGULAR, "H-LU: zero pivot in a diagonal leaf"};
}

void hsolve(hm_handle_s *h, MV X)
{
    trsm_L_mv(h, h->root, X);
    trsm_U_mv(h, h->root, X);
}

Block *clone_tree(hm_handle_s *h, Block *b, std::vector<Block *> &owned)
{
    Block *c = new Block(*b);
    owned.push_back(c);
    c->piv = nullptr;
    c->D = c->U = c->V = nullptr;
    if (b->type == B_DENSE) {
        c->D = zalloc(h, (size_t)b->nr * b->nc);
        HM_CUDA(cudaMemcpyAsync(c->D, b->D, sizeof(zc) * (size_t)b->nr * b->nc, cudaMemcpyDeviceToDevice, h->stream));
    } else if (b->type == B_LR) {
        if (b->k) {
            c->U = zalloc(h, (size_t)b->nr * b->k);
            c->V = zalloc(h, (size_t)b->nc * b->k);
            HM_CUDA(cudaMemcpyAsync(c->U, b->U, sizeof(zc) * (size_t)b->nr * b->k, cudaMemcpyDeviceToDevice, h->stream));
            HM_CUDA(cudaMemcpyAsync(c->V, b->V, sizeof(zc) * (size_t)b->nc * b->k, cudaMemcpyDeviceToDevice, h->stream));
        }
    } else {
        for (int i = 0; i < 4; ++i) c->ch[i] = clone_tree(h, b->ch[i], owned);
    }
    return c;
}

void free_tree(hm_handle_s *h, std::vector<Block *> &owned)
{
    for (Block *b : owned) {
        if (b->D) dfree(h, b->D);
        if (b->U) dfree(h, b->U);
        if (b->V) dfree(h, b->V);
        if (b->piv) dfree(h, b->piv);
        delete b;
    }
    owned.clear();
}
