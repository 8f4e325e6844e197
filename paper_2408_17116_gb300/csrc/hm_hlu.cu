// H-LU factorisation (Sec. III: block LU of Eq. 23 applied recursively) on the
// entire-matrix block cluster tree (Sec. III.B: one tree over all unknowns).  The
// substitutions of Eqs. 24-28 with the factors run as block-row sweeps (hm_tiles.cu); the
// H-triangular solves below serve the factorisation itself (L^-1 and U^-1 applied to the
// off-diagonal blocks).
//
// Recursion on a diagonal block A = [[A11, A12], [A21, A22]]:
//   A11 = P1^T L11 U11                       (recursive; partial pivoting inside dense leaves)
//   U12 = L11^-1 P1 A12,  L21 = A21 U11^-1   (H-triangular solves)
//   S   = A22 - L21 U12                      (formatted multiply-add with truncation)
//   S   = P2^T L22 U22                       (recursive)
// so that A x = b is solved by y1 = L11^-1 P1 b1, y2 = L22^-1 P2 (b2 - L21 y1),
// x2 = U22^-1 y2, x1 = U11^-1 (y1 - U12 x2).  Low-rank blocks are U V^H; every
// low-rank sum is recompressed (QR + SVD) to the factorisation's truncation
// tolerance.  Everything is a template over the storage precision: complex128 for
// the FP64 method, complex64 for the FP32 factor used as a preconditioner.
#include <algorithm>

#include "hm_internal.h"

template <class Z>
static inline MVT<Z> rows_of(MVT<Z> X, int r0, int nr) { return MVT<Z>{X.p + r0, nr, X.cols, X.ld}; }
template <class Z>
void flush(hm_handle_s *h, BlockT<Z> *b);

template <class Z>
static Z *zalloc(hm_handle_s *h, size_t n) { return (Z *)dalloc(h, sizeof(Z) * std::max<size_t>(n, 1)); }

template <class Z>
static void zzero(hm_handle_s *h, MVT<Z> X)
{
    if (X.rows <= 0 || X.cols <= 0) return;
    if (X.ld == X.rows) {
        HM_CUDA(cudaMemsetAsync(X.p, 0, sizeof(Z) * (size_t)X.rows * X.cols, h->stream));
    } else {
        for (int j = 0; j < X.cols; ++j)
            HM_CUDA(cudaMemsetAsync(X.p + (size_t)j * X.ld, 0, sizeof(Z) * X.rows, h->stream));
    }
}

// Y += alpha op(A) X,  op = N (X rows = A.nc) or C (X rows = A.nr)
template <class Z>
void hmatvec(hm_handle_s *h, BlockT<Z> *A, MVT<Z> X, MVT<Z> Y, Z alpha, bool ct)
{
    if (X.cols <= 0) return;
    if (A->pend_k) flush(h, A);
    switch (A->type) {
    case B_DENSE:
        if (!ct)
            zgemm<Z>(h, 'N', 'N', A->nr, X.cols, A->nc, alpha, A->D, A->nr, X.p, X.ld, cmk<Z>(1, 0), Y.p, Y.ld);
        else
            zgemm<Z>(h, 'C', 'N', A->nc, X.cols, A->nr, alpha, A->D, A->nr, X.p, X.ld, cmk<Z>(1, 0), Y.p, Y.ld);
        break;
    case B_LR: {
        if (A->k == 0) return;
        Z *t = zalloc<Z>(h, (size_t)A->k * X.cols);
        if (!ct) {
            zgemm<Z>(h, 'C', 'N', A->k, X.cols, A->nc, cmk<Z>(1, 0), A->V, A->nc, X.p, X.ld, cmk<Z>(0, 0), t, A->k);
            zgemm<Z>(h, 'N', 'N', A->nr, X.cols, A->k, alpha, A->U, A->nr, t, A->k, cmk<Z>(1, 0), Y.p, Y.ld);
        } else {
            zgemm<Z>(h, 'C', 'N', A->k, X.cols, A->nr, cmk<Z>(1, 0), A->U, A->nr, X.p, X.ld, cmk<Z>(0, 0), t, A->k);
            zgemm<Z>(h, 'N', 'N', A->nc, X.cols, A->k, alpha, A->V, A->nc, t, A->k, cmk<Z>(1, 0), Y.p, Y.ld);
        }
        dfree(h, t);
        break;
    }
    case B_HIER:
        for (int c = 0; c < 4; ++c) {
            BlockT<Z> *b = A->ch[c];
            int ro = b->r0 - A->r0, co = b->c0 - A->c0;
            if (!ct)
                hmatvec(h, b, rows_of(X, co, b->nc), rows_of(Y, ro, b->nr), alpha, false);
            else
                hmatvec(h, b, rows_of(X, ro, b->nr), rows_of(Y, co, b->nc), alpha, true);
        }
        break;
    }
}


template <class Z>
static void collect_pending(BlockT<Z> *b, std::vector<BlockT<Z> *> &out)
{
    if (b->type == B_HIER) {
        for (int i = 0; i < 4; ++i) collect_pending(b->ch[i], out);
    } else if (b->type == B_LR && b->pend_k > 0 && !b->in_batch) {
        b->in_batch = true;
        out.push_back(b);
    }
}

template <class Z>
std::vector<BlockT<Z> *> &dirty_list(hm_handle_s *h);
template <>
std::vector<Block *> &dirty_list<zc>(hm_handle_s *h)
{
    return h->dirty64;
}
template <>
std::vector<Block32 *> &dirty_list<cf>(hm_handle_s *h)
{
    return h->dirty32;
}

// Recompress, in one batch, every low-rank block of b's subtree that has pending
// updates, together with every block queued as dirty anywhere in the matrix:
// [U | Up_1 | ...] [V | Vp_1 | ...]^H -> truncated U' V'^H.
template <class Z>
void flush(hm_handle_s *h, BlockT<Z> *b)
{
    std::vector<BlockT<Z> *> list;
    collect_pending(b, list);
    std::vector<BlockT<Z> *> &dl = dirty_list<Z>(h);
    for (BlockT<Z> *d : dl) {
        d->dirty = false;
        if (d->pend_k > 0 && !d->in_batch) {
            d->in_batch = true;
            list.push_back(d);
        }
    }
    dl.clear();
    for (BlockT<Z> *c : list) c->in_batch = false;
    if (list.empty()) return;
    std::vector<int> ranks;
    for (BlockT<Z> *c : list) {
        int K = c->k + c->pend_k;
        Z *Us = zalloc<Z>(h, (size_t)c->nr * K), *Vs = zalloc<Z>(h, (size_t)c->nc * K);
        int off = 0;
        if (c->k) {
            zcopy2d(h, MVT<Z>{Us, c->nr, c->k, c->nr}, MVT<Z>{c->U, c->nr, c->k, c->nr});
            zcopy2d(h, MVT<Z>{Vs, c->nc, c->k, c->nc}, MVT<Z>{c->V, c->nc, c->k, c->nc});
            off = c->k;
        }
        for (size_t i = 0; i < c->pu.size(); ++i) {
            zcopy2d(h, MVT<Z>{Us + (size_t)off * c->nr, c->nr, c->pk[i], c->nr}, MVT<Z>{c->pu[i], c->nr, c->pk[i], c->nr});
            zcopy2d(h, MVT<Z>{Vs + (size_t)off * c->nc, c->nc, c->pk[i], c->nc}, MVT<Z>{c->pv[i], c->nc, c->pk[i], c->nc});
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
    batched_truncate(h, list, ranks, h->cur_tol);
}

// C += alpha U V^H  (U: C.nr x k, V: C.nc x k)
template <class Z>
static void add_lr(hm_handle_s *h, BlockT<Z> *C, MVT<Z> U, MVT<Z> V, Z alpha)
{
    int k = U.cols;
    if (k <= 0) return;
    switch (C->type) {
    case B_DENSE:
        zgemm<Z>(h, 'N', 'C', C->nr, C->nc, k, alpha, U.p, U.ld, V.p, V.ld, cmk<Z>(1, 0), C->D, C->nr);
        break;
    case B_LR: {
        // append (alpha U) V^H to the pending updates; recompressed at the next flush
        Z *Up = zalloc<Z>(h, (size_t)C->nr * k), *Vp = zalloc<Z>(h, (size_t)C->nc * k);
        zcopy2d(h, MVT<Z>{Up, C->nr, k, C->nr}, U);
        zcopy2d(h, MVT<Z>{Vp, C->nc, k, C->nc}, V);
        if (alpha.x != 1.0 || alpha.y != 0.0)  // zgemm with k = 0 computes C = alpha C
            zgemm<Z>(h, 'N', 'N', C->nr, k, 0, cmk<Z>(0, 0), nullptr, 1, nullptr, 1, alpha, Up, C->nr);
        C->pu.push_back(Up);
        C->pv.push_back(Vp);
        C->pk.push_back(k);
        C->pend_k += k;
        // once the pending columns reach the current rank (at least 32) the block is
        // queued for the next batched recompression; beyond four times that bound it is
        // recompressed at once
        if (C->pend_k >= std::max(32, C->k)) {
            if (C->k + C->pend_k > 4 * std::max(64, C->k)) {
                flush(h, C);
            } else if (!C->dirty) {
                C->dirty = true;
                dirty_list<Z>(h).push_back(C);
            }
        }
        break;
    }
    case B_HIER:
        for (int c = 0; c < 4; ++c) {
            BlockT<Z> *b = C->ch[c];
            add_lr(h, b, rows_of(U, b->r0 - C->r0, b->nr), rows_of(V, b->c0 - C->c0, b->nc), alpha);
        }
        break;
    }
}

// P += alpha A B into a dense view P (A.nr x B.nc)
template <class Z>
static void mul_dense(hm_handle_s *h, MVT<Z> P, BlockT<Z> *A, BlockT<Z> *B, Z alpha)
{
    if (A->type == B_LR) {
        if (A->k == 0) return;
        Z *Y = zalloc<Z>(h, (size_t)B->nc * A->k);
        zzero(h, MVT<Z>{Y, B->nc, A->k, B->nc});
        hmatvec(h, B, MVT<Z>{A->V, A->nc, A->k, A->nc}, MVT<Z>{Y, B->nc, A->k, B->nc}, cmk<Z>(1, 0), true);
        zgemm<Z>(h, 'N', 'C', A->nr, B->nc, A->k, alpha, A->U, A->nr, Y, B->nc, cmk<Z>(1, 0), P.p, P.ld);
        dfree(h, Y);
    } else if (B->type == B_LR) {
        if (B->k == 0) return;
        Z *X = zalloc<Z>(h, (size_t)A->nr * B->k);
        zzero(h, MVT<Z>{X, A->nr, B->k, A->nr});
        hmatvec(h, A, MVT<Z>{B->U, B->nr, B->k, B->nr}, MVT<Z>{X, A->nr, B->k, A->nr}, cmk<Z>(1, 0), false);
        zgemm<Z>(h, 'N', 'C', A->nr, B->nc, B->k, alpha, X, A->nr, B->V, B->nc, cmk<Z>(1, 0), P.p, P.ld);
        dfree(h, X);
    } else if (A->type == B_DENSE && B->type == B_DENSE) {
        zgemm<Z>(h, 'N', 'N', A->nr, B->nc, A->nc, alpha, A->D, A->nr, B->D, B->nr, cmk<Z>(1, 0), P.p, P.ld);
    } else if (A->type == B_HIER && B->type == B_HIER) {
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j)
                for (int l = 0; l < 2; ++l) {
                    BlockT<Z> *a = A->ch[2 * i + l], *b = B->ch[2 * l + j];
                    MVT<Z> Pij{P.p + (size_t)(b->c0 - B->c0) * P.ld + (a->r0 - A->r0), a->nr, b->nc, P.ld};
                    mul_dense(h, Pij, a, b, alpha);
                }
    } else {
        throw HmError{HM_ERR_STATE, "mul_dense: mixed dense/hierarchical operands"};
    }
}

template <class Z>
__global__ void k_identity(Z *I, int n)
{
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)n * n) return;
    I[idx] = cmk<Z>((idx % n) == (idx / n) ? 1.0 : 0.0, 0.0);
}

template <class Z>
__global__ void k_ctrans(const Z *A, int lda, int m, int n, Z *B)  // B (n x m) = A^H
{
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)m * n) return;
    int i = (int)(idx % m), j = (int)(idx / m);
    B[(size_t)i * n + j] = zconj(A[(size_t)j * lda + i]);
}

// C += alpha A B  (formatted)
template <class Z>
static void addmul(hm_handle_s *h, BlockT<Z> *C, BlockT<Z> *A, BlockT<Z> *B, Z alpha)
{
    if (A->pend_k) flush(h, A);
    if (B->pend_k) flush(h, B);
    if (A->type == B_LR) {
        if (A->k == 0) return;
        Z *Y = zalloc<Z>(h, (size_t)B->nc * A->k);  // Y = B^H V_A
        zzero(h, MVT<Z>{Y, B->nc, A->k, B->nc});
        hmatvec(h, B, MVT<Z>{A->V, A->nc, A->k, A->nc}, MVT<Z>{Y, B->nc, A->k, B->nc}, cmk<Z>(1, 0), true);
        add_lr(h, C, MVT<Z>{A->U, A->nr, A->k, A->nr}, MVT<Z>{Y, B->nc, A->k, B->nc}, alpha);
        dfree(h, Y);
        return;
    }
    if (B->type == B_LR) {
        if (B->k == 0) return;
        Z *X = zalloc<Z>(h, (size_t)A->nr * B->k);  // X = A U_B
        zzero(h, MVT<Z>{X, A->nr, B->k, A->nr});
        hmatvec(h, A, MVT<Z>{B->U, B->nr, B->k, B->nr}, MVT<Z>{X, A->nr, B->k, A->nr}, cmk<Z>(1, 0), false);
        add_lr(h, C, MVT<Z>{X, A->nr, B->k, A->nr}, MVT<Z>{B->V, B->nc, B->k, B->nc}, alpha);
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
        mul_dense(h, MVT<Z>{C->D, C->nr, C->nc, C->nr}, A, B, alpha);
        return;
    }
    if (C->type == B_LR) {
        if (A->type == B_DENSE && B->type == B_DENSE) {
            // A B = A (B^H)^H: exact low-rank form of rank A.nc
            Z *Bh = zalloc<Z>(h, (size_t)B->nc * B->nr);
            size_t n = (size_t)B->nr * B->nc;
            k_ctrans<Z><<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(B->D, B->nr, B->nr, B->nc, Bh);
            HM_CHECK_LAUNCH();
            count_launch(h);
            add_lr(h, C, MVT<Z>{A->D, A->nr, A->nc, A->nr}, MVT<Z>{Bh, B->nc, B->nr, B->nc}, alpha);
            dfree(h, Bh);
            return;
        }
        if (A->type == B_HIER && B->type == B_HIER) {
            // hierarchical product into a low-rank block: products of the 2 x 2 children into
            // temporary low-rank blocks, agglomerated and recompressed into C
            BlockT<Z> T[4];
            for (int i = 0; i < 2; ++i)
                for (int j = 0; j < 2; ++j) {
                    BlockT<Z> &t = T[2 * i + j];
                    t.type = B_LR;
                    t.r0 = A->ch[2 * i]->r0;
                    t.nr = A->ch[2 * i]->nr;
                    t.c0 = B->ch[j]->c0;
                    t.nc = B->ch[j]->nc;
                    t.k = 0;
                }
            for (int i = 0; i < 2; ++i)
                for (int j = 0; j < 2; ++j)
                    for (int l = 0; l < 2; ++l) addmul(h, &T[2 * i + j], A->ch[2 * i + l], B->ch[2 * l + j], cmk<Z>(1, 0));
            {
                // recompress the four temporaries in one batch
                BlockT<Z> Hh;
                Hh.type = B_HIER;
                for (int t = 0; t < 4; ++t) Hh.ch[t] = &T[t];
                flush(h, &Hh);
            }
            int K = T[0].k + T[1].k + T[2].k + T[3].k;
            if (K > 0) {
                Z *Ua = zalloc<Z>(h, (size_t)C->nr * K), *Va = zalloc<Z>(h, (size_t)C->nc * K);
                zzero(h, MVT<Z>{Ua, C->nr, K, C->nr});
                zzero(h, MVT<Z>{Va, C->nc, K, C->nc});
                int off = 0;
                for (int t = 0; t < 4; ++t) {
                    if (!T[t].k) continue;
                    zcopy2d(h, MVT<Z>{Ua + (size_t)off * C->nr + (T[t].r0 - C->r0), T[t].nr, T[t].k, C->nr},
                            MVT<Z>{T[t].U, T[t].nr, T[t].k, T[t].nr});
                    zcopy2d(h, MVT<Z>{Va + (size_t)off * C->nc + (T[t].c0 - C->c0), T[t].nc, T[t].k, C->nc},
                            MVT<Z>{T[t].V, T[t].nc, T[t].k, T[t].nc});
                    off += T[t].k;
                }
                add_lr(h, C, MVT<Z>{Ua, C->nr, K, C->nr}, MVT<Z>{Va, C->nc, K, C->nc}, alpha);
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
        Z *P = zalloc<Z>(h, (size_t)C->nr * C->nc);
        zzero(h, MVT<Z>{P, C->nr, C->nc, C->nr});
        mul_dense(h, MVT<Z>{P, C->nr, C->nc, C->nr}, A, B, cmk<Z>(1, 0));
        Z *I = zalloc<Z>(h, (size_t)C->nc * C->nc);
        size_t n = (size_t)C->nc * C->nc;
        k_identity<Z><<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(I, C->nc);
        HM_CHECK_LAUNCH();
        count_launch(h);
        add_lr(h, C, MVT<Z>{P, C->nr, C->nc, C->nr}, MVT<Z>{I, C->nc, C->nc, C->nc}, alpha);
        dfree(h, P);
        dfree(h, I);
        return;
    }
    throw HmError{HM_ERR_STATE, "addmul: unsupported block formats"};
}

// X <- L^-1 P X for a factored diagonal block L (rows of X = L.nr)
template <class Z>
static void trsm_L_mv(hm_handle_s *h, BlockT<Z> *L, MVT<Z> X)
{
    if (X.cols <= 0) return;
    if (L->type == B_DENSE) {
        zlaswp(h, X, L->piv, L->nr);
        ztrsm_lln(h, L->D, L->nr, L->nr, X);
        return;
    }
    BlockT<Z> *L11 = L->ch[0], *L21 = L->ch[2], *L22 = L->ch[3];
    MVT<Z> X1 = rows_of(X, 0, L11->nr), X2 = rows_of(X, L11->nr, L22->nr);
    trsm_L_mv(h, L11, X1);
    hmatvec(h, L21, X1, X2, cmk<Z>(-1, 0), false);
    trsm_L_mv(h, L22, X2);
}

// X <- U^-1 X
template <class Z>
static void trsm_U_mv(hm_handle_s *h, BlockT<Z> *U, MVT<Z> X)
{
    if (X.cols <= 0) return;
    if (U->type == B_DENSE) {
        ztrsm_lun(h, U->D, U->nr, U->nr, X);
        return;
    }
    BlockT<Z> *U11 = U->ch[0], *U12 = U->ch[1], *U22 = U->ch[3];
    MVT<Z> X1 = rows_of(X, 0, U11->nr), X2 = rows_of(X, U11->nr, U22->nr);
    trsm_U_mv(h, U22, X2);
    hmatvec(h, U12, X2, X1, cmk<Z>(-1, 0), false);
    trsm_U_mv(h, U11, X1);
}

// X <- U^-H X
template <class Z>
static void trsm_UH_mv(hm_handle_s *h, BlockT<Z> *U, MVT<Z> X)
{
    if (X.cols <= 0) return;
    if (U->type == B_DENSE) {
        ztrsm_luh(h, U->D, U->nr, U->nr, X);
        return;
    }
    BlockT<Z> *U11 = U->ch[0], *U12 = U->ch[1], *U22 = U->ch[3];
    MVT<Z> X1 = rows_of(X, 0, U11->nr), X2 = rows_of(X, U11->nr, U22->nr);
    trsm_UH_mv(h, U11, X1);
    hmatvec(h, U12, X1, X2, cmk<Z>(-1, 0), true);
    trsm_UH_mv(h, U22, X2);
}


// B <- L^-1 P B  (B has the row cluster of L)
template <class Z>
static void trsm_L_block(hm_handle_s *h, BlockT<Z> *L, BlockT<Z> *B)
{
    flush(h, B);
    if (B->type == B_LR) {
        trsm_L_mv(h, L, MVT<Z>{B->U, B->nr, B->k, B->nr});
        return;
    }
    if (B->type == B_DENSE) {
        trsm_L_mv(h, L, MVT<Z>{B->D, B->nr, B->nc, B->nr});
        return;
    }
    if (L->type != B_HIER) throw HmError{HM_ERR_STATE, "trsm_L_block: hierarchical B under a dense L"};
    for (int j = 0; j < 2; ++j) {
        trsm_L_block(h, L->ch[0], B->ch[j]);
        addmul(h, B->ch[2 + j], L->ch[2], B->ch[j], cmk<Z>(-1, 0));
        trsm_L_block(h, L->ch[3], B->ch[2 + j]);
    }
}

// B <- B U^-1  (B has the column cluster of U)
template <class Z>
static void trsm_U_right_block(hm_handle_s *h, BlockT<Z> *U, BlockT<Z> *B)
{
    flush(h, B);
    if (B->type == B_LR) {
        trsm_UH_mv(h, U, MVT<Z>{B->V, B->nc, B->k, B->nc});
        return;
    }
    if (B->type == B_DENSE) {
        if (U->type == B_DENSE && U->nr <= 256) {  // row-parallel solve; larger blocks go through U^-H B^H
            ztrsm_run(h, U->D, U->nr, U->nr, MVT<Z>{B->D, B->nr, B->nc, B->nr});
            return;
        }
        // B U^-1 = (U^-H B^H)^H
        Z *Bh = zalloc<Z>(h, (size_t)B->nc * B->nr);
        size_t n = (size_t)B->nr * B->nc;
        k_ctrans<Z><<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(B->D, B->nr, B->nr, B->nc, Bh);
        HM_CHECK_LAUNCH();
        trsm_UH_mv(h, U, MVT<Z>{Bh, B->nc, B->nr, B->nc});
        k_ctrans<Z><<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(Bh, B->nc, B->nc, B->nr, B->D);
        HM_CHECK_LAUNCH();
        count_launch(h, 2);
        dfree(h, Bh);
        return;
    }
    if (U->type != B_HIER) throw HmError{HM_ERR_STATE, "trsm_U_right_block: hierarchical B under a dense U"};
    for (int i = 0; i < 2; ++i) {
        trsm_U_right_block(h, U->ch[0], B->ch[2 * i]);
        addmul(h, B->ch[2 * i + 1], B->ch[2 * i], U->ch[1], cmk<Z>(-1, 0));
        trsm_U_right_block(h, U->ch[3], B->ch[2 * i + 1]);
    }
}

template <class Z>
static void hlu_rec(hm_handle_s *h, BlockT<Z> *A, int *d_info)
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
    addmul(h, A->ch[3], A->ch[2], A->ch[1], cmk<Z>(-1, 0));
    hlu_rec(h, A->ch[3], d_info);
}

// Invariant: operands of addmul / hmatvec are free of pending updates (every
// triangular solve and every diagonal step flushes its target subtree first), so
// only low-rank leaves are checked there.  tol: truncation tolerance of every
// recompression performed by the factorisation.
// Independent bodies with each body's diagonal block dense: every block above the bodies is
// hierarchical with zero off-diagonal children, so the H-LU is one dense LU per body.  The
// diagonal blocks, or false when the tree has another shape.
template <class Z>
static bool collect_body_blocks(BlockT<Z> *b, std::vector<BlockT<Z> *> &out)
{
    if (b->type == B_DENSE) {
        out.push_back(b);
        return true;
    }
    if (b->type != B_HIER) return false;
    for (int i = 1; i <= 2; ++i)
        if (!(b->ch[i]->type == B_LR && b->ch[i]->k == 0 && b->ch[i]->pend_k == 0)) return false;
    return collect_body_blocks(b->ch[0], out) && collect_body_blocks(b->ch[3], out);
}

// The per-body LUs of a batch, concurrently on the stream pool (largest first, round robin).
template <class Z>
static bool hlu_factor_bodies(hm_handle_s *h, BlockT<Z> *root)
{
    std::vector<BlockT<Z> *> diag;
    if (!collect_body_blocks(root, diag) || diag.size() < 2) return false;
    std::stable_sort(diag.begin(), diag.end(), [](const BlockT<Z> *a, const BlockT<Z> *b) { return a->nr > b->nr; });
    int *d_info = (int *)dalloc(h, sizeof(int));
    HM_CUDA(cudaMemsetAsync(d_info, 0, sizeof(int), h->stream));
    for (BlockT<Z> *d : diag)
        if (!d->piv) d->piv = (int *)dalloc(h, sizeof(int) * d->nr);
    const int ns = (int)std::min<size_t>(HM_POOL_STREAMS, diag.size());
    h->d_info_cur = d_info;
    pool_fork(h, ns);
    cudaStream_t main = h->stream;
    try {
        for (size_t i = 0; i < diag.size(); ++i) {
            h->stream = h->pool[i % ns];
            zgetrf(h, diag[i]->nr, diag[i]->D, diag[i]->nr, diag[i]->piv, d_info);
        }
    } catch (...) {
        h->stream = main;
        pool_join(h, ns);
        h->d_info_cur = nullptr;
        cudaStreamSynchronize(h->stream);
        dfree(h, d_info);
        throw;
    }
    h->stream = main;
    pool_join(h, ns);
    h->d_info_cur = nullptr;
    int info = 0;
    HM_CUDA(cudaMemcpyAsync(&info, d_info, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    HM_CUDA(cudaStreamSynchronize(h->stream));
    dfree(h, d_info);
    if (info < 0) throw HmError{HM_ERR_TIMEOUT, "H-LU: a bounded grid barrier of the panel LU expired"};
    if (info) throw HmError{HM_ERR_SINGULAR, "H-LU: zero pivot in a diagonal leaf"};
    return true;
}

template <class Z>
void hlu_factor(hm_handle_s *h, BlockT<Z> *root, double tol)
{
    if (h->prm.independent && h->dense_lev == HM_MERGE_BODIES && hlu_factor_bodies(h, root)) return;
    double saved = h->cur_tol;
    h->cur_tol = tol;
    int *d_info = (int *)dalloc(h, sizeof(int));
    HM_CUDA(cudaMemsetAsync(d_info, 0, sizeof(int), h->stream));
    h->d_info_cur = d_info;
    try {
        hlu_rec(h, root, d_info);
        flush(h, root);
    } catch (...) {
        h->d_info_cur = nullptr;
        h->cur_tol = saved;
        cudaStreamSynchronize(h->stream);
        dfree(h, d_info);
        throw;
    }
    h->d_info_cur = nullptr;
    int info = 0;
    HM_CUDA(cudaMemcpyAsync(&info, d_info, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    HM_CUDA(cudaStreamSynchronize(h->stream));
    dfree(h, d_info);
    h->cur_tol = saved;
    if (info < 0) throw HmError{HM_ERR_TIMEOUT, "H-LU: a bounded grid barrier of the panel LU expired"};
    if (info) throw HmError{HM_ERR_SINGULAR, "H-LU: zero pivot in a diagonal leaf"};
}

template <class Ti, class To>
__global__ void k_convert(const Ti *__restrict__ x, To *__restrict__ y, size_t n)
{
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) cconv(x[i], y[i]);
}

template <class Ti, class To>
void convert_vec(hm_handle_s *h, const Ti *x, To *y, size_t n)
{
    if (n == 0) return;
    k_convert<Ti, To><<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(x, y, n);
    HM_CHECK_LAUNCH();
    count_launch(h);
}

template <class Z>
BlockT<Z> *clone_tree(hm_handle_s *h, Block *b, std::vector<BlockT<Z> *> &owned)
{
    BlockT<Z> *c = new BlockT<Z>();
    owned.push_back(c);
    c->type = b->type;
    c->r0 = b->r0;
    c->nr = b->nr;
    c->c0 = b->c0;
    c->nc = b->nc;
    c->t = b->t;
    c->s = b->s;
    c->k = b->k;
    c->zero = b->zero;
    c->leaf_id = b->leaf_id;
    if (b->type == B_DENSE) {
        c->D = zalloc<Z>(h, (size_t)b->nr * b->nc);
        convert_vec(h, b->D, c->D, (size_t)b->nr * b->nc);
    } else if (b->type == B_LR) {
        if (b->k) {
            c->U = zalloc<Z>(h, (size_t)b->nr * b->k);
            c->V = zalloc<Z>(h, (size_t)b->nc * b->k);
            convert_vec(h, b->U, c->U, (size_t)b->nr * b->k);
            convert_vec(h, b->V, c->V, (size_t)b->nc * b->k);
        }
    } else {
        for (int i = 0; i < 4; ++i) c->ch[i] = clone_tree<Z>(h, b->ch[i], owned);
    }
    return c;
}

// ---------------------------------------------------------------------------
// Complex64 copy of the FP64 tree with every hierarchical block on cluster level `level`
// or deeper stored as one dense block, written directly from the FP64 leaves below it by
// one batched launch: one CTA per 64 x 64 tile of a leaf (dense leaves converted, low-rank
// leaves expanded as U V^H in FP32 from the converted factors).
// ---------------------------------------------------------------------------
struct ExpandJob {
    const zc *D, *U, *V;  // FP64 leaf: dense (D) or low-rank (U, V, rank k)
    int nr, nc, k;
    int i0, j0;           // tile origin inside the leaf
    cf *dst;              // the leaf's top-left entry in the dense block
    int ld;
};

#define EX_T 256
#define EX_KC 32

__global__ void __launch_bounds__(EX_T) k_expand(const ExpandJob *__restrict__ jobs)
{
    const ExpandJob J = jobs[blockIdx.x];
    const int tid = threadIdx.x;
    const int mi = min(64, J.nr - J.i0), mj = min(64, J.nc - J.j0);
    if (!J.U) {
        for (int e = tid; e < 64 * 64; e += EX_T) {
            const int ii = e & 63, jj = e >> 6;
            if (ii < mi && jj < mj) {
                const zc v = J.D ? J.D[(size_t)(J.j0 + jj) * J.nr + J.i0 + ii] : zmake(0, 0);
                J.dst[(size_t)(J.j0 + jj) * J.ld + J.i0 + ii] = make_float2((float)v.x, (float)v.y);
            }
        }
        return;
    }
    __shared__ cf Us[EX_KC][64], Vs[EX_KC][65];
    const int tx = tid & 15, ty = tid >> 4;  // outputs (tx + 16 a, ty + 16 b)
    cf acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = make_float2(0.f, 0.f);
    for (int p0 = 0; p0 < J.k; p0 += EX_KC) {
        const int kc = min(EX_KC, J.k - p0);
        __syncthreads();
        for (int e = tid; e < EX_KC * 64; e += EX_T) {
            const int r = e & 63, q = e >> 6;
            zc u = zmake(0, 0), v = zmake(0, 0);
            if (q < kc && r < mi) u = J.U[(size_t)(p0 + q) * J.nr + J.i0 + r];
            if (q < kc && r < mj) v = J.V[(size_t)(p0 + q) * J.nc + J.j0 + r];
            Us[q][r] = make_float2((float)u.x, (float)u.y);
            Vs[q][r] = make_float2((float)v.x, (float)-v.y);  // conj(V)
        }
        __syncthreads();
        for (int q = 0; q < kc; ++q) {
            cf ua[4], vb[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) ua[a] = Us[q][tx + 16 * a];
#pragma unroll
            for (int b = 0; b < 4; ++b) vb[b] = Vs[q][ty + 16 * b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = zfma(ua[a], vb[b], acc[a][b]);
        }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int ii = tx + 16 * a, jj = ty + 16 * b;
            if (ii < mi && jj < mj) J.dst[(size_t)(J.j0 + jj) * J.ld + J.i0 + ii] = acc[a][b];
        }
}

static void expand_jobs(const Block *b, cf *D, int ld, int r0, int c0, std::vector<ExpandJob> &jobs)
{
    if (b->type == B_HIER) {
        for (int i = 0; i < 4; ++i) expand_jobs(b->ch[i], D, ld, r0, c0, jobs);
        return;
    }
    ExpandJob J;
    J.D = b->type == B_DENSE ? b->D : nullptr;
    J.U = b->type == B_LR && b->k ? b->U : nullptr;
    J.V = b->type == B_LR && b->k ? b->V : nullptr;
    J.nr = b->nr;
    J.nc = b->nc;
    J.k = b->type == B_LR ? b->k : 0;
    J.dst = D + (size_t)(b->c0 - c0) * ld + (b->r0 - r0);
    J.ld = ld;
    for (int i0 = 0; i0 < b->nr; i0 += 64)
        for (int j0 = 0; j0 < b->nc; j0 += 64) {
            J.i0 = i0;
            J.j0 = j0;
            jobs.push_back(J);
        }
}

static Block32 *clone_merged_rec(hm_handle_s *h, Block *b, int level, std::vector<Block32 *> &owned,
                                 std::vector<ExpandJob> &jobs)
{
    Block32 *c = new Block32();
    owned.push_back(c);
    c->type = b->type;
    c->r0 = b->r0;
    c->nr = b->nr;
    c->c0 = b->c0;
    c->nc = b->nc;
    c->t = b->t;
    c->s = b->s;
    c->k = b->k;
    c->zero = b->zero;
    c->leaf_id = b->leaf_id;
    if (b->type == B_HIER && merges_at(h, b, level)) {
        c->type = B_DENSE;
        c->k = 0;
        c->D = zalloc<cf>(h, (size_t)b->nr * b->nc);
        expand_jobs(b, c->D, b->nr, b->r0, b->c0, jobs);
    } else if (b->type == B_DENSE) {
        c->D = zalloc<cf>(h, (size_t)b->nr * b->nc);
        convert_vec(h, b->D, c->D, (size_t)b->nr * b->nc);
    } else if (b->type == B_LR) {
        if (b->k) {
            c->U = zalloc<cf>(h, (size_t)b->nr * b->k);
            c->V = zalloc<cf>(h, (size_t)b->nc * b->k);
            convert_vec(h, b->U, c->U, (size_t)b->nr * b->k);
            convert_vec(h, b->V, c->V, (size_t)b->nc * b->k);
        }
    } else {
        for (int i = 0; i < 4; ++i) c->ch[i] = clone_merged_rec(h, b->ch[i], level, owned, jobs);
    }
    return c;
}

Block32 *clone_tree_merged(hm_handle_s *h, Block *root, int level, std::vector<Block32 *> &owned)
{
    std::vector<ExpandJob> jobs;
    Block32 *r = clone_merged_rec(h, root, level, owned, jobs);
    // one launch per 2^20 tiles (grid limit headroom)
    const size_t CH = (size_t)1 << 20;
    for (size_t j0 = 0; j0 < jobs.size(); j0 += CH) {
        const size_t nj = std::min(CH, jobs.size() - j0);
        ExpandJob *d = (ExpandJob *)dalloc(h, sizeof(ExpandJob) * nj);
        HM_CUDA(cudaMemcpyAsync(d, jobs.data() + j0, sizeof(ExpandJob) * nj, cudaMemcpyHostToDevice, h->stream));
        k_expand<<<(unsigned)nj, EX_T, 0, h->stream>>>(d);
        HM_CHECK_LAUNCH();
        count_launch(h);
        dfree(h, d);
    }
    // the host job list must outlive the asynchronous copies
    HM_CUDA(cudaStreamSynchronize(h->stream));
    return r;
}

template <class Z>
void free_tree(hm_handle_s *h, std::vector<BlockT<Z> *> &owned)
{
    for (BlockT<Z> *b : owned) {
        if (b->D) dfree(h, b->D);
        if (b->U) dfree(h, b->U);
        if (b->V) dfree(h, b->V);
        if (b->piv) dfree(h, b->piv);
        for (Z *q : b->pu) dfree(h, q);
        for (Z *q : b->pv) dfree(h, q);
        delete b;
    }
    owned.clear();
}

// Write the content of block b (dense leaves copied, low-rank leaves as U V^H) into the
// dense column-major view D (ld) whose top-left entry is unknown (r0, c0).
template <class Z>
static void expand_into(hm_handle_s *h, BlockT<Z> *b, Z *D, int ld, int r0, int c0)
{
    Z *dst = D + (size_t)(b->c0 - c0) * ld + (b->r0 - r0);
    switch (b->type) {
    case B_DENSE:
        zcopy2d(h, MVT<Z>{dst, b->nr, b->nc, ld}, MVT<Z>{b->D, b->nr, b->nc, b->nr});
        break;
    case B_LR:
        if (b->k)
            zgemm<Z>(h, 'N', 'C', b->nr, b->nc, b->k, cmk<Z>(1, 0), b->U, b->nr, b->V, b->nc, cmk<Z>(0, 0), dst, ld);
        else
            zgemm<Z>(h, 'N', 'N', b->nr, b->nc, 0, cmk<Z>(0, 0), nullptr, 1, nullptr, 1, cmk<Z>(0, 0), dst, ld);
        break;
    case B_HIER:
        for (int i = 0; i < 4; ++i) expand_into(h, b->ch[i], D, ld, r0, c0);
        break;
    }
}

template <class Z>
static void release_subtree(hm_handle_s *h, BlockT<Z> *b)
{
    if (b->type == B_HIER)
        for (int i = 0; i < 4; ++i) release_subtree(h, b->ch[i]);
    if (b->D) dfree(h, b->D);
    if (b->U) dfree(h, b->U);
    if (b->V) dfree(h, b->V);
    b->D = b->U = b->V = nullptr;
    b->k = 0;
}

// Coarsening of a block tree for its H-LU: every hierarchical block whose clusters lie on
// cluster level `level` or deeper becomes one dense block holding the same entries
// (exact: dense leaves are copied and low-rank leaves expanded).  Blocks on coarser levels
// keep their format, so every block row of the dense level holds dense blocks or whole
// low-rank blocks of that level and above, and the partial pivoting of a dense diagonal
// block stays within its own rows.
// Whether the hierarchical block b becomes one dense block at the given merge level:
// clusters on that level or deeper, or (HM_MERGE_BODIES) the diagonal block of one body.
template <class Z>
bool merges_at(const hm_handle_s *h, const BlockT<Z> *b, int level)
{
    if (level == HM_MERGE_BODIES) return b->t == b->s && h->clusters[b->t].body_root;
    return h->clusters[b->t].level >= level;
}

template <class Z>
void coarsen_tree(hm_handle_s *h, BlockT<Z> *b, int level)
{
    if (b->type != B_HIER) return;
    if (merges_at(h, b, level)) {
        Z *D = (Z *)dalloc(h, sizeof(Z) * (size_t)b->nr * b->nc);
        for (int i = 0; i < 4; ++i) expand_into(h, b->ch[i], D, b->nr, b->r0, b->c0);
        for (int i = 0; i < 4; ++i) {
            release_subtree(h, b->ch[i]);
            b->ch[i] = nullptr;
        }
        b->type = B_DENSE;
        b->D = D;
        return;
    }
    for (int i = 0; i < 4; ++i) coarsen_tree(h, b->ch[i], level);
}

template <class Z>
static double subtree_words(const BlockT<Z> *b)
{
    if (b->type == B_DENSE) return (double)b->nr * b->nc;
    if (b->type == B_LR) return (double)b->k * (b->nr + b->nc);
    double s = 0;
    for (int i = 0; i < 4; ++i) s += subtree_words(b->ch[i]);
    return s;
}

template <class Z>
static void level_words(hm_handle_s *h, const BlockT<Z> *b, std::vector<double> &hw, std::vector<double> &dw)
{
    if (b->type == B_LR) return;  // low-rank blocks keep their format at every level
    const int L = h->clusters[b->t].level;
    if ((int)hw.size() <= L) {
        hw.resize(L + 1, 0.0);
        dw.resize(L + 1, 0.0);
    }
    hw[L] += subtree_words(b);
    dw[L] += (double)b->nr * b->nc;
    if (b->type == B_HIER)
        for (int i = 0; i < 4; ++i) level_words(h, b->ch[i], hw, dw);
}

// The coarsest cluster level whose clusters hold at most `cap` unknowns and whose
// non-low-rank blocks (the ones a merge turns dense) store, in H-format, at least `theta`
// of their dense size: merging there costs little memory and removes the formatted
// arithmetic below it.  -1 when no level qualifies.
template <class Z>
int dense_level_by_storage(hm_handle_s *h, BlockT<Z> *root, int cap, double theta)
{
    std::vector<double> hw, dw;
    level_words(h, root, hw, dw);
    for (int L = 0; L < (int)hw.size(); ++L) {
        if (h->dof * ((h->nnode + (1 << L) - 1) >> L) > cap) continue;
        if (dw[L] > 0 && hw[L] >= theta * dw[L]) return L;
    }
    return -1;
}

// The coarsest cluster level at which merging every non-low-rank block into one dense block
// keeps the tree's storage within budget_words complex words (-1: none).
template <class Z>
int dense_level_by_memory(hm_handle_s *h, BlockT<Z> *root, double budget_words)
{
    std::vector<double> hw, dw;
    level_words(h, root, hw, dw);
    const double total = subtree_words(root);
    for (int L = 0; L < (int)hw.size(); ++L)
        if (dw[L] > 0 && total - hw[L] + dw[L] <= budget_words) return L;
    return -1;
}

#define HM_INST_HLU(Z)                                                                             \
    template void hlu_factor<Z>(hm_handle_s *, BlockT<Z> *, double);                               \
    template void hmatvec<Z>(hm_handle_s *, BlockT<Z> *, MVT<Z>, MVT<Z>, Z, bool);                 \
    template BlockT<Z> *clone_tree<Z>(hm_handle_s *, Block *, std::vector<BlockT<Z> *> &);         \
    template void free_tree<Z>(hm_handle_s *, std::vector<BlockT<Z> *> &);                         \
    template void coarsen_tree<Z>(hm_handle_s *, BlockT<Z> *, int);                                \
    template bool merges_at<Z>(const hm_handle_s *, const BlockT<Z> *, int);                       \
    template int dense_level_by_storage<Z>(hm_handle_s *, BlockT<Z> *, int, double);              \
    template int dense_level_by_memory<Z>(hm_handle_s *, BlockT<Z> *, double);
HM_INST_HLU(zc)
HM_INST_HLU(cf)
template void convert_vec<zc, cf>(hm_handle_s *, const zc *, cf *, size_t);
template void convert_vec<cf, zc>(hm_handle_s *, const cf *, zc *, size_t);
