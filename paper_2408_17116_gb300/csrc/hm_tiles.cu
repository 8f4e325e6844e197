// Block-row form of the H-matrix product and of the H-forward/back substitution
// (Sec. III.A, Eqs. 24-28) on the leaf partition of the block cluster tree.
//
// The diagonal blocks of the tree are dense leaves (c, c) of the leaf clusters c; they
// partition the unknowns into row tiles.  Every other leaf (t, s) lies entirely left or
// right of the diagonal and covers whole tiles of its row cluster t.  Restricted to the
// rows of tile i, a dense leaf gives D[rows_i, :] and a low-rank leaf U[rows_i, :] V^H.
//
//   product:    y_i += sum over all leaves in block row i of (leaf rows_i) x_cols
//   forward:    y_i  = L_ii^-1 P_i (b_i - sum_{leaves left of the diagonal} (leaf rows_i) y_cols)
//   backward:   x_i  = U_ii^-1 (y_i - sum_{leaves right of the diagonal} (leaf rows_i) x_cols)
//
// This is the same arithmetic as the recursive substitution of the H-LU factors: the
// recursion subtracts, level by level, L21 X1 from X2 before the permutation of a
// diagonal leaf is applied to its own rows, so every tile receives exactly the sum of its
// block row's left leaves times the final values of their columns.  Here each step of a
// sweep has one CTA per chunk of the tile's pieces writing a partial sum; the partials are
// then subtracted in a fixed order, the pivots applied and the result multiplied by
// the explicit inverse of the diagonal factor (computed once after the factorisation):
// a gather of the subtracted right-hand side by the block's pivot permutation, then a
// product with the inverse over CTAs of 256 rows (three launches per step).
// The product is one launch over every chunk of every tile plus one reduction launch.
// Summation order is fixed, so results are deterministic.
//
// A dense diagonal block larger than a row tile (a merged block of the factor) is split
// into a group of row tiles.  Its pivots permute rows across the whole block, so the
// forward sweep of a group first subtracts the leaves left of the block from every tile of
// the group, then applies the block's permutation to all of its rows, then substitutes
// tile by tile with the block's own L_ij (j < i) as further left pieces.  The backward
// sweep has no permutation: the block's U_ij (j > i) are right pieces like any other leaf.
#include <algorithm>
#include <cstring>

#include "hm_internal.h"

#define TL_T 256   // threads per CTA
#define TL_NRB 4   // right-hand sides per pass
#define TL_KC 128  // rank columns per pass of a low-rank piece
#define TL_JC 256  // columns of a dense piece staged per pass
// largest row tile (a diagonal block of the tree): the tile's accumulators of
// k_tile_partial live in shared memory
template <class C> struct TileRows;
template <> struct TileRows<cf> { static constexpr int value = 4096; };
template <> struct TileRows<zc> { static constexpr int value = 2048; };

template <class C>
struct TPiece {
    const C *A;     // dense: rows [rofs, rofs + rows) of D; low-rank: the same rows of U (ld = leaf rows)
    const C *V;     // low-rank: V (ncol x k, ld = ncol); dense: null
    int ld;         // leading dimension of A
    int c0, ncol;   // columns of the leaf (tree order)
    int k;          // rank (low-rank), 0 for dense
    int toff;       // product plan: first rank column of the leaf's V^H X in the per-call buffer
                    // (computed once per leaf by k_leaf_vhx); -1: the CTA forms V^H X itself
};

struct TChunk {
    int p0, p1;   // pieces [p0, p1), all of one tile
    int rows;     // rows of the tile
    int slot;     // partial-sum slot
};

// acc[r][c] (shared, rows x nrb) += A[r, :] Z[:, c] for A (rows x n, ld) and Z staged in
// shared memory (zs[j * TL_NRB + c], j < n).  Threads split the columns into G groups
// that add their partial sums in group order (deterministic).
template <class C, bool CONJ_Z>
__device__ __forceinline__ void tile_gemv(const C *__restrict__ A, int ld, int rows, int n, const C *zs, int nrb,
                                          C *acc)
{
    const int tid = threadIdx.x;
    if (rows > TL_T) {
        // tiles taller than the CTA: each thread owns rows tid, tid + TL_T, ...; four columns
        // per step, their loads issued together (memory-level parallelism)
        for (int r = tid; r < rows; r += TL_T) {
            C a[TL_NRB];
#pragma unroll
            for (int c = 0; c < TL_NRB; ++c) a[c] = cmk<C>(0, 0);
            int j = 0;
            for (; j + 4 <= n; j += 4) {
                C v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) v[u] = A[(size_t)(j + u) * ld + r];
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int c = 0; c < TL_NRB; ++c)
                        if (c < nrb) a[c] = zfma(v[u], zs[(j + u) * TL_NRB + c], a[c]);
            }
            for (; j < n; ++j) {
                C v = A[(size_t)j * ld + r];
#pragma unroll
                for (int c = 0; c < TL_NRB; ++c)
                    if (c < nrb) a[c] = zfma(v, zs[j * TL_NRB + c], a[c]);
            }
#pragma unroll
            for (int c = 0; c < TL_NRB; ++c)
                if (c < nrb) acc[r * TL_NRB + c] = zadd(acc[r * TL_NRB + c], a[c]);
        }
        __syncthreads();
        return;
    }
    const int G = max(1, TL_T / rows);
    const int r = tid % rows, g = tid / rows;
    C a[TL_NRB];
#pragma unroll
    for (int c = 0; c < TL_NRB; ++c) a[c] = cmk<C>(0, 0);
    if (g < G && tid < G * rows) {
        int j = g;
        for (; j + 3 * G < n; j += 4 * G) {
            C v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = A[(size_t)(j + u * G) * ld + r];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int c = 0; c < TL_NRB; ++c)
                    if (c < nrb) a[c] = zfma(v[u], zs[(j + u * G) * TL_NRB + c], a[c]);
        }
        for (; j < n; j += G) {
            C v = A[(size_t)j * ld + r];
#pragma unroll
            for (int c = 0; c < TL_NRB; ++c)
                if (c < nrb) a[c] = zfma(v, zs[j * TL_NRB + c], a[c]);
        }
    }
    for (int gg = 0; gg < G; ++gg) {
        if (g == gg && tid < G * rows) {
#pragma unroll
            for (int c = 0; c < TL_NRB; ++c)
                if (c < nrb) acc[r * TL_NRB + c] = zadd(acc[r * TL_NRB + c], a[c]);
        }
        __syncthreads();
    }
}

// One CTA per chunk: part[slot][c][i] = sum over the chunk's pieces of (piece rows) X(:, c).
// X: tree-ordered columns, ld = ldx.  part: [slots][nrhs][rmax].
template <class C>
__global__ void __launch_bounds__(TL_T) k_tile_partial(const TPiece<C> *__restrict__ pieces,
                                                         const TChunk *__restrict__ chunks, const C *__restrict__ X,
                                                         int ldx, int nrhs, C *__restrict__ part, int rmax,
                                                         const C *__restrict__ tbuf)
{
    extern __shared__ __align__(16) unsigned char tp_raw[];
    C *acc = (C *)tp_raw;  // [rmax][TL_NRB]
    __shared__ C zs[(TL_JC > TL_KC ? TL_JC : TL_KC) * TL_NRB];
    const TChunk ch = chunks[blockIdx.x];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int rows = ch.rows;
    for (int cb = 0; cb < nrhs; cb += TL_NRB) {
        const int nrb = min(TL_NRB, nrhs - cb);
        for (int e = tid; e < rows * TL_NRB; e += TL_T) acc[e] = cmk<C>(0, 0);
        __syncthreads();
        for (int p = ch.p0; p < ch.p1; ++p) {
            const TPiece<C> P = pieces[p];
            if (P.k == 0) {
                for (int j0 = 0; j0 < P.ncol; j0 += TL_JC) {
                    const int n = min(TL_JC, P.ncol - j0);
                    for (int e = tid; e < n * TL_NRB; e += TL_T) {
                        int j = e / TL_NRB, c = e - j * TL_NRB;
                        zs[e] = c < nrb ? X[(size_t)(cb + c) * ldx + P.c0 + j0 + j] : cmk<C>(0, 0);
                    }
                    __syncthreads();
                    tile_gemv<C, false>(P.A + (size_t)j0 * P.ld, P.ld, rows, n, zs, nrb, acc);
                }
            } else {
                for (int k0 = 0; k0 < P.k; k0 += TL_KC) {
                    const int kc = min(TL_KC, P.k - k0);
                    if (P.toff >= 0) {
                        // V^H X of this leaf, formed once for all its row tiles
                        for (int e = tid; e < kc * TL_NRB; e += TL_T) {
                            const int kk = e / TL_NRB, c = e - kk * TL_NRB;
                            zs[e] = c < nrb ? tbuf[(size_t)(P.toff + k0 + kk) * nrhs + cb + c] : cmk<C>(0, 0);
                        }
                        __syncthreads();
                        tile_gemv<C, false>(P.A + (size_t)k0 * P.ld, P.ld, rows, kc, zs, nrb, acc);
                        continue;
                    }
                    // t[kk][c] = sum_j conj(V[j, k0 + kk]) X[c0 + j, cb + c]: one warp per column kk
                    for (int kk = warp; kk < kc; kk += TL_T / 32) {
                        const C *v = P.V + (size_t)(k0 + kk) * P.ncol;
                        C s[TL_NRB];
#pragma unroll
                        for (int c = 0; c < TL_NRB; ++c) s[c] = cmk<C>(0, 0);
                        for (int j = lane; j < P.ncol; j += 32) {
                            C vv = v[j];
#pragma unroll
                            for (int c = 0; c < TL_NRB; ++c)
                                if (c < nrb) s[c] = zfmac(vv, X[(size_t)(cb + c) * ldx + P.c0 + j], s[c]);
                        }
#pragma unroll
                        for (int c = 0; c < TL_NRB; ++c) {
                            for (int o = 16; o > 0; o >>= 1) {
                                s[c].x += __shfl_down_sync(0xffffffff, s[c].x, o);
                                s[c].y += __shfl_down_sync(0xffffffff, s[c].y, o);
                            }
                        }
                        if (lane == 0) {
#pragma unroll
                            for (int c = 0; c < TL_NRB; ++c) zs[kk * TL_NRB + c] = c < nrb ? s[c] : cmk<C>(0, 0);
                        }
                    }
                    __syncthreads();
                    tile_gemv<C, false>(P.A + (size_t)k0 * P.ld, P.ld, rows, kc, zs, nrb, acc);
                }
            }
        }
        C *out = part + (size_t)ch.slot * nrhs * rmax;
        for (int e = tid; e < rows * nrb; e += TL_T) {
            int r = e / nrb, c = e - r * nrb;
            out[(size_t)(cb + c) * rmax + r] = acc[r * TL_NRB + c];
        }
        __syncthreads();
    }
}

// V^H X of every low-rank leaf of a product plan, once per leaf: one warp per (leaf, rank
// column) job; t[(toff + kk) nrhs + c] = sum_j conj(V[j, kk]) X[c0 + j, c].
struct TLeaf {
    int c0, ncol, toff;
};
template <class C>
__global__ void __launch_bounds__(TL_T) k_leaf_vhx(const TLeaf *__restrict__ leaves, const int2 *__restrict__ jobs,
                                                     const C *const *__restrict__ vptr, int njobs,
                                                     const C *__restrict__ X, int ldx, int nrhs, C *__restrict__ t)
{
    const int lane = threadIdx.x & 31;
    const int job = blockIdx.x * (TL_T / 32) + (threadIdx.x >> 5);
    if (job >= njobs) return;
    const int2 jb = jobs[job];
    const TLeaf L = leaves[jb.x];
    const C *v = vptr[jb.x] + (size_t)jb.y * L.ncol;
    for (int cb = 0; cb < nrhs; cb += TL_NRB) {
        const int nrb = min(TL_NRB, nrhs - cb);
        C s[TL_NRB];
#pragma unroll
        for (int c = 0; c < TL_NRB; ++c) s[c] = cmk<C>(0, 0);
        for (int j = lane; j < L.ncol; j += 32) {
            const C vv = v[j];
#pragma unroll
            for (int c = 0; c < TL_NRB; ++c)
                if (c < nrb) s[c] = zfmac(vv, X[(size_t)(cb + c) * ldx + L.c0 + j], s[c]);
        }
#pragma unroll
        for (int c = 0; c < TL_NRB; ++c)
            for (int o = 16; o > 0; o >>= 1) {
                s[c].x += __shfl_down_sync(0xffffffffu, s[c].x, o);
                s[c].y += __shfl_down_sync(0xffffffffu, s[c].y, o);
            }
        if (lane == 0)
            for (int c = 0; c < nrb; ++c) t[(size_t)(L.toff + jb.y) * nrhs + cb + c] = s[c];
    }
}

// Product finish: one CTA per tile, Y[r0 + i, c] += alpha sum_{s in [s0, s1)} part[s][c][i].
template <class C>
__global__ void k_tile_reduce(const int *__restrict__ tr0, const int *__restrict__ trows,
                              const int *__restrict__ ts0, const int *__restrict__ ts1, const C *__restrict__ part,
                              int nrhs, int rmax, C alpha, C *Y, int ldy)
{
    const int t = blockIdx.x, r0 = tr0[t], rows = trows[t], s0 = ts0[t], s1 = ts1[t];
    for (int e = threadIdx.x; e < rows * nrhs; e += blockDim.x) {
        int c = e / rows, i = e - c * rows;
        C s = cmk<C>(0, 0);
        for (int q = s0; q < s1; ++q) s = zadd(s, part[((size_t)q * nrhs + c) * rmax + i]);
        C &y = Y[(size_t)c * ldy + r0 + i];
        y = zfma(alpha, s, y);
    }
}

// Sweep step, part 1 (CTAs over the tile's rows): z[j][c] = X[r0 + g(j), c] - sum_s
// part[s][c][g(j)] in a fixed order, g = the diagonal block's row permutation (the pivots
// applied in order; the identity for the backward sweep).  z: [nrhs][rows].
template <class C>
__global__ void k_tile_prep(int r0, int rows, int nslots, const C *__restrict__ part, int nrhs, int rmax,
                            const int *__restrict__ gperm, const C *__restrict__ X, int ldx, C *__restrict__ z)
{
    const size_t n = (size_t)rows * nrhs;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(e / rows), j = (int)(e - (size_t)c * rows);
        const int g = gperm ? gperm[j] : j;
        C s = X[(size_t)c * ldx + r0 + g];
        for (int q = 0; q < nslots; ++q) s = zsub(s, part[((size_t)q * nrhs + c) * rmax + g]);
        z[(size_t)c * rows + j] = s;
    }
}

// X[r0 + j, c] -= sum_s part[s][c][j] (fixed order): the leaves left of a grouped block.
template <class C>
__global__ void k_tile_sub(int r0, int rows, int nslots, const C *__restrict__ part, int nrhs, int rmax, C *X,
                           int ldx)
{
    const size_t n = (size_t)rows * nrhs;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(e / rows), j = (int)(e - (size_t)c * rows);
        C s = X[(size_t)c * ldx + r0 + j];
        for (int q = 0; q < nslots; ++q) s = zsub(s, part[((size_t)q * nrhs + c) * rmax + j]);
        X[(size_t)c * ldx + r0 + j] = s;
    }
}

// X[r0 + j, c] = z[c][j]
template <class C>
__global__ void k_tile_put(int r0, int rows, int nrhs, const C *__restrict__ z, C *X, int ldx)
{
    const size_t n = (size_t)rows * nrhs;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(e / rows), j = (int)(e - (size_t)c * rows);
        X[(size_t)c * ldx + r0 + j] = z[(size_t)c * rows + j];
    }
}

// Sweep step, part 2: X[r0 + i, c] = sum_j Minv[i][j] z[j][c], Minv the explicit inverse of
// the diagonal block's triangular factor (column-major).  A CTA owns 32 rows; its 8 warps
// take every 8th column (lane = row, so each column's 32 entries load as one 256-byte
// transaction) and their partial sums are added in warp order (deterministic).
#define TM_R 32
#define TM_G (TL_T / TM_R)
template <class C>
__global__ void __launch_bounds__(TL_T) k_tile_mul(int r0, int rows, int nrhs, const C *__restrict__ Minv,
                                                     const C *__restrict__ z, C *X, int ldx)
{
    __shared__ C zs[TL_T * TL_NRB];
    __shared__ C red[TM_G][TM_R][TL_NRB];
    const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
    const int i = blockIdx.x * TM_R + lane;
    for (int cb = 0; cb < nrhs; cb += TL_NRB) {
        const int nrb = min(TL_NRB, nrhs - cb);
        C a[TL_NRB];
#pragma unroll
        for (int c = 0; c < TL_NRB; ++c) a[c] = cmk<C>(0, 0);
        for (int j0 = 0; j0 < rows; j0 += TL_T) {
            const int nj = min(TL_T, rows - j0);
            __syncthreads();
            for (int e = threadIdx.x; e < nj * TL_NRB; e += TL_T) {
                int j = e / TL_NRB, c = e - j * TL_NRB;
                zs[e] = c < nrb ? z[(size_t)(cb + c) * rows + j0 + j] : cmk<C>(0, 0);
            }
            __syncthreads();
            if (i < rows) {
                int j = g;
                for (; j + 3 * TM_G < nj; j += 4 * TM_G) {
                    C mv[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) mv[u] = Minv[(size_t)(j0 + j + u * TM_G) * rows + i];
#pragma unroll
                    for (int u = 0; u < 4; ++u)
#pragma unroll
                        for (int c = 0; c < TL_NRB; ++c) a[c] = zfma(mv[u], zs[(j + u * TM_G) * TL_NRB + c], a[c]);
                }
                for (; j < nj; j += TM_G) {
                    const C m = Minv[(size_t)(j0 + j) * rows + i];
#pragma unroll
                    for (int c = 0; c < TL_NRB; ++c) a[c] = zfma(m, zs[j * TL_NRB + c], a[c]);
                }
            }
        }
#pragma unroll
        for (int c = 0; c < TL_NRB; ++c) red[g][lane][c] = a[c];
        __syncthreads();
        if (g == 0 && i < rows)
            for (int c = 0; c < nrb; ++c) {
                C s = red[0][lane][c];
                for (int q = 1; q < TM_G; ++q) s = zadd(s, red[q][lane][c]);
                X[(size_t)(cb + c) * ldx + r0 + i] = s;
            }
        __syncthreads();
    }
}

// Dynamic shared memory of k_tile_partial (the accumulators of one tile); raises the
// kernel's limit when a tile needs more than the default 48 KB.
template <class C>
static size_t partial_smem(int rmax)
{
    const size_t bytes = sizeof(C) * (size_t)std::max(rmax, 1) * TL_NRB;
    const size_t stat = sizeof(C) * (TL_JC > TL_KC ? TL_JC : TL_KC) * TL_NRB;
    if (bytes + stat > 48 * 1024)
        HM_CUDA(cudaFuncSetAttribute(k_tile_partial<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    return bytes;
}

template <class C>
struct TileOp {
    int N = 0, ntile = 0, rmax = 0;
    std::vector<int> r0, rows;              // tiles
    // product over all leaves
    TPiece<C> *d_pa = nullptr;
    TChunk *d_ca = nullptr;
    int nca = 0;
    int *d_tr0 = nullptr, *d_trows = nullptr, *d_ts0 = nullptr, *d_ts1 = nullptr;
    // sweeps of a factored tree
    bool factored = false;
    TPiece<C> *d_pl = nullptr, *d_pu = nullptr;
    TChunk *d_cl = nullptr, *d_cu = nullptr;
    std::vector<int> cl0, cl1, cu0, cu1;  // chunk ranges per tile
    int maxchunks = 0;
    C *d_inv = nullptr;                   // per tile: L^-1 then U^-1 (rows x rows each)
    std::vector<size_t> inv_off;
    std::vector<const int *> gperm;       // per tile: row permutation of its pivots (device; null in a group)
    // groups of row tiles splitting one dense diagonal block larger than a tile
    std::vector<int> grp0, grpn;          // per tile: first tile of its group, tiles in the group
    std::vector<const int *> ggperm;      // per tile: the group's row permutation (set on its first tile)
    TPiece<C> *d_po = nullptr;            // per grouped tile: leaves left of the whole block
    TChunk *d_co = nullptr;
    std::vector<int> co0, co1;
    int maxgrow = 0;                      // rows of the largest group
    // product plan: V^H X once per low-rank leaf
    TLeaf *d_tl = nullptr;
    int2 *d_tjobs = nullptr;
    const C **d_tv = nullptr;
    int ntjobs = 0;                       // = total rank of the low-rank leaves
    std::vector<void *> owned;
};

namespace {

template <class C>
void collect(BlockT<C> *b, std::vector<BlockT<C> *> &out)
{
    if (b->type == B_HIER) {
        for (int i = 0; i < 4; ++i) collect(b->ch[i], out);
    } else {
        out.push_back(b);
    }
}

template <class C>
double piece_cost(const TPiece<C> &p, int rows)
{
    return p.k ? (double)p.k * (rows + p.ncol) : (double)rows * p.ncol;
}

// Chunks of one tile's pieces, each of at most `target` cost (at least one piece).
template <class C>
void make_chunks(const std::vector<TPiece<C>> &pcs, int p0, int p1, int rows, double target,
                 std::vector<TChunk> &out, int &slot)
{
    int s = p0;
    double acc = 0;
    for (int p = p0; p < p1; ++p) {
        double c = piece_cost(pcs[p], rows);
        if (p > s && acc + c > target) {
            out.push_back(TChunk{s, p, rows, slot++});
            s = p;
            acc = 0;
        }
        acc += c;
    }
    if (p1 > s) out.push_back(TChunk{s, p1, rows, slot++});
}

// Dense pieces of more than TL_SPLIT entries are cut into column blocks so that a large
// dense leaf (a merged block of the factor) is streamed by many CTAs, not one.
#define TL_SPLIT (1 << 20)

template <class C>
void push_piece(std::vector<TPiece<C>> &v, const TPiece<C> &p, int rows)
{
    if (p.k != 0 || (double)rows * p.ncol <= TL_SPLIT) {
        v.push_back(p);
        return;
    }
    const int nb = (int)(((double)rows * p.ncol + TL_SPLIT - 1) / TL_SPLIT);
    for (int q = 0; q < nb; ++q) {
        const int j0 = (int)((long long)q * p.ncol / nb), j1 = (int)((long long)(q + 1) * p.ncol / nb);
        if (j1 <= j0) continue;
        TPiece<C> s = p;
        s.A = p.A + (size_t)j0 * p.ld;
        s.c0 = p.c0 + j0;
        s.ncol = j1 - j0;
        v.push_back(s);
    }
}

template <class T>
T *upload(hm_handle_s *h, const std::vector<T> &v, std::vector<void *> &owned)
{
    T *d = (T *)dalloc(h, sizeof(T) * std::max<size_t>(v.size(), 1));
    if (!v.empty()) HM_CUDA(cudaMemcpyAsync(d, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, h->stream));
    owned.push_back(d);
    return d;
}

}  // namespace

template <class C>
TileOp<C> *tile_build(hm_handle_s *h, BlockT<C> *root, bool factored)
{
    TileOp<C> *T = new TileOp<C>();
    PhaseScope ps(h, PH_TILE_BUILD);
    try {
        std::vector<BlockT<C> *> leaves;
        collect(root, leaves);
        std::vector<BlockT<C> *> diag;
        for (BlockT<C> *b : leaves)
            if (b->r0 == b->c0 && b->nr == b->nc && b->type == B_DENSE) diag.push_back(b);
        std::sort(diag.begin(), diag.end(), [](BlockT<C> *a, BlockT<C> *b) { return a->r0 < b->r0; });
        // row tiles: one per diagonal leaf, or a group of nearly equal tiles when the leaf has
        // more rows than a tile holds
        std::vector<BlockT<C> *> tdiag;  // per tile: its diagonal leaf
        int pos = 0;
        for (BlockT<C> *d : diag) {
            if (d->r0 != pos) throw HmError{HM_ERR_STATE, "tile plan: diagonal leaves do not partition the unknowns"};
            const int nsub = (d->nr + TileRows<C>::value - 1) / TileRows<C>::value;
            const int g0 = (int)T->r0.size();
            for (int q = 0; q < nsub; ++q) {
                const int o0 = (int)((long long)q * d->nr / nsub), o1 = (int)((long long)(q + 1) * d->nr / nsub);
                T->r0.push_back(d->r0 + o0);
                T->rows.push_back(o1 - o0);
                T->rmax = std::max(T->rmax, o1 - o0);
                T->grp0.push_back(g0);
                T->grpn.push_back(nsub);
                tdiag.push_back(d);
            }
            if (nsub > 1) T->maxgrow = std::max(T->maxgrow, d->nr);
            pos += d->nr;
        }
        T->N = pos;
        T->ntile = (int)T->r0.size();
        auto tile_of = [&](int r) {
            int i = (int)(std::upper_bound(T->r0.begin(), T->r0.end(), r) - T->r0.begin()) - 1;
            return i;
        };
        // pieces per tile: all / left of the diagonal (outside the tile's own diagonal leaf, and
        // inside it for a group) / right of the diagonal
        std::vector<std::vector<TPiece<C>>> all(T->ntile), left(T->ntile), lin(T->ntile), right(T->ntile);
        std::vector<TLeaf> tl;
        std::vector<int2> tjobs;
        std::vector<const C *> tv;
        for (BlockT<C> *b : leaves) {
            if (b->type == B_LR && b->k == 0) continue;
            int toff = -1;
            if (b->type == B_LR) {
                toff = (int)tjobs.size();
                for (int kk = 0; kk < b->k; ++kk) tjobs.push_back(make_int2((int)tl.size(), kk));
                tl.push_back(TLeaf{b->c0, b->nc, toff});
                tv.push_back(b->V);
            }
            const bool isdiag = b->r0 == b->c0 && b->type == B_DENSE && b->nr == b->nc;
            for (int i = tile_of(b->r0); i < T->ntile && T->r0[i] < b->r0 + b->nr; ++i) {
                if (T->r0[i] < b->r0 || T->r0[i] + T->rows[i] > b->r0 + b->nr)
                    throw HmError{HM_ERR_STATE, "tile plan: a leaf does not cover whole tiles"};
                const int rofs = T->r0[i] - b->r0;
                TPiece<C> p;
                p.ld = b->nr;
                p.c0 = b->c0;
                p.ncol = b->nc;
                p.toff = -1;
                if (b->type == B_DENSE) {
                    p.A = b->D + rofs;
                    p.V = nullptr;
                    p.k = 0;
                } else {
                    p.A = b->U + rofs;
                    p.V = b->V;
                    p.k = b->k;
                }
                {
                    TPiece<C> pa = p;
                    pa.toff = toff;  // the product plan reads V^H X from the per-call buffer
                    push_piece(all[i], pa, T->rows[i]);
                }
                if (isdiag) {
                    // a grouped diagonal leaf: its off-diagonal tile blocks L_ij (j < i), U_ij (j > i)
                    for (int j = T->grp0[i]; j < T->grp0[i] + T->grpn[i]; ++j) {
                        if (j == i) continue;
                        TPiece<C> q;
                        q.A = b->D + rofs + (size_t)(T->r0[j] - b->r0) * b->nr;
                        q.V = nullptr;
                        q.ld = b->nr;
                        q.c0 = T->r0[j];
                        q.ncol = T->rows[j];
                        q.k = 0;
                        q.toff = -1;
                        push_piece(j < i ? lin[i] : right[i], q, T->rows[i]);
                    }
                    continue;
                }
                if (b->c0 + b->nc <= T->r0[i])
                    push_piece(left[i], p, T->rows[i]);
                else if (b->c0 >= T->r0[i] + T->rows[i])
                    push_piece(right[i], p, T->rows[i]);
                else
                    throw HmError{HM_ERR_STATE, "tile plan: an off-diagonal leaf crosses the diagonal"};
            }
        }
        // product plan: chunks sized so that the launch has a few CTAs per SM
        {
            std::vector<TPiece<C>> pcs;
            std::vector<TChunk> chs;
            std::vector<int> s0(T->ntile), s1(T->ntile);
            double tot = 0;
            for (int i = 0; i < T->ntile; ++i)
                for (auto &p : all[i]) tot += piece_cost(p, T->rows[i]);
            const double target = std::max(tot / (4.0 * 152.0), 1.0);
            int slot = 0;
            for (int i = 0; i < T->ntile; ++i) {
                int p0 = (int)pcs.size();
                pcs.insert(pcs.end(), all[i].begin(), all[i].end());
                s0[i] = slot;
                make_chunks(pcs, p0, (int)pcs.size(), T->rows[i], target, chs, slot);
                s1[i] = slot;
            }
            T->nca = (int)chs.size();
            T->ntjobs = (int)tjobs.size();
            T->d_tl = upload(h, tl, T->owned);
            T->d_tjobs = upload(h, tjobs, T->owned);
            T->d_tv = upload(h, tv, T->owned);
            T->d_pa = upload(h, pcs, T->owned);
            T->d_ca = upload(h, chs, T->owned);
            T->d_tr0 = upload(h, T->r0, T->owned);
            T->d_trows = upload(h, T->rows, T->owned);
            T->d_ts0 = upload(h, s0, T->owned);
            T->d_ts1 = upload(h, s1, T->owned);
        }
        if (factored) {
            T->factored = true;
            std::vector<TPiece<C>> pl, pu, po;
            std::vector<TChunk> cl, cu, co;
            T->cl0.resize(T->ntile);
            T->cl1.resize(T->ntile);
            T->cu0.resize(T->ntile);
            T->cu1.resize(T->ntile);
            T->co0.resize(T->ntile);
            T->co1.resize(T->ntile);
            for (int i = 0; i < T->ntile; ++i) {
                // about 2 CTAs per SM per step; a grouped tile substitutes with its block's L_ij
                // and subtracts the outside leaves in a separate pass
                const bool grouped = T->grpn[i] > 1;
                const std::vector<TPiece<C>> &L = grouped ? lin[i] : left[i];
                double tl = 0, tu = 0, to = 0;
                for (auto &p : L) tl += piece_cost(p, T->rows[i]);
                for (auto &p : right[i]) tu += piece_cost(p, T->rows[i]);
                int sl = 0, su = 0, so = 0;
                int p0 = (int)pl.size();
                pl.insert(pl.end(), L.begin(), L.end());
                T->cl0[i] = (int)cl.size();
                make_chunks(pl, p0, (int)pl.size(), T->rows[i], std::max(tl / 304.0, 1.0), cl, sl);
                T->cl1[i] = (int)cl.size();
                p0 = (int)pu.size();
                pu.insert(pu.end(), right[i].begin(), right[i].end());
                T->cu0[i] = (int)cu.size();
                make_chunks(pu, p0, (int)pu.size(), T->rows[i], std::max(tu / 304.0, 1.0), cu, su);
                T->cu1[i] = (int)cu.size();
                T->co0[i] = T->co1[i] = (int)co.size();
                if (grouped) {
                    for (auto &p : left[i]) to += piece_cost(p, T->rows[i]);
                    p0 = (int)po.size();
                    po.insert(po.end(), left[i].begin(), left[i].end());
                    make_chunks(po, p0, (int)po.size(), T->rows[i], std::max(to / 304.0, 1.0), co, so);
                    T->co1[i] = (int)co.size();
                }
                T->maxchunks = std::max(T->maxchunks, std::max(sl, std::max(su, so)));
            }
            T->d_pl = upload(h, pl, T->owned);
            T->d_pu = upload(h, pu, T->owned);
            T->d_cl = upload(h, cl, T->owned);
            T->d_cu = upload(h, cu, T->owned);
            T->d_po = upload(h, po, T->owned);
            T->d_co = upload(h, co, T->owned);
            // explicit inverses of the diagonal factors of every tile: L_ii^-1 (unit lower) and
            // U_ii^-1, from the tile's diagonal sub-block of its leaf
            size_t tot = 0;
            for (int i = 0; i < T->ntile; ++i) {
                T->inv_off.push_back(tot);
                tot += 2 * (size_t)T->rows[i] * T->rows[i];
            }
            T->d_inv = (C *)dalloc(h, sizeof(C) * std::max<size_t>(tot, 1));
            T->owned.push_back(T->d_inv);
            // the tiles' inverses are independent: concurrently on the stream pool
            const int ns = std::min(HM_POOL_STREAMS, T->ntile);
            pool_fork(h, ns);
            cudaStream_t main = h->stream;
            try {
                for (int i = 0; i < T->ntile; ++i) {
                    h->stream = h->pool[i % ns];
                    const int n = T->rows[i];
                    BlockT<C> *d = tdiag[i];
                    const size_t o = (size_t)(T->r0[i] - d->r0);
                    const C *Dii = d->D + o + o * d->nr;
                    C *Li = T->d_inv + T->inv_off[i], *Ui = Li + (size_t)n * n;
                    ztri_inverses(h, Dii, d->nr, n, Li, Ui);
                }
            } catch (...) {
                h->stream = main;
                pool_join(h, ns);
                throw;
            }
            h->stream = main;
            pool_join(h, ns);
            // the pivots of each diagonal leaf as one gather: applying the interchanges
            // k <-> piv[k] in order to z is z_new[j] = z_old[g[j]]
            std::vector<int> gall;
            std::vector<size_t> goff;
            for (BlockT<C> *d : diag) {
                const int n = d->nr;
                std::vector<int> pv(n), g(n);
                HM_CUDA(cudaMemcpyAsync(pv.data(), d->piv, sizeof(int) * n, cudaMemcpyDeviceToHost, h->stream));
                HM_CUDA(cudaStreamSynchronize(h->stream));
                for (int k = 0; k < n; ++k) g[k] = k;
                for (int k = 0; k < n; ++k) {
                    const int q = pv[k];
                    if (q < 0 || q >= n) throw HmError{HM_ERR_NUMERIC, "tile plan: pivot index out of range"};
                    std::swap(g[k], g[q]);
                }
                goff.push_back(gall.size());
                gall.insert(gall.end(), g.begin(), g.end());
            }
            const int *d_g = upload(h, gall, T->owned);
            T->gperm.assign(T->ntile, nullptr);
            T->ggperm.assign(T->ntile, nullptr);
            for (int i = 0, di = -1; i < T->ntile; ++i) {
                if (T->grp0[i] == i) ++di;
                if (T->grpn[i] == 1)
                    T->gperm[i] = d_g + goff[di];
                else if (T->grp0[i] == i)
                    T->ggperm[i] = d_g + goff[di];
            }
        }
    } catch (...) {
        tile_free(h, T);
        throw;
    }
    return T;
}

template <class C>
void tile_free(hm_handle_s *h, TileOp<C> *T)
{
    if (!T) return;
    for (void *p : T->owned) dfree(h, p);
    delete T;
}

// Y += alpha A X (tree order; X, Y: N x nrhs with ld N).
template <class C>
void tile_matvec(hm_handle_s *h, TileOp<C> *T, const C *X, C *Y, int nrhs, C alpha)
{
    if (nrhs <= 0 || T->ntile == 0) return;
    C *part = (C *)dalloc(h, sizeof(C) * (size_t)std::max(T->nca, 1) * nrhs * T->rmax);
    C *tbuf = (C *)dalloc(h, sizeof(C) * (size_t)std::max(T->ntjobs, 1) * nrhs);
    const size_t smem = partial_smem<C>(T->rmax);
    if (T->ntjobs) {
        const int per = TL_T / 32;
        k_leaf_vhx<C><<<(T->ntjobs + per - 1) / per, TL_T, 0, h->stream>>>(T->d_tl, T->d_tjobs, T->d_tv, T->ntjobs, X,
                                                                           T->N, nrhs, tbuf);
        HM_CHECK_LAUNCH();
        count_launch(h);
    }
    if (T->nca) {
        k_tile_partial<C><<<T->nca, TL_T, smem, h->stream>>>(T->d_pa, T->d_ca, X, T->N, nrhs, part, T->rmax, tbuf);
        HM_CHECK_LAUNCH();
    }
    k_tile_reduce<C><<<T->ntile, TL_T, 0, h->stream>>>(T->d_tr0, T->d_trows, T->d_ts0, T->d_ts1, part, nrhs,
                                                        T->rmax, alpha, Y, T->N);
    HM_CHECK_LAUNCH();
    count_launch(h, T->nca ? 2 : 1);
    dfree(h, part);
    dfree(h, tbuf);
}

// X <- A^-1 X with the H-LU factors (tree order, N x nrhs, ld N).
template <class C>
void tile_solve(hm_handle_s *h, TileOp<C> *T, C *X, int nrhs)
{
    if (!T->factored) throw HmError{HM_ERR_STATE, "tile_solve on an unfactored plan"};
    if (nrhs <= 0 || T->ntile == 0) return;
    C *part = (C *)dalloc(h, sizeof(C) * (size_t)std::max(T->maxchunks, 1) * nrhs * T->rmax);
    C *z = (C *)dalloc(h, sizeof(C) * (size_t)std::max(T->rmax, T->maxgrow) * nrhs);
    const size_t psmem = partial_smem<C>(T->rmax);
    auto grid_of = [&](int rows) { return std::max(1, std::min(64, (int)((rows * (size_t)nrhs + TL_T - 1) / TL_T))); };
    auto partial = [&](const TPiece<C> *pcs, const TChunk *chs, int nch) {
        if (!nch) return;
        k_tile_partial<C><<<nch, TL_T, psmem, h->stream>>>(pcs, chs, X, T->N, nrhs, part, T->rmax, nullptr);
        HM_CHECK_LAUNCH();
        count_launch(h);
    };
    auto step = [&](int i, const TPiece<C> *pcs, const TChunk *chs, int nch, const int *g, const C *Minv) {
        partial(pcs, chs, nch);
        const int rows = T->rows[i];
        k_tile_prep<C><<<grid_of(rows), TL_T, 0, h->stream>>>(T->r0[i], rows, nch, part, nrhs, T->rmax, g, X, T->N, z);
        HM_CHECK_LAUNCH();
        k_tile_mul<C><<<(rows + TM_R - 1) / TM_R, TL_T, 0, h->stream>>>(T->r0[i], rows, nrhs, Minv, z, X, T->N);
        HM_CHECK_LAUNCH();
        count_launch(h, 2);
    };
    for (int i = 0; i < T->ntile;) {
        const int gn = T->grpn[i];
        if (gn == 1) {
            step(i, T->d_pl, T->d_cl + T->cl0[i], T->cl1[i] - T->cl0[i], T->gperm[i], T->d_inv + T->inv_off[i]);
            ++i;
            continue;
        }
        // a group: the leaves left of the block, then the block's permutation, then its L
        for (int j = i; j < i + gn; ++j) {
            const int nch = T->co1[j] - T->co0[j];
            if (!nch) continue;
            partial(T->d_po, T->d_co + T->co0[j], nch);
            k_tile_sub<C><<<grid_of(T->rows[j]), TL_T, 0, h->stream>>>(T->r0[j], T->rows[j], nch, part, nrhs,
                                                                      T->rmax, X, T->N);
            HM_CHECK_LAUNCH();
            count_launch(h);
        }
        const int r0 = T->r0[i], rows = T->r0[i + gn - 1] + T->rows[i + gn - 1] - r0;
        k_tile_prep<C><<<grid_of(rows), TL_T, 0, h->stream>>>(r0, rows, 0, part, nrhs, T->rmax, T->ggperm[i], X, T->N,
                                                              z);
        HM_CHECK_LAUNCH();
        k_tile_put<C><<<grid_of(rows), TL_T, 0, h->stream>>>(r0, rows, nrhs, z, X, T->N);
        HM_CHECK_LAUNCH();
        count_launch(h, 2);
        for (int j = i; j < i + gn; ++j)
            step(j, T->d_pl, T->d_cl + T->cl0[j], T->cl1[j] - T->cl0[j], nullptr, T->d_inv + T->inv_off[j]);
        i += gn;
    }
    for (int i = T->ntile - 1; i >= 0; --i)
        step(i, T->d_pu, T->d_cu + T->cu0[i], T->cu1[i] - T->cu0[i], nullptr,
             T->d_inv + T->inv_off[i] + (size_t)T->rows[i] * T->rows[i]);
    dfree(h, part);
    dfree(h, z);
}

#define HM_INST_TILES(Z)                                                              \
    template TileOp<Z> *tile_build<Z>(hm_handle_s *, BlockT<Z> *, bool);              \
    template void tile_free<Z>(hm_handle_s *, TileOp<Z> *);                           \
    template void tile_matvec<Z>(hm_handle_s *, TileOp<Z> *, const Z *, Z *, int, Z); \
    template void tile_solve<Z>(hm_handle_s *, TileOp<Z> *, Z *, int);
HM_INST_TILES(zc)
HM_INST_TILES(cf)
