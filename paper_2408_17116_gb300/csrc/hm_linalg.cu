// Complex FP64 dense kernels for the H-matrix arithmetic: GEMM, leaf LU with
// partial pivoting, triangular solves, Householder QR, one-sided Jacobi SVD and
// the truncated recompression of low-rank sums (Sec. III: "fast formatted matrix
// addition and multiplication", H-LU of ref. [23]).
//
// On GB300 FP64 runs on the CUDA-core FP64 pipe; these kernels are bound by it.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <type_traits>

#include "hm_internal.h"

// ---------------------------------------------------------------------------
// GEMM: C = alpha op(A) op(B) + beta C, 64 x 64 tiles, BK = 8, 256 threads,
// 4 x 4 outputs per thread; optional deterministic split-K through a workspace.
// ---------------------------------------------------------------------------
#define GB_M 64
#define GB_N 64
#define GB_K 16

template <class C>
struct GemmArgs {
    int opA, opB;  // 0 'N', 1 'C'
    int m, n, k;
    C alpha, beta;
    const C *A;
    int lda;
    const C *B;
    int ldb;
    C *Cm;
    int ldc;
    C *work;      // split-K partials [splits][m][n] (column-major m x n each), or null
    int kchunk;
};

template <class C>
__device__ __forceinline__ C loadA(const GemmArgs<C> &g, int i, int p)
{
    if (i >= g.m || p >= g.k) return cmk<C>(0, 0);
    return g.opA ? zconj(g.A[(size_t)i * g.lda + p]) : g.A[(size_t)p * g.lda + i];
}
template <class C>
__device__ __forceinline__ C loadB(const GemmArgs<C> &g, int p, int j)
{
    if (j >= g.n || p >= g.k) return cmk<C>(0, 0);
    return g.opB ? zconj(g.B[(size_t)p * g.ldb + j]) : g.B[(size_t)j * g.ldb + p];
}

// Products of one staged k-slice into the NX x NY groups of 16 outputs a thread owns.
// NX, NY are compile-time so a partial tile issues no products for padding (the
// FP64 pipe of GB300 is the bound of the complex128 GEMMs).
template <class C, int NX, int NY>
__device__ __forceinline__ void gemm_slice(C (&acc)[4][4], const C (*As)[GB_M], const C (*Bs)[GB_N + 1], int tx,
                                           int ty)
{
#pragma unroll
    for (int pp = 0; pp < GB_K; ++pp) {
        C a[NX], b[NY];
#pragma unroll
        for (int q = 0; q < NX; ++q) a[q] = As[pp][tx + 16 * q];
#pragma unroll
        for (int q = 0; q < NY; ++q) b[q] = Bs[pp][ty + 16 * q];
#pragma unroll
        for (int x = 0; x < NX; ++x)
#pragma unroll
            for (int y = 0; y < NY; ++y) acc[x][y] = zfma(a[x], b[y], acc[x][y]);
    }
}

template <class C, int NX>
__device__ __forceinline__ void gemm_slice_nx(C (&acc)[4][4], const C (*As)[GB_M], const C (*Bs)[GB_N + 1], int tx,
                                              int ty, int ny)
{
    switch (ny) {
    case 1: gemm_slice<C, NX, 1>(acc, As, Bs, tx, ty); break;
    case 2: gemm_slice<C, NX, 2>(acc, As, Bs, tx, ty); break;
    case 3: gemm_slice<C, NX, 3>(acc, As, Bs, tx, ty); break;
    case 4: gemm_slice<C, NX, 4>(acc, As, Bs, tx, ty); break;
    default: break;  // no outputs in this warp
    }
}

template <class C>
__global__ void __launch_bounds__(256) k_zgemm(GemmArgs<C> g)
{
    __shared__ C As[GB_K][GB_M];
    __shared__ C Bs[GB_K][GB_N + 1];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int i0 = blockIdx.x * GB_M, j0 = blockIdx.y * GB_N;
    const int kb = blockIdx.z * g.kchunk, ke = min(g.k, kb + g.kchunk);
    C acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = cmk<C>(0, 0);
    // 16-row groups holding outputs (uniform over the CTA) and 16-column groups holding
    // outputs for this warp's threads (uniform over the warp)
    const int wy0 = j0 + ((tid >> 5) << 1);  // first column of this warp's threads
    const int nx = min(4, (g.m - i0 + 15) / 16);
    const int ny = wy0 < g.n ? min(4, (g.n - wy0 + 15) / 16) : 0;
    for (int p0 = kb; p0 < ke; p0 += GB_K) {
        // load 64 x GB_K of A and GB_K x 64 of B: 64 GB_K elements each, GB_K / 4 per thread
#pragma unroll
        for (int r = 0; r < GB_K / 4; ++r) {
            int e = tid + r * 256;
            int ii = e & 63, pp = e >> 6;
            int gp = p0 + pp;
            As[pp][ii] = (gp < ke) ? loadA(g, i0 + ii, gp) : cmk<C>(0, 0);
            int jj = e & 63;
            Bs[pp][jj] = (gp < ke) ? loadB(g, gp, j0 + jj) : cmk<C>(0, 0);
        }
        __syncthreads();
        switch (nx) {
        case 1: gemm_slice_nx<C, 1>(acc, As, Bs, tx, ty, ny); break;
        case 2: gemm_slice_nx<C, 2>(acc, As, Bs, tx, ty, ny); break;
        case 3: gemm_slice_nx<C, 3>(acc, As, Bs, tx, ty, ny); break;
        default: gemm_slice_nx<C, 4>(acc, As, Bs, tx, ty, ny); break;
        }
        __syncthreads();
    }
#pragma unroll
    for (int x = 0; x < 4; ++x) {
        int i = i0 + tx + 16 * x;
        if (i >= g.m) continue;
#pragma unroll
        for (int y = 0; y < 4; ++y) {
            int j = j0 + ty + 16 * y;
            if (j >= g.n) continue;
            if (g.work) {
                g.work[(size_t)blockIdx.z * g.m * g.n + (size_t)j * g.m + i] = acc[x][y];
            } else {
                C v = zmul(g.alpha, acc[x][y]);
                C *c = g.Cm + (size_t)j * g.ldc + i;
                if (g.beta.x != 0.0 || g.beta.y != 0.0) v = zfma(g.beta, *c, v);
                *c = v;
            }
        }
    }
}

template <class C>
__global__ void k_splitk_reduce(GemmArgs<C> g, int splits)
{
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t mn = (size_t)g.m * g.n;
    if (idx >= mn) return;
    C s = cmk<C>(0, 0);
    for (int z = 0; z < splits; ++z) s = zadd(s, g.work[(size_t)z * mn + idx]);
    int i = (int)(idx % g.m), j = (int)(idx / g.m);
    C v = zmul(g.alpha, s);
    C *c = g.Cm + (size_t)j * g.ldc + i;
    if (g.beta.x != 0.0 || g.beta.y != 0.0) v = zfma(g.beta, *c, v);
    *c = v;
}

template <class C>
__global__ void k_scale(C *Cm, int m, int n, int ldc, C beta)
{
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)m * n) return;
    int i = (int)(idx % m), j = (int)(idx / m);
    C *c = Cm + (size_t)j * ldc + i;
    *c = (beta.x == 0 && beta.y == 0) ? cmk<C>(0, 0) : zmul(beta, *c);
}

template <class C>
void zgemm(hm_handle_s *h, char opA, char opB, int m, int n, int k, C alpha, const C *A, int lda, const C *B, int ldb,
           C beta, C *Cm, int ldc)
{
    if (m <= 0 || n <= 0) return;
    if (k <= 0) {
        size_t mn = (size_t)m * n;
        k_scale<C><<<(unsigned)((mn + 255) / 256), 256, 0, h->stream>>>(Cm, m, n, ldc, beta);
        HM_CHECK_LAUNCH();
        count_launch(h);
        return;
    }
    if constexpr (std::is_same<C, cf>::value) {
        if (tc_eligible(h, m, n, k)) {
            tc_gemm(h, opA, opB, m, n, k, alpha, A, lda, B, ldb, beta, Cm, ldc);
            return;
        }
    }
    GemmArgs<C> g;
    g.opA = (opA == 'C');
    g.opB = (opB == 'C');
    g.m = m;
    g.n = n;
    g.k = k;
    g.alpha = alpha;
    g.beta = beta;
    g.A = A;
    g.lda = lda;
    g.B = B;
    g.ldb = ldb;
    g.Cm = Cm;
    g.ldc = ldc;
    int gm = (m + GB_M - 1) / GB_M, gn = (n + GB_N - 1) / GB_N;
    int tiles = gm * gn;
    int splits = 1;
    // split K when the output has few tiles and the inner dimension is long
    if (tiles < 76 && k >= 512) splits = std::min(std::max(1, 152 / tiles), std::max(1, k / 256));
    h->flops_factor += 8.0 * m * n * k;
    if (splits > 1) {
        g.kchunk = ((k + splits - 1) / splits + GB_K - 1) / GB_K * GB_K;
        splits = (k + g.kchunk - 1) / g.kchunk;
        g.work = (C *)dalloc(h, sizeof(C) * (size_t)m * n * splits);
        k_zgemm<C><<<dim3(gm, gn, splits), 256, 0, h->stream>>>(g);
        HM_CHECK_LAUNCH();
        size_t mn = (size_t)m * n;
        k_splitk_reduce<C><<<(unsigned)((mn + 255) / 256), 256, 0, h->stream>>>(g, splits);
        HM_CHECK_LAUNCH();
        count_launch(h, 2);
        dfree(h, g.work);
    } else {
        g.work = nullptr;
        g.kchunk = k;
        // the large products (at least 1e9 real flops) are timed with CUDA events around
        // the launch; their durations are read after the factorisation (gemm_timing_collect)
        const double fl = 8.0 * m * n * k;
        const bool timed = fl >= 1e9;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (timed) {
            e0 = gemm_event(h);
            e1 = gemm_event(h);
            HM_CUDA(cudaEventRecord(e0, h->stream));
        }
        k_zgemm<C><<<dim3(gm, gn, 1), 256, 0, h->stream>>>(g);
        HM_CHECK_LAUNCH();
        if (timed) {
            HM_CUDA(cudaEventRecord(e1, h->stream));
            h->gemm_pending.push_back(GemmTiming{e0, e1, fl});
        }
        count_launch(h);
    }
}

void phase_collect(hm_handle_s *h)
{
    for (const PhaseMark &m : h->phase_pending) {
        float ms = 0;
        if (cudaEventElapsedTime(&ms, m.e0, m.e1) == cudaSuccess) h->phase_s[m.id] += 1e-3 * ms;
        h->gemm_free.push_back(m.e0);
        h->gemm_free.push_back(m.e1);
    }
    h->phase_pending.clear();
}

cudaEvent_t gemm_event(hm_handle_s *h)
{
    if (h->gemm_free.empty()) {
        cudaEvent_t e;
        HM_CUDA(cudaEventCreate(&e));
        return e;
    }
    cudaEvent_t e = h->gemm_free.back();
    h->gemm_free.pop_back();
    return e;
}

// Accumulate the device time of the timed products recorded since the last call (the
// stream must have been synchronised) and return their events to the pool.
void gemm_timing_collect(hm_handle_s *h)
{
    for (const GemmTiming &t : h->gemm_pending) {
        float ms = 0;
        if (cudaEventElapsedTime(&ms, t.e0, t.e1) == cudaSuccess) {
            if (t.kind) {
                h->ktc_s += 1e-3 * ms;
                h->ktc_flops += t.flops;
                h->ktc_n += 1;
            } else {
                h->kgemm_s += 1e-3 * ms;
                h->kgemm_flops += t.flops;
                h->kgemm_n += 1;
            }
        }
        h->gemm_free.push_back(t.e0);
        h->gemm_free.push_back(t.e1);
    }
    h->gemm_pending.clear();
}

// ---------------------------------------------------------------------------
// LU with partial pivoting of one n x n leaf (n <= 1024), one CTA.
// Pivot: largest modulus in the column, ties to the lowest row.  piv[k] = row
// swapped with k (0-based, applied in order k = 0..n-1).  info: 0 or k+1 on a zero pivot.
// ---------------------------------------------------------------------------
template <class C>
__global__ void __launch_bounds__(1024) k_getrf(int n, C *A, int lda, int *piv, int *info)
{
    typedef typename CReal<C>::R R;
    __shared__ R sv[33];
    __shared__ int si[33];
    __shared__ int s_p;
    __shared__ C s_inv;
    const int tid = threadIdx.x, nt = blockDim.x;
    int bad = 0;
    for (int k = 0; k < n; ++k) {
        // argmax |A[i,k]|, i >= k
        R bv = -1;
        int bi = 0x7fffffff;
        for (int i = k + tid; i < n; i += nt) {
            R v = zabs2(A[(size_t)k * lda + i]);
            if (v > bv || (v == bv && i < bi)) {
                bv = v;
                bi = i;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            R v2 = __shfl_down_sync(0xffffffff, bv, o);
            int i2 = __shfl_down_sync(0xffffffff, bi, o);
            if (v2 > bv || (v2 == bv && i2 < bi)) {
                bv = v2;
                bi = i2;
            }
        }
        if ((tid & 31) == 0) {
            sv[tid >> 5] = bv;
            si[tid >> 5] = bi;
        }
        __syncthreads();
        if (tid == 0) {
            R v = sv[0];
            int ii = si[0];
            for (int w = 1; w < (nt + 31) / 32; ++w)
                if (sv[w] > v || (sv[w] == v && si[w] < ii)) {
                    v = sv[w];
                    ii = si[w];
                }
            // a column without a finite entry leaves no valid argmax: no interchange (the
            // zero / non-finite pivot is reported through info below)
            if (ii < k || ii >= n) ii = k;
            s_p = ii;
            piv[k] = ii;
            if (!(v > 0)) {
                if (!bad) *info = k + 1;
                bad = 1;
                s_inv = cmk<C>(0, 0);
            } else {
                C pv = A[(size_t)k * lda + ii];
                s_inv = zdiv(cmk<C>(1, 0), pv);
            }
        }
        __syncthreads();
        const int p = s_p;
        if (p != k)
            for (int j = tid; j < n; j += nt) {
                C t = A[(size_t)j * lda + k];
                A[(size_t)j * lda + k] = A[(size_t)j * lda + p];
                A[(size_t)j * lda + p] = t;
            }
        __syncthreads();
        const C inv = s_inv;
        for (int i = k + 1 + tid; i < n; i += nt) A[(size_t)k * lda + i] = zmul(A[(size_t)k * lda + i], inv);
        __syncthreads();
        const int m = n - k - 1;
        for (int e = tid; e < m * m; e += nt) {
            int i = k + 1 + e % m, j = k + 1 + e / m;
            A[(size_t)j * lda + i] = zsub(A[(size_t)j * lda + i], zmul(A[(size_t)k * lda + i], A[(size_t)j * lda + k]));
        }
        __syncthreads();
    }
    if (tid == 0 && !bad && info) {
        // keep info untouched when zero (caller initialised)
    }
}

template <class C>
void ztrsm_lln(hm_handle_s *h, const C *L, int ldl, int n, MVT<C> X);

// Panel of the blocked LU: columns [j0, j0 + nb) of an m x m block (rows j0 .. m), one CTA,
// partial pivoting over the rows below the diagonal (ties to the lowest row); the row
// interchanges are applied to the panel's columns only (k_laswp_range does the rest).
template <class C>
__global__ void __launch_bounds__(512) k_getf2_panel(int m, C *A, int lda, int j0, int nb, int *piv, int *info)
{
    typedef typename CReal<C>::R R;
    __shared__ R sv[32];
    __shared__ int si[32];
    __shared__ int s_p;
    __shared__ C s_inv;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int k = j0; k < j0 + nb; ++k) {
        R bv = -1;
        int bi = 0x7fffffff;
        for (int i = k + tid; i < m; i += nt) {
            R v = zabs2(A[(size_t)k * lda + i]);
            if (v > bv || (v == bv && i < bi)) {
                bv = v;
                bi = i;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            R v2 = __shfl_down_sync(0xffffffff, bv, o);
            int i2 = __shfl_down_sync(0xffffffff, bi, o);
            if (v2 > bv || (v2 == bv && i2 < bi)) {
                bv = v2;
                bi = i2;
            }
        }
        if ((tid & 31) == 0) {
            sv[tid >> 5] = bv;
            si[tid >> 5] = bi;
        }
        __syncthreads();
        if (tid == 0) {
            R v = sv[0];
            int ii = si[0];
            for (int w = 1; w < (nt + 31) / 32; ++w)
                if (sv[w] > v || (sv[w] == v && si[w] < ii)) {
                    v = sv[w];
                    ii = si[w];
                }
            if (ii < k || ii >= m) ii = k;
            s_p = ii;
            piv[k] = ii;
            if (!(v > 0)) {
                if (*info == 0) *info = k + 1;
                s_inv = cmk<C>(0, 0);
            } else {
                s_inv = zdiv(cmk<C>(1, 0), A[(size_t)k * lda + ii]);
            }
        }
        __syncthreads();
        const int p = s_p;
        if (p != k)
            for (int j = j0 + tid; j < j0 + nb; j += nt) {
                C t = A[(size_t)j * lda + k];
                A[(size_t)j * lda + k] = A[(size_t)j * lda + p];
                A[(size_t)j * lda + p] = t;
            }
        __syncthreads();
        const C inv = s_inv;
        for (int i = k + 1 + tid; i < m; i += nt) A[(size_t)k * lda + i] = zmul(A[(size_t)k * lda + i], inv);
        __syncthreads();
        const int rows = m - k - 1, cols = j0 + nb - k - 1;
        for (int e = tid; e < rows * cols; e += nt) {
            int i = k + 1 + e % rows, j = k + 1 + e / rows;
            A[(size_t)j * lda + i] = zsub(A[(size_t)j * lda + i], zmul(A[(size_t)k * lda + i], A[(size_t)j * lda + k]));
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Panel LU on many CTAs (tall panels): columns [j0, j0 + nb) of an n x n block over rows
// [j0, n).  The rows are split into slabs of R rows, one slab per CTA, held in shared
// memory for the whole panel.  Per column k each CTA proposes the entry of largest
// modulus in its slab together with that row (and the owner of row k publishes row k);
// after one grid barrier every CTA takes the same pivot (largest modulus, ties to the
// lowest row), the owners of rows k and p exchange them, and each CTA scales its part of
// the column and updates its slab.  Proposals are double-buffered by column parity (no CTA
// runs more than one barrier ahead of another).  The same partial pivoting as the
// one-CTA panel; the barrier waits are bounded (2 s): on expiry info is set to -1.
// ---------------------------------------------------------------------------
#define PC_T 256
#define PC_NBMAX 64

struct GridBar {
    unsigned count, gen;
};

__device__ __forceinline__ uint64_t pc_timer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// All CTAs of the (cooperative) grid meet; false on a 2 s timeout or when another CTA
// has reported one (info < 0).
__device__ bool pc_barrier(GridBar *gb, unsigned nblocks, int *info)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *vgen = &gb->gen;
        const unsigned my = *vgen;
        __threadfence();
        int ok = 1;
        if (atomicAdd(&gb->count, 1u) == nblocks - 1) {
            atomicExch(&gb->count, 0u);
            __threadfence();
            atomicAdd(&gb->gen, 1u);
        } else {
            const uint64_t t0 = pc_timer();
            for (unsigned it = 1; *vgen == my; ++it) {
                if ((it & 1023) == 0) {
                    if (*(volatile int *)info < 0 || pc_timer() - t0 > 2000000000ull) {
                        atomicExch(info, -1);
                        ok = 0;
                        break;
                    }
                }
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// (v, p) reduction over the CTA: largest v, ties to the lowest p; w travels with p.
template <class R>
__device__ void pc_argmax(R &v, int &p, int &w)
{
    __shared__ R sv[PC_T / 32];
    __shared__ int sp[PC_T / 32], sw[PC_T / 32];
    for (int o = 16; o > 0; o >>= 1) {
        R v2 = __shfl_down_sync(0xffffffffu, v, o);
        int p2 = __shfl_down_sync(0xffffffffu, p, o), w2 = __shfl_down_sync(0xffffffffu, w, o);
        if (v2 > v || (v2 == v && p2 < p)) {
            v = v2;
            p = p2;
            w = w2;
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        sv[warp] = v;
        sp[warp] = p;
        sw[warp] = w;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 1; q < PC_T / 32; ++q)
            if (sv[q] > v || (sv[q] == v && sp[q] < p)) {
                v = sv[q];
                p = sp[q];
                w = sw[q];
            }
        sv[0] = v;
        sp[0] = p;
        sw[0] = w;
    }
    __syncthreads();
    v = sv[0];
    p = sp[0];
    w = sw[0];
    __syncthreads();
}

template <class C>
__global__ void __launch_bounds__(PC_T) k_getf2_coop(int n, C *A, int lda, int j0, int nb, int R, int *piv, int *info,
                                                     C *cand_rows, typename CReal<C>::R *cand_val, int *cand_pos,
                                                     C *krow, GridBar *gb)
{
    typedef typename CReal<C>::R Rl;
    extern __shared__ __align__(16) unsigned char pc_raw[];
    C *S = (C *)pc_raw;  // S[j * R + i] = A[r0 + i, j0 + j]
    __shared__ C s_prow[PC_NBMAX];
    const int G = gridDim.x, c = blockIdx.x, tid = threadIdx.x;
    const int r0 = j0 + c * R;
    const int rn = max(0, min(R, n - r0));
    for (int e = tid; e < nb * R; e += PC_T) {
        const int j = e / R, i = e - j * R;
        S[e] = i < rn ? A[(size_t)(j0 + j) * lda + r0 + i] : cmk<C>(0, 0);
    }
    __syncthreads();
    for (int kk = 0; kk < nb; ++kk) {
        const int k = j0 + kk, par = kk & 1;
        // 1. this slab's proposal among rows >= k
        Rl v = -1;
        int p = 0x7fffffff, w = c;
        for (int i = max(0, k - r0) + tid; i < rn; i += PC_T) {
            const Rl a = zabs2(S[kk * R + i]);
            if (a > v || (a == v && r0 + i < p)) {
                v = a;
                p = r0 + i;
            }
        }
        pc_argmax(v, p, w);
        // 2. publish it (and row k from its owner)
        if (tid == 0) {
            cand_val[par * G + c] = v;
            cand_pos[par * G + c] = p;
        }
        if (p != 0x7fffffff)
            for (int j = tid; j < nb; j += PC_T) cand_rows[((size_t)par * G + c) * nb + j] = S[j * R + (p - r0)];
        if (k >= r0 && k < r0 + rn)
            for (int j = tid; j < nb; j += PC_T) krow[par * nb + j] = S[j * R + (k - r0)];
        __threadfence();
        // 3. all proposals are in
        if (!pc_barrier(gb, G, info)) return;
        // 4. the common pivot
        v = -1;
        p = 0x7fffffff;
        w = 0;
        for (int q = tid; q < G; q += PC_T) {
            const Rl vq = __ldcg(cand_val + par * G + q);
            const int pq = __ldcg(cand_pos + par * G + q);
            if (pq != 0x7fffffff && (vq > v || (vq == v && pq < p))) {
                v = vq;
                p = pq;
                w = q;
            }
        }
        pc_argmax(v, p, w);
        if (p < k || p >= n) p = k;  // cannot happen: the owner of row k always proposes
        for (int j = tid; j < nb; j += PC_T) s_prow[j] = __ldcg(cand_rows + ((size_t)par * G + w) * nb + j);
        if (c == 0 && tid == 0) {
            piv[k] = p;
            if (!(v > 0) && *info == 0) *info = k + 1;
        }
        __syncthreads();
        // 5. rows k and p change places
        if (p != k) {
            if (k >= r0 && k < r0 + rn)
                for (int j = tid; j < nb; j += PC_T) S[j * R + (k - r0)] = s_prow[j];
            if (p >= r0 && p < r0 + rn)
                for (int j = tid; j < nb; j += PC_T) S[j * R + (p - r0)] = __ldcg(krow + par * nb + j);
        }
        __syncthreads();
        // 6. multipliers and the rank-1 update of the slab below row k
        const C inv = v > 0 ? zdiv(cmk<C>(1, 0), s_prow[kk]) : cmk<C>(0, 0);
        for (int i = max(0, k + 1 - r0) + tid; i < rn; i += PC_T) {
            const C l = zmul(S[kk * R + i], inv);
            S[kk * R + i] = l;
            for (int j = kk + 1; j < nb; ++j) S[j * R + i] = zsub(S[j * R + i], zmul(l, s_prow[j]));
        }
        __syncthreads();
    }
    for (int e = tid; e < nb * R; e += PC_T) {
        const int j = e / R, i = e - j * R;
        if (i < rn) A[(size_t)(j0 + j) * lda + r0 + i] = S[e];
    }
}

// Workspace and launch geometry of the many-CTA panel for a block of n rows.
template <class C>
struct PanelCoop {
    int G = 0;            // CTAs (at most one per SM)
    C *rows = nullptr;    // [2][G][PC_NBMAX]
    typename CReal<C>::R *val = nullptr;
    int *pos = nullptr;
    C *krow = nullptr;    // [2][PC_NBMAX]
    GridBar *gb = nullptr;
    void *buf = nullptr;
};

template <class C>
static bool panel_coop_init(hm_handle_s *h, PanelCoop<C> &P)
{
    int dev = 0, nsm = 0;
    HM_CUDA(cudaGetDevice(&dev));
    HM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    P.G = nsm;
    const size_t b_rows = sizeof(C) * 2 * (size_t)P.G * PC_NBMAX, b_val = sizeof(typename CReal<C>::R) * 2 * P.G;
    const size_t b_pos = sizeof(int) * 2 * P.G, b_k = sizeof(C) * 2 * PC_NBMAX;
    const size_t tot = b_rows + b_val + b_pos + b_k + sizeof(GridBar) + 64;
    P.buf = dalloc(h, tot);
    char *q = (char *)P.buf;
    P.rows = (C *)q;
    q += b_rows;
    P.krow = (C *)q;
    q += b_k;
    P.val = (typename CReal<C>::R *)q;
    q += b_val;
    P.pos = (int *)q;
    q += b_pos;
    P.gb = (GridBar *)(((uintptr_t)q + 15) & ~(uintptr_t)15);
    return true;
}

// Factor columns [j0, j0 + nb) over rows [j0, n) on G CTAs; nb and the slab height fit in
// shared memory (checked by the caller through panel_width).
template <class C>
static void panel_coop(hm_handle_s *h, PanelCoop<C> &P, int n, C *A, int lda, int j0, int nb, int *piv, int *info)
{
    const int m = n - j0;
    const int G = std::min(P.G, std::max(1, (m + 63) / 64));
    const int R = (m + G - 1) / G;
    const size_t smem = sizeof(C) * (size_t)nb * R;
    static bool attr[2] = {false, false};
    bool &a = attr[sizeof(C) == sizeof(cf) ? 0 : 1];
    if (!a) {
        HM_CUDA(cudaFuncSetAttribute(k_getf2_coop<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, 210 * 1024));
        a = true;
    }
    HM_CUDA(cudaMemsetAsync(P.gb, 0, sizeof(GridBar), h->stream));
    void *args[] = {(void *)&n, (void *)&A, (void *)&lda, (void *)&j0, (void *)&nb, (void *)&R, (void *)&piv,
                    (void *)&info, (void *)&P.rows, (void *)&P.val, (void *)&P.pos, (void *)&P.krow, (void *)&P.gb};
    HM_CUDA(cudaLaunchCooperativeKernel((const void *)k_getf2_coop<C>, dim3(G), dim3(PC_T), args, smem, h->stream));
}

// Columns of an inner panel step for a panel of m rows: the widest of 64, 32, 16 whose
// slabs fit in 200 KB of shared memory on nsm CTAs; 0 when none does (one-CTA panel).
template <class C>
static int panel_width(int m, int nsm)
{
    const int G = std::min(nsm, std::max(1, (m + 63) / 64));
    const size_t R = (size_t)((m + G - 1) / G);
    for (int nb = PC_NBMAX; nb >= 16; nb /= 2)
        if (sizeof(C) * nb * R <= 200 * 1024) return nb;
    return 0;
}

// Row interchanges k <-> piv[k], k in [k0, k1), on the columns [0, c_lo) and [c_hi, n).
template <class C>
__global__ void k_laswp_range(C *A, int lda, int c_lo, int c_hi, int n, const int *piv, int k0, int k1)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    int j = t < c_lo ? t : c_hi + (t - c_lo);
    if (j >= n) return;
    C *x = A + (size_t)j * lda;
    for (int k = k0; k < k1; ++k) {
        int p = piv[k];
        if (p != k) {
            C tmp = x[k];
            x[k] = x[p];
            x[p] = tmp;
        }
    }
}

template <class C>
__global__ void k_eye(C *I, int n)
{
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < (size_t)n * n) I[idx] = cmk<C>((idx % n) == (idx / n) ? 1 : 0, 0);
}

template <class C>
static void trsm_left(hm_handle_s *h, int mode, const C *T, int ldt, int n, MVT<C> X);
template <class C>
void zcopy2d(hm_handle_s *h, MVT<C> dst, MVT<C> src);

#define LU_NB 32    // columns of a panel step (one CTA)
#define LU_NBO 512  // columns of an outer step: its trailing update is a product of depth 512

template <class C>
void zgetrf(hm_handle_s *h, int n, C *A, int lda, int *piv, int *d_info)
{
    if (n <= 0) return;
    h->flops_factor += 8.0 / 3.0 * n * (double)n * n;
    if (n <= 256) {
        int T = n >= 128 ? 512 : 256;
        k_getrf<C><<<1, T, 0, h->stream>>>(n, A, lda, piv, d_info);
        HM_CHECK_LAUNCH();
        count_launch(h);
        return;
    }
    // blocked right-looking LU with the same partial pivoting over the whole block, in two
    // levels: an outer step factors a column panel of LU_NBO columns (inner steps of LU_NB
    // columns whose updates stay inside the panel), applies its interchanges to the other
    // columns, forms U12 = L11^-1 A12 and updates A22 -= L21 U12 with one product of depth
    // LU_NBO (the tensor cores for complex64)
    const double saved = h->flops_factor;
    // complex64 on the tensor cores: U12 = (L11^-1) A12 as a product with the explicit
    // inverse of the unit lower panel block (one small solve on the identity) instead of a
    // column-sequential solve over the whole row block
    C *work = nullptr;
    const bool inv12 = std::is_same<C, cf>::value && !h->prm.simt_gemm && n > 2 * LU_NBO;
    if (inv12) work = (C *)dalloc(h, sizeof(C) * ((size_t)LU_NBO * LU_NBO + (size_t)LU_NBO * (n - LU_NBO)));
    // tall panels (at least PC_MIN_ROWS rows) factor on many CTAs
    const int PC_MIN_ROWS = 2048;
    PanelCoop<C> pc;
    int nsm = 0;
    if (n >= PC_MIN_ROWS) {
        panel_coop_init<C>(h, pc);
        nsm = pc.G;
    }
    for (int J0 = 0; J0 < n; J0 += LU_NBO) {
        const int NB = std::min(LU_NBO, n - J0), REST = n - J0 - NB;
        PhaseScope ps_panel(h, PH_LU_PANEL);
        const int wc = (n - J0 >= PC_MIN_ROWS) ? panel_width<C>(n - J0, nsm) : 0;
        const int step = wc ? wc : LU_NB;
        for (int j0 = J0; j0 < J0 + NB; j0 += step) {
            const int nb = std::min(step, J0 + NB - j0), rest = J0 + NB - j0 - nb;
            if (wc) {
                panel_coop<C>(h, pc, n, A, lda, j0, nb, piv, d_info);
            } else {
                k_getf2_panel<C><<<1, 512, 0, h->stream>>>(n, A, lda, j0, nb, piv, d_info);
                HM_CHECK_LAUNCH();
            }
            const int ncols = NB - nb;  // the panel's other columns
            if (ncols > 0) {
                k_laswp_range<C><<<(ncols + 127) / 128, 128, 0, h->stream>>>(A + (size_t)J0 * lda, lda, j0 - J0,
                                                                            j0 + nb - J0, NB, piv, j0, j0 + nb);
                HM_CHECK_LAUNCH();
            }
            count_launch(h, ncols > 0 ? 2 : 1);
            if (rest > 0) {
                ztrsm_lln<C>(h, A + (size_t)j0 * lda + j0, lda, nb,
                             MVT<C>{A + (size_t)(j0 + nb) * lda + j0, nb, rest, lda});
                zgemm<C>(h, 'N', 'N', n - j0 - nb, rest, nb, cmk<C>(-1, 0), A + (size_t)j0 * lda + j0 + nb, lda,
                         A + (size_t)(j0 + nb) * lda + j0, lda, cmk<C>(1, 0),
                         A + (size_t)(j0 + nb) * lda + j0 + nb, lda);
            }
        }
        ps_panel.end();
        PhaseScope ps_u12(h, PH_LU_U12);
        const int ocols = n - NB;  // columns outside the panel
        if (ocols > 0) {
            k_laswp_range<C><<<(ocols + 127) / 128, 128, 0, h->stream>>>(A, lda, J0, J0 + NB, n, piv, J0, J0 + NB);
            HM_CHECK_LAUNCH();
            count_launch(h);
        }
        if (REST > 0) {
            C *A12 = A + (size_t)(J0 + NB) * lda + J0;
            if (inv12) {
                C *Li = work, *T12 = work + (size_t)LU_NBO * LU_NBO;
                const size_t nn = (size_t)NB * NB;
                k_eye<C><<<(unsigned)((nn + 255) / 256), 256, 0, h->stream>>>(Li, NB);
                HM_CHECK_LAUNCH();
                count_launch(h);
                trsm_left(h, 0, A + (size_t)J0 * lda + J0, lda, NB, MVT<C>{Li, NB, NB, NB});
                zgemm<C>(h, 'N', 'N', NB, REST, NB, cmk<C>(1, 0), Li, NB, A12, lda, cmk<C>(0, 0), T12, NB);
                zcopy2d<C>(h, MVT<C>{A12, NB, REST, lda}, MVT<C>{T12, NB, REST, NB});
            } else {
                ztrsm_lln<C>(h, A + (size_t)J0 * lda + J0, lda, NB, MVT<C>{A12, NB, REST, lda});
            }
            ps_u12.end();
            zgemm<C>(h, 'N', 'N', REST, REST, NB, cmk<C>(-1, 0), A + (size_t)J0 * lda + J0 + NB, lda, A12, lda,
                     cmk<C>(1, 0), A + (size_t)(J0 + NB) * lda + J0 + NB, lda);
        }
    }
    if (work) dfree(h, work);
    if (pc.buf) dfree(h, pc.buf);
    h->flops_factor = saved;  // counted once above
}

// ---------------------------------------------------------------------------
// Row interchanges and triangular solves on multi-vectors X (rows x cols, ld)
// ---------------------------------------------------------------------------
template <class C>
__global__ void k_laswp(C *X, int ld, int cols, const int *piv, int n)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= cols) return;
    C *x = X + (size_t)j * ld;
    for (int k = 0; k < n; ++k) {
        int p = piv[k];
        if (p != k) {
            C t = x[k];
            x[k] = x[p];
            x[p] = t;
        }
    }
}

template <class C>
void zlaswp(hm_handle_s *h, MVT<C> X, const int *piv, int n)
{
    if (X.cols <= 0 || n <= 0) return;
    k_laswp<C><<<(X.cols + 127) / 128, 128, 0, h->stream>>>(X.p, X.ld, X.cols, piv, n);
    HM_CHECK_LAUNCH();
    count_launch(h);
}

// Left solves: one CTA per group of TRS_CB columns; the columns live in shared memory.
#define TRS_CB 8
#define TRS_T 256

// mode 0: X = L^-1 X (unit lower); 1: X = U^-1 X (upper); 2: X = U^-H X (U^H lower, non-unit)
template <class C>
__global__ void __launch_bounds__(TRS_T) k_trsm_left(int mode, const C *__restrict__ T, int ldt, int n, C *X, int ldx,
                                                      int cols, int cb)
{
    extern __shared__ __align__(16) unsigned char trs_raw[];
    C *xs = (C *)trs_raw;  // [cb][n]
    const int c0 = blockIdx.x * cb;
    const int nc = min(cb, cols - c0);
    const int tid = threadIdx.x;
    for (int e = tid; e < nc * n; e += TRS_T) {
        int c = e / n, i = e - c * n;
        xs[c * n + i] = X[(size_t)(c0 + c) * ldx + i];
    }
    __syncthreads();
    if (mode == 0) {
        for (int j = 0; j < n; ++j) {
            for (int e = tid; e < nc * (n - j - 1); e += TRS_T) {
                int c = e / (n - j - 1), i = j + 1 + e % (n - j - 1);
                xs[c * n + i] = zsub(xs[c * n + i], zmul(T[(size_t)j * ldt + i], xs[c * n + j]));
            }
            __syncthreads();
        }
    } else if (mode == 1) {
        for (int j = n - 1; j >= 0; --j) {
            if (tid < nc) xs[tid * n + j] = zdiv(xs[tid * n + j], T[(size_t)j * ldt + j]);
            __syncthreads();
            for (int e = tid; e < nc * j; e += TRS_T) {
                int c = e / j, i = e % j;
                xs[c * n + i] = zsub(xs[c * n + i], zmul(T[(size_t)j * ldt + i], xs[c * n + j]));
            }
            __syncthreads();
        }
    } else {
        for (int j = 0; j < n; ++j) {
            if (tid < nc) xs[tid * n + j] = zdiv(xs[tid * n + j], zconj(T[(size_t)j * ldt + j]));
            __syncthreads();
            for (int e = tid; e < nc * (n - j - 1); e += TRS_T) {
                int c = e / (n - j - 1), i = j + 1 + e % (n - j - 1);
                // (U^H)[i,j] = conj(U[j,i])
                xs[c * n + i] = zsub(xs[c * n + i], zmul(zconj(T[(size_t)i * ldt + j]), xs[c * n + j]));
            }
            __syncthreads();
        }
    }
    for (int e = tid; e < nc * n; e += TRS_T) {
        int c = e / n, i = e - c * n;
        X[(size_t)(c0 + c) * ldx + i] = xs[c * n + i];
    }
}

template <class C>
static void trsm_left(hm_handle_s *h, int mode, const C *T, int ldt, int n, MVT<C> X)
{
    if (X.cols <= 0 || n <= 0) return;
    // columns per CTA: TRS_CB, fewer when the staged columns would exceed 200 KB of shared memory
    const int cb = (int)std::max<size_t>(1, std::min<size_t>(TRS_CB, (size_t)200 * 1024 / (sizeof(C) * (size_t)n)));
    const size_t smem = sizeof(C) * cb * (size_t)n;
    if (smem > 227 * 1024) throw HmError{HM_ERR_ARG, "triangular solve: block of " + std::to_string(n) + " rows too large"};
    if (smem > 48 * 1024)
        HM_CUDA(cudaFuncSetAttribute(k_trsm_left<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_trsm_left<C><<<(X.cols + cb - 1) / cb, TRS_T, smem, h->stream>>>(mode, T, ldt, n, X.p, X.ld, X.cols, cb);
    HM_CHECK_LAUNCH();
    count_launch(h);
    h->flops_factor += 4.0 * n * (double)n * X.cols;
}

// Blocks of more than 2 TRS_BLK rows are solved in diagonal blocks of TRS_BLK rows, the rows
// below (forward) or above (backward) updated by one product per block (the tensor cores
// for complex64).
#define TRS_BLK 256

template <class C>
void ztrsm_lln(hm_handle_s *h, const C *L, int ldl, int n, MVT<C> X)
{
    if (n <= 2 * TRS_BLK) {
        trsm_left(h, 0, L, ldl, n, X);
        return;
    }
    for (int b0 = 0; b0 < n; b0 += TRS_BLK) {
        const int nb = std::min(TRS_BLK, n - b0), rest = n - b0 - nb;
        trsm_left(h, 0, L + b0 + (size_t)b0 * ldl, ldl, nb, MVT<C>{X.p + b0, nb, X.cols, X.ld});
        if (rest > 0)
            zgemm<C>(h, 'N', 'N', rest, X.cols, nb, cmk<C>(-1, 0), L + (b0 + nb) + (size_t)b0 * ldl, ldl, X.p + b0,
                     X.ld, cmk<C>(1, 0), X.p + b0 + nb, X.ld);
    }
}
template <class C>
void ztrsm_lun(hm_handle_s *h, const C *U, int ldu, int n, MVT<C> X)
{
    if (n <= 2 * TRS_BLK) {
        trsm_left(h, 1, U, ldu, n, X);
        return;
    }
    for (int b1 = n; b1 > 0; b1 -= TRS_BLK) {
        const int b0 = std::max(0, b1 - TRS_BLK), nb = b1 - b0;
        trsm_left(h, 1, U + b0 + (size_t)b0 * ldu, ldu, nb, MVT<C>{X.p + b0, nb, X.cols, X.ld});
        if (b0 > 0)
            zgemm<C>(h, 'N', 'N', b0, X.cols, nb, cmk<C>(-1, 0), U + (size_t)b0 * ldu, ldu, X.p + b0, X.ld,
                     cmk<C>(1, 0), X.p, X.ld);
    }
}
template <class C>
void ztrsm_luh(hm_handle_s *h, const C *U, int ldu, int n, MVT<C> X)
{
    if (n <= 2 * TRS_BLK) {
        trsm_left(h, 2, U, ldu, n, X);
        return;
    }
    // U^H is lower triangular: forward over blocks; (U^H)[rest, b] = (U[b, rest])^H
    for (int b0 = 0; b0 < n; b0 += TRS_BLK) {
        const int nb = std::min(TRS_BLK, n - b0), rest = n - b0 - nb;
        trsm_left(h, 2, U + b0 + (size_t)b0 * ldu, ldu, nb, MVT<C>{X.p + b0, nb, X.cols, X.ld});
        if (rest > 0)
            zgemm<C>(h, 'C', 'N', rest, X.cols, nb, cmk<C>(-1, 0), U + b0 + (size_t)(b0 + nb) * ldu, ldu, X.p + b0,
                     X.ld, cmk<C>(1, 0), X.p + b0 + nb, X.ld);
    }
}

// Explicit inverses of the triangular factors of a diagonal block: Li = L^-1 (unit lower)
// and Ui = U^-1 (upper), n x n with ld n, L and U read from T (ld ldt).  Blocked substitution
// on the identity restricted to the columns that can be nonzero: row block b of L^-1 has
// nonzeros only in columns [0, b1), row block b of U^-1 only in columns [b0, n) (half the
// work of a solve against the full identity).
template <class C>
void ztri_inverses(hm_handle_s *h, const C *T, int ldt, int n, C *Li, C *Ui)
{
    const size_t nn = (size_t)n * n;
    k_eye<C><<<(unsigned)((nn + 255) / 256), 256, 0, h->stream>>>(Li, n);
    HM_CHECK_LAUNCH();
    k_eye<C><<<(unsigned)((nn + 255) / 256), 256, 0, h->stream>>>(Ui, n);
    HM_CHECK_LAUNCH();
    count_launch(h, 2);
    for (int b0 = 0; b0 < n; b0 += TRS_BLK) {
        const int nb = std::min(TRS_BLK, n - b0), b1 = b0 + nb, rest = n - b1;
        trsm_left(h, 0, T + b0 + (size_t)b0 * ldt, ldt, nb, MVT<C>{Li + b0, nb, b1, n});
        if (rest > 0)
            zgemm<C>(h, 'N', 'N', rest, b1, nb, cmk<C>(-1, 0), T + b1 + (size_t)b0 * ldt, ldt, Li + b0, n,
                     cmk<C>(1, 0), Li + b1, n);
    }
    for (int b1 = n; b1 > 0; b1 -= TRS_BLK) {
        const int b0 = std::max(0, b1 - TRS_BLK), nb = b1 - b0;
        trsm_left(h, 1, T + b0 + (size_t)b0 * ldt, ldt, nb, MVT<C>{Ui + b0 + (size_t)b0 * n, nb, n - b0, n});
        if (b0 > 0)
            zgemm<C>(h, 'N', 'N', b0, n - b0, nb, cmk<C>(-1, 0), T + (size_t)b0 * ldt, ldt, Ui + b0 + (size_t)b0 * n,
                     n, cmk<C>(1, 0), Ui + (size_t)b0 * n, n);
    }
}

// X = X U^-1 (X rows x n): one thread per row, sequential over columns.
template <class C>
__global__ void k_trsm_right_upper(const C *__restrict__ U, int ldu, int n, C *X, int ldx, int rows)
{
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    for (int j = 0; j < n; ++j) {
        C s = X[(size_t)j * ldx + r];
        for (int i = 0; i < j; ++i) s = zsub(s, zmul(X[(size_t)i * ldx + r], U[(size_t)j * ldu + i]));
        X[(size_t)j * ldx + r] = zdiv(s, U[(size_t)j * ldu + j]);
    }
}

template <class C>
void ztrsm_run(hm_handle_s *h, const C *U, int ldu, int n, MVT<C> X)
{
    if (X.rows <= 0 || n <= 0) return;
    k_trsm_right_upper<C><<<(X.rows + 63) / 64, 64, 0, h->stream>>>(U, ldu, n, X.p, X.ld, X.rows);
    HM_CHECK_LAUNCH();
    count_launch(h);
    h->flops_factor += 4.0 * n * (double)n * X.rows;
}

template <class C>
__global__ void k_copy2d(C *dst, int ldd, const C *src, int lds, int rows, int cols)
{
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)rows * cols) return;
    int i = (int)(idx % rows), j = (int)(idx / rows);
    dst[(size_t)j * ldd + i] = src[(size_t)j * lds + i];
}

template <class C>
void zcopy2d(hm_handle_s *h, MVT<C> dst, MVT<C> src)
{
    size_t n = (size_t)src.rows * src.cols;
    if (n == 0) return;
    k_copy2d<C><<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(dst.p, dst.ld, src.p, src.ld, src.rows, src.cols);
    HM_CHECK_LAUNCH();
    count_launch(h);
}

template <class C>
__global__ void k_scale_cols(C *X, int ld, int rows, int cols, const typename CReal<C>::R *s)
{
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)rows * cols) return;
    int i = (int)(idx % rows), j = (int)(idx / rows);
    X[(size_t)j * ld + i] = zscale(X[(size_t)j * ld + i], s[j]);
}

template <class C>
void zscale_cols(hm_handle_s *h, MVT<C> X, const typename CReal<C>::R *d_s)
{
    size_t n = (size_t)X.rows * X.cols;
    if (n == 0) return;
    k_scale_cols<C><<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(X.p, X.ld, X.rows, X.cols, d_s);
    HM_CHECK_LAUNCH();
    count_launch(h);
}

// ---------------------------------------------------------------------------
// Householder QR, one CTA per matrix: A (m x K, ld m) -> Q (m x r), R (r x K), r = min(m, K).
// H_j = I - 2 v v^H / (v^H v), v = x - alpha e_1, alpha = -exp(i arg x_0) |x|, H_j x = alpha e_1.
// ---------------------------------------------------------------------------
template <class C>
struct QRDesc {
    C *A;        // input, overwritten (reflectors)
    int m, K;
    C *Q;        // m x r
    C *R;        // r x K
    typename CReal<C>::R *beta;  // workspace [r]
};

#define QR_T 512

template <class R>
__device__ R qr_block_sum(R v, R *sh)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffff, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        R s = 0;
        for (int w = 0; w < QR_T / 32; ++w) s += sh[w];
        sh[32] = s;
    }
    __syncthreads();
    R r = sh[32];
    __syncthreads();
    return r;
}

template <class C>
__global__ void __launch_bounds__(QR_T) k_qr(const QRDesc<C> *__restrict__ descs)
{
    typedef typename CReal<C>::R R;
    const QRDesc<C> d = descs[blockIdx.x];
    const int m = d.m, K = d.K, r = min(m, K);
    __shared__ R sh[33];
    __shared__ C s_alpha;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = QR_T / 32;
    C *A = d.A;
    for (int j = 0; j < r; ++j) {
        C *x = A + (size_t)j * m;
        R nrm2 = 0;
        for (int i = j + tid; i < m; i += QR_T) nrm2 += zabs2(x[i]);
        nrm2 = qr_block_sum(nrm2, sh);
        R nrm = sqrt(nrm2);
        if (tid == 0) {
            C x0 = x[j];
            R a0 = sqrt(zabs2(x0));
            C ph = a0 > 0 ? zscale(x0, (R)1 / a0) : cmk<C>(1, 0);
            C alpha = zscale(ph, -nrm);
            s_alpha = alpha;
            // v = x - alpha e1; v^H v = 2 (|x|^2 + |x| |x0|)
            x[j] = zsub(x0, alpha);
            R vhv = 2 * (nrm2 + nrm * a0);
            d.beta[j] = vhv > 0 ? 2 / vhv : 0;
        }
        __syncthreads();
        const R beta = d.beta[j];
        // apply H to columns c > j: a -= beta v (v^H a)
        for (int c = j + 1 + warp; c < K; c += nw) {
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
        // R row j
        if (tid == 0) d.R[(size_t)j * r + j] = s_alpha;
        for (int c = j + 1 + tid; c < K; c += QR_T) d.R[(size_t)c * r + j] = A[(size_t)c * m + j];
        for (int c = tid; c < j && c < K; c += QR_T) d.R[(size_t)c * r + j] = cmk<C>(0, 0);
        __syncthreads();
    }
    // Q = H_0 ... H_{r-1} [I_r; 0]
    for (int e = tid; e < m * r; e += QR_T) {
        int i = e % m, c = e / m;
        d.Q[(size_t)c * m + i] = cmk<C>(i == c ? 1 : 0, 0);
    }
    __syncthreads();
    for (int j = r - 1; j >= 0; --j) {
        const C *v = A + (size_t)j * m;
        const R beta = d.beta[j];
        for (int c = j + warp; c < r; c += nw) {
            C *q = d.Q + (size_t)c * m;
            C s = cmk<C>(0, 0);
            for (int i = j + lane; i < m; i += 32) s = zfmac(v[i], q[i], s);
            for (int o = 16; o > 0; o >>= 1) {
                s.x += __shfl_xor_sync(0xffffffff, s.x, o);
                s.y += __shfl_xor_sync(0xffffffff, s.y, o);
            }
            s = zscale(s, beta);
            for (int i = j + lane; i < m; i += 32) q[i] = zsub(q[i], zmul(v[i], s));
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// One-sided Jacobi SVD, one CTA per matrix: M (p x q, ld p) -> M Y = X Sigma with
// Y (q x q) unitary; on exit M holds X Sigma (orthogonal columns), S[j] = |col j|,
// ord[] = column order by decreasing S.  Round-robin pairs, one warp per pair.
// ---------------------------------------------------------------------------
template <class C>
struct SVDDesc {
    C *M;
    int p, q;
    C *Y;
    typename CReal<C>::R *S;
    int *ord;
};

// Real flops of a complex Householder QR of an M x K matrix, r = min(M, K) reflectors,
// with the explicit M x r Q: each reflector j updates the (M - j) x (K - j - 1) trailing
// block (8 real flops per complex multiply-add, two passes) and later the (M - j) x (r - j)
// block of Q.
static double householder_flops(int M, int K, int r)
{
    double f = 0;
    for (int j = 0; j < r; ++j) f += 16.0 * (M - j) * ((K - j - 1) + (r - j));
    return f;
}

// Relative size of an off-diagonal inner product below which a Jacobi rotation is skipped.
template <class R> __device__ __forceinline__ R jacobi_eps();
template <> __device__ __forceinline__ double jacobi_eps<double>() { return 1e-14; }
template <> __device__ __forceinline__ float jacobi_eps<float>() { return 1e-6f; }

#define SVD_T 512
#define SVD_QMAX 4096

template <class C>
__global__ void __launch_bounds__(SVD_T) k_svd(const SVDDesc<C> *__restrict__ descs)
{
    typedef typename CReal<C>::R R;
    const SVDDesc<C> d = descs[blockIdx.x];
    const int p = d.p, q = d.q;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = SVD_T / 32;
    __shared__ int s_rot;
    for (int e = tid; e < q * q; e += SVD_T) {
        int i = e % q, j = e / q;
        d.Y[(size_t)j * q + i] = cmk<C>(i == j ? 1 : 0, 0);
    }
    const int qe = (q + 1) & ~1;  // even count (a dummy column when q is odd)
    __syncthreads();
    // Round-robin ordering: position 0 holds column 0; in round r position k >= 1 holds
    // column 1 + ((k - 1 - r) mod (qe - 1)); round r pairs positions pr and qe - 1 - pr.
    for (int sweep = 0; sweep < 40; ++sweep) {
        if (tid == 0) s_rot = 0;
        __syncthreads();
        for (int round = 0; round < qe - 1; ++round) {
            for (int pr = warp; pr < qe / 2; pr += nw) {
                const int pa = pr, pb = qe - 1 - pr;
                int a = pa == 0 ? 0 : 1 + ((pa - 1 - round) % (qe - 1) + (qe - 1)) % (qe - 1);
                int b = 1 + ((pb - 1 - round) % (qe - 1) + (qe - 1)) % (qe - 1);
                if (a >= q || b >= q) continue;
                if (a > b) {
                    int t = a;
                    a = b;
                    b = t;
                }
                C *ca = d.M + (size_t)a * p, *cb = d.M + (size_t)b * p;
                R al = 0, be = 0;
                C ga = cmk<C>(0, 0);
                for (int i = lane; i < p; i += 32) {
                    al += zabs2(ca[i]);
                    be += zabs2(cb[i]);
                    ga = zfmac(ca[i], cb[i], ga);
                }
                for (int o = 16; o > 0; o >>= 1) {
                    al += __shfl_xor_sync(0xffffffff, al, o);
                    be += __shfl_xor_sync(0xffffffff, be, o);
                    ga.x += __shfl_xor_sync(0xffffffff, ga.x, o);
                    ga.y += __shfl_xor_sync(0xffffffff, ga.y, o);
                }
                R g = sqrt(zabs2(ga));
                if (!(g > jacobi_eps<R>() * sqrt(al * be)) || g == 0) continue;
                if (lane == 0) s_rot = 1;
                C eph = zscale(ga, (R)1 / g);  // exp(i phi)
                R zeta = (be - al) / (2 * g);
                R t = (zeta >= 0 ? (R)1 : (R)-1) / (fabs(zeta) + sqrt(1 + zeta * zeta));
                R c = 1 / sqrt(1 + t * t), s = c * t;
                C sem = zscale(zconj(eph), s), sep = zscale(eph, s);
                for (int i = lane; i < p; i += 32) {
                    C x = ca[i], y = cb[i];
                    ca[i] = zsub(zscale(x, c), zmul(sem, y));
                    cb[i] = zadd(zmul(sep, x), zscale(y, c));
                }
                C *ya = d.Y + (size_t)a * q, *yb = d.Y + (size_t)b * q;
                for (int i = lane; i < q; i += 32) {
                    C x = ya[i], y = yb[i];
                    ya[i] = zsub(zscale(x, c), zmul(sem, y));
                    yb[i] = zadd(zmul(sep, x), zscale(y, c));
                }
            }
            __syncthreads();
        }
        if (!s_rot) break;
        __syncthreads();
    }
    for (int j = warp; j < q; j += nw) {
        R s = 0;
        for (int i = lane; i < p; i += 32) s += zabs2(d.M[(size_t)j * p + i]);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffff, s, o);
        if (lane == 0) d.S[j] = sqrt(s);
    }
    __syncthreads();
    // order by decreasing S (ties: lower index first): each column's rank is the number
    // of columns that precede it; a NaN norm sorts last so that ord stays a permutation
    for (int j = tid; j < q; j += SVD_T) {
        const R sj = d.S[j] == d.S[j] ? d.S[j] : (R)-1;
        int rank = 0;
        for (int i = 0; i < q; ++i) {
            const R si = d.S[i] == d.S[i] ? d.S[i] : (R)-1;
            rank += (si > sj) || (si == sj && i < j);
        }
        d.ord[rank] = j;
    }
}

// Assemble the truncated factors: Uo[:, t] = Q_U * (X col ord[t]) / S * sqrt(S) ... done as
// gather + scale: G[:, t] = M[:, ord[t]] * f(S), H[:, t] = Y[:, ord[t]] * sqrt(S)
template <class C>
__global__ void k_gather_cols(const C *M, int p, const int *ord, const typename CReal<C>::R *S, int kk, int q, C *G,
                              int mode)
{
    typedef typename CReal<C>::R R;
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)p * kk) return;
    int i = (int)(idx % p), t = (int)(idx / p);
    int c = ord[t];
    if (c < 0 || c >= q) {  // never taken after the host's check of ord; keeps the access in bounds
        G[(size_t)t * p + i] = cmk<C>(0, 0);
        return;
    }
    R s = S[c];
    R f;
    if (mode == 0)
        f = s > 0 ? 1 / sqrt(s) : 0;  // X Sigma -> X sqrt(Sigma)
    else
        f = sqrt(s);  // Y -> Y sqrt(Sigma)
    G[(size_t)t * p + i] = zscale(M[(size_t)c * p + i], f);
}

// ---------------------------------------------------------------------------
// Column-pivoted Householder QR of the core, stopped at the Frobenius tolerance
// (the complex64 factor's truncation), one CTA per core M (p x q, ld p):
//   M Pi = Q R;  stop at the first j with sum_{l >= j} |trailing column l|^2 <= tol2 |M|_F^2,
// so |M - Q[:, :k] R[:k, :] Pi^T|_F <= tol |M|_F with k the returned rank.
// Outputs: Qc (p x k) explicit, W (q x k) = (R[:k, :] Pi^T)^H, *rank = k.
// Scratch (global): cn [q] column norms, perm [q], beta [min(p, q)], diag [min(p, q)].
// ---------------------------------------------------------------------------
template <class C>
struct QRCPDesc {
    C *M;
    int p, q;
    C *Qc, *W;
    typename CReal<C>::R *cn, *beta, *diag_re, *diag_im;
    int *perm;
    int *rank;
};

template <class R>
__device__ R qrcp_sum(R v, R *sh)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffff, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        R s = 0;
        for (int w = 0; w < QR_T / 32; ++w) s += sh[w];
        sh[32] = s;
    }
    __syncthreads();
    R r = sh[32];
    __syncthreads();
    return r;
}

template <class C>
__global__ void __launch_bounds__(QR_T) k_qrcp(const QRCPDesc<C> *__restrict__ descs, double tol2)
{
    typedef typename CReal<C>::R R;
    const QRCPDesc<C> d = descs[blockIdx.x];
    const int p = d.p, q = d.q, r = min(p, q);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = QR_T / 32;
    __shared__ R sh[33];
    __shared__ R shv[QR_T / 32];
    __shared__ int shi[QR_T / 32];
    __shared__ int s_piv;
    C *M = d.M;
    // column norms and the identity permutation
    for (int l = warp; l < q; l += nw) {
        R s = 0;
        for (int i = lane; i < p; i += 32) s += zabs2(M[(size_t)l * p + i]);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffff, s, o);
        if (lane == 0) {
            d.cn[l] = s;
            d.perm[l] = l;
        }
    }
    __syncthreads();
    R part = 0;
    for (int l = tid; l < q; l += QR_T) part += d.cn[l];
    const R total = qrcp_sum(part, sh);
    int k = 0;
    for (int j = 0; j < r; ++j) {
        // remaining squared Frobenius norm and the pivot column (largest, ties to lowest)
        R rem = 0, bv = -1;
        int bi = 0x7fffffff;
        for (int l = j + tid; l < q; l += QR_T) {
            R c = d.cn[l];
            rem += c;
            if (c > bv) {
                bv = c;
                bi = l;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            R v2 = __shfl_down_sync(0xffffffff, bv, o);
            int i2 = __shfl_down_sync(0xffffffff, bi, o);
            if (v2 > bv || (v2 == bv && i2 < bi)) {
                bv = v2;
                bi = i2;
            }
        }
        if (lane == 0) {
            shv[warp] = bv;
            shi[warp] = bi;
        }
        rem = qrcp_sum(rem, sh);  // contains the barriers that publish shv / shi
        if (tid == 0) {
            R v = shv[0];
            int ii = shi[0];
            for (int w = 1; w < nw; ++w)
                if (shv[w] > v || (shv[w] == v && shi[w] < ii)) {
                    v = shv[w];
                    ii = shi[w];
                }
            s_piv = ii;
        }
        __syncthreads();
        if (!(rem > (R)tol2 * total)) break;
        const int pv = s_piv;
        if (pv != j) {
            for (int i = tid; i < p; i += QR_T) {
                C t = M[(size_t)j * p + i];
                M[(size_t)j * p + i] = M[(size_t)pv * p + i];
                M[(size_t)pv * p + i] = t;
            }
            if (tid == 0) {
                R t = d.cn[j];
                d.cn[j] = d.cn[pv];
                d.cn[pv] = t;
                int tp = d.perm[j];
                d.perm[j] = d.perm[pv];
                d.perm[pv] = tp;
            }
            __syncthreads();
        }
        // Householder reflector of M[j:, j]
        C *x = M + (size_t)j * p;
        R nrm2 = 0;
        for (int i = j + tid; i < p; i += QR_T) nrm2 += zabs2(x[i]);
        nrm2 = qrcp_sum(nrm2, sh);
        if (tid == 0) {
            R nrm = sqrt(nrm2);
            C x0 = x[j];
            R a0 = sqrt(zabs2(x0));
            C ph = a0 > 0 ? zscale(x0, (R)1 / a0) : cmk<C>(1, 0);
            C alpha = zscale(ph, -nrm);
            x[j] = zsub(x0, alpha);
            R vhv = 2 * (nrm2 + nrm * a0);
            d.beta[j] = vhv > 0 ? 2 / vhv : 0;
            d.diag_re[j] = alpha.x;
            d.diag_im[j] = alpha.y;
        }
        __syncthreads();
        const R beta = d.beta[j];
        // apply to the trailing columns and recompute their norms below row j
        for (int l = j + 1 + warp; l < q; l += nw) {
            C *a = M + (size_t)l * p;
            C s = cmk<C>(0, 0);
            for (int i = j + lane; i < p; i += 32) s = zfmac(x[i], a[i], s);
            for (int o = 16; o > 0; o >>= 1) {
                s.x += __shfl_xor_sync(0xffffffff, s.x, o);
                s.y += __shfl_xor_sync(0xffffffff, s.y, o);
            }
            s = zscale(s, beta);
            R nn = 0;
            for (int i = j + lane; i < p; i += 32) {
                C v = zsub(a[i], zmul(x[i], s));
                a[i] = v;
                if (i > j) nn += zabs2(v);
            }
            for (int o = 16; o > 0; o >>= 1) nn += __shfl_xor_sync(0xffffffff, nn, o);
            if (lane == 0) d.cn[l] = nn;
        }
        __syncthreads();
        k = j + 1;
    }
    if (tid == 0) *d.rank = k;
    if (k == 0) return;
    // W (q x k): W[perm[l], t] = conj(R[t, l]),  R[t, l] = M[t, l] (t < l), alpha_t (t = l), 0 (t > l)
    for (int e = tid; e < q * k; e += QR_T) {
        const int l = e % q, t = e / q;
        C v = t < l ? M[(size_t)l * p + t] : (t == l ? cmk<C>(d.diag_re[t], d.diag_im[t]) : cmk<C>(0, 0));
        d.W[(size_t)t * q + d.perm[l]] = zconj(v);
    }
    // Qc (p x k) = H_0 ... H_{k-1} [I_k; 0]
    for (int e = tid; e < p * k; e += QR_T) {
        const int i = e % p, c = e / p;
        d.Qc[(size_t)c * p + i] = cmk<C>(i == c ? 1 : 0, 0);
    }
    __syncthreads();
    for (int j = k - 1; j >= 0; --j) {
        const C *v = M + (size_t)j * p;
        const R beta = d.beta[j];
        for (int c = j + warp; c < k; c += nw) {
            C *qc = d.Qc + (size_t)c * p;
            C s = cmk<C>(0, 0);
            for (int i = j + lane; i < p; i += 32) s = zfmac(v[i], qc[i], s);
            for (int o = 16; o > 0; o >>= 1) {
                s.x += __shfl_xor_sync(0xffffffff, s.x, o);
                s.y += __shfl_xor_sync(0xffffffff, s.y, o);
            }
            s = zscale(s, beta);
            for (int i = j + lane; i < p; i += 32) qc[i] = zsub(qc[i], zmul(v[i], s));
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Truncated recompression of U V^H (batched): QR of both factors, SVD of the core
// R_U R_V^H, keep the smallest rank k' with sqrt(sum_{i>k'} s_i^2) <= tol |s|_2.
// ---------------------------------------------------------------------------
// Core factorisation of a truncation: column-pivoted QR stopped at the tolerance (the
// complex64 factor, and every recompression inside an H-LU) or one-sided Jacobi SVD (the
// recompression of the complex128 H-matrix after ACA).
template <class C>
static bool use_qrcp(const hm_handle_s *h)
{
    return std::is_same<C, cf>::value || h->d_info_cur != nullptr;
}

template <class C>
struct TruncJob {
    typedef typename CReal<C>::R R;
    int m, n, K;
    const C *U;
    int ldu;
    const C *V;
    int ldv;
    int kmax;
    // work
    C *Ua, *Va, *QU, *QV, *RU, *RV, *Mc, *Y;
    R *bU, *bV, *S;
    int *ord;
    int r1, r2;
};

template <class C>
static void trunc_stage1(hm_handle_s *h, std::vector<TruncJob<C>> &jobs)
{
    typedef typename CReal<C>::R R;
    const bool qrcp = use_qrcp<C>(h);
    // workspace and copies
    std::vector<QRJob<C>> qd;
    for (auto &J : jobs) {
        J.r1 = std::min(J.m, J.K);
        J.r2 = std::min(J.n, J.K);
        J.Ua = (C *)dalloc(h, sizeof(C) * (size_t)J.m * J.K);
        J.Va = (C *)dalloc(h, sizeof(C) * (size_t)J.n * J.K);
        J.QU = (C *)dalloc(h, sizeof(C) * (size_t)J.m * J.r1);
        J.QV = (C *)dalloc(h, sizeof(C) * (size_t)J.n * J.r2);
        J.RU = (C *)dalloc(h, sizeof(C) * (size_t)J.r1 * J.K);
        J.RV = (C *)dalloc(h, sizeof(C) * (size_t)J.r2 * J.K);
        J.Mc = (C *)dalloc(h, sizeof(C) * (size_t)J.r1 * J.r2);
        J.Y = qrcp ? nullptr : (C *)dalloc(h, sizeof(C) * (size_t)J.r2 * J.r2);
        J.bU = (R *)dalloc(h, sizeof(R) * (J.r1 + 3 * J.r2));
        J.bV = J.bU + J.r1;
        J.S = J.bV + J.r2;
        J.ord = (int *)dalloc(h, sizeof(int) * (J.r2 + 1));
        zcopy2d(h, MVT<C>{J.Ua, J.m, J.K, J.m}, MVT<C>{(C *)J.U, J.m, J.K, J.ldu});
        zcopy2d(h, MVT<C>{J.Va, J.n, J.K, J.n}, MVT<C>{(C *)J.V, J.n, J.K, J.ldv});
        qd.push_back(QRJob<C>{J.Ua, J.m, J.K, J.QU, J.RU});
        qd.push_back(QRJob<C>{J.Va, J.n, J.K, J.QV, J.RV});
        h->flops_factor += 16.0 * ((double)J.m + J.n) * J.K * J.K;
    }
    for (int e = 0; e < 4; ++e)
        if (!h->ev[e]) HM_CUDA(cudaEventCreate(&h->ev[e]));
    HM_CUDA(cudaEventRecord(h->ev[0], h->stream));
    batched_qr<C>(h, qd);
    HM_CUDA(cudaEventRecord(h->ev[1], h->stream));
    for (auto &J : jobs) h->kqr_flops += householder_flops(J.m, J.K, J.r1) + householder_flops(J.n, J.K, J.r2);
    // core M = R_U R_V^H
    for (auto &J : jobs)
        zgemm<C>(h, 'N', 'C', J.r1, J.r2, J.K, cmk<C>(1, 0), J.RU, J.r1, J.RV, J.r2, cmk<C>(0, 0), J.Mc, J.r1);
    void *d_desc = nullptr;
    if (qrcp) {
        // complex64 factor: column-pivoted QR of the core, stopped at the tolerance;
        // Qc -> RU, W -> RV (both large enough), scratch in bU/bV/S, perm and rank in ord
        std::vector<QRCPDesc<C>> cd;
        for (auto &J : jobs)
            cd.push_back(QRCPDesc<C>{J.Mc, J.r1, J.r2, J.RU, J.RV, J.S, J.bU, J.bV, J.S + J.r2, J.ord,
                                     J.ord + J.r2});
        d_desc = dalloc(h, sizeof(QRCPDesc<C>) * cd.size());
        HM_CUDA(cudaMemcpyAsync(d_desc, cd.data(), sizeof(QRCPDesc<C>) * cd.size(), cudaMemcpyHostToDevice,
                                h->stream));
        HM_CUDA(cudaEventRecord(h->ev[2], h->stream));
        k_qrcp<C><<<(unsigned)cd.size(), QR_T, 0, h->stream>>>((const QRCPDesc<C> *)d_desc, h->cur_tol * h->cur_tol);
    } else {
        std::vector<SVDDesc<C>> sd;
        for (auto &J : jobs) sd.push_back(SVDDesc<C>{J.Mc, J.r1, J.r2, J.Y, J.S, J.ord});
        int qmax = 0;
        for (auto &J : jobs) qmax = std::max(qmax, J.r2);
        if (qmax > SVD_QMAX) throw HmError{HM_ERR_NUMERIC, "recompression core too large: " + std::to_string(qmax)};
        d_desc = dalloc(h, sizeof(SVDDesc<C>) * sd.size());
        HM_CUDA(cudaMemcpyAsync(d_desc, sd.data(), sizeof(SVDDesc<C>) * sd.size(), cudaMemcpyHostToDevice, h->stream));
        HM_CUDA(cudaEventRecord(h->ev[2], h->stream));
        k_svd<C><<<(unsigned)sd.size(), SVD_T, 0, h->stream>>>((const SVDDesc<C> *)d_desc);
    }
    HM_CHECK_LAUNCH();
    HM_CUDA(cudaEventRecord(h->ev[3], h->stream));
    count_launch(h);
    dfree(h, d_desc);  // stream-ordered: released after the kernel
}

// QRCP variant of stage 2: U' = Q_U Qc, V' = Q_V W with the rank the kernel chose.
template <class C>
static int trunc_stage2_qrcp(hm_handle_s *h, TruncJob<C> &J, int kk, C **Uo, C **Vo)
{
    *Uo = nullptr;
    *Vo = nullptr;
    if (kk > 0) {
        *Uo = (C *)dalloc(h, sizeof(C) * (size_t)J.m * kk);
        *Vo = (C *)dalloc(h, sizeof(C) * (size_t)J.n * kk);
        zgemm<C>(h, 'N', 'N', J.m, kk, J.r1, cmk<C>(1, 0), J.QU, J.m, J.RU, J.r1, cmk<C>(0, 0), *Uo, J.m);
        zgemm<C>(h, 'N', 'N', J.n, kk, J.r2, cmk<C>(1, 0), J.QV, J.n, J.RV, J.r2, cmk<C>(0, 0), *Vo, J.n);
    }
    dfree(h, J.Ua);
    dfree(h, J.Va);
    dfree(h, J.QU);
    dfree(h, J.QV);
    dfree(h, J.RU);
    dfree(h, J.RV);
    dfree(h, J.Mc);
    dfree(h, J.bU);
    dfree(h, J.ord);
    return kk;
}

// After the batch's synchronisation: accumulate the device times of its two kernels.
static void account_kernels(hm_handle_s *h)
{
    float a = 0, b = 0;
    HM_CUDA(cudaEventElapsedTime(&a, h->ev[0], h->ev[1]));
    HM_CUDA(cudaEventElapsedTime(&b, h->ev[2], h->ev[3]));
    h->kqr_s += 1e-3 * a;
    h->kqr_n += 1;
    h->kcore_s += 1e-3 * b;
    h->kcore_n += 1;
}

// returns the kept rank; allocates *Uo (m x k'), *Vo (n x k')
template <class C>
static int trunc_stage2(hm_handle_s *h, TruncJob<C> &J, const std::vector<double> &S, const std::vector<int> &ord,
                        double tol, C **Uo, C **Vo)
{
    for (size_t t = 0; t < S.size(); ++t)
        if (!std::isfinite(S[t]) || ord[t] < 0 || ord[t] >= (int)S.size())
            throw HmError{HM_ERR_NUMERIC, "recompression of a block with non-finite values"};
    double tot = 0;
    for (double s : S) tot += s * s;
    int kk = (int)S.size();
    double tail = 0;
    while (kk > 0) {
        double s = S[ord[kk - 1]];
        if (tail + s * s > tol * tol * tot) break;
        tail += s * s;
        --kk;
    }
    if (tot == 0.0) kk = 0;
    kk = std::min(kk, J.kmax > 0 ? J.kmax : kk);
    C *G = nullptr, *Hh = nullptr;
    *Uo = nullptr;
    *Vo = nullptr;
    if (kk > 0) {
        G = (C *)dalloc(h, sizeof(C) * (size_t)J.r1 * kk);
        Hh = (C *)dalloc(h, sizeof(C) * (size_t)J.r2 * kk);
        size_t n1 = (size_t)J.r1 * kk, n2 = (size_t)J.r2 * kk;
        k_gather_cols<C><<<(unsigned)((n1 + 255) / 256), 256, 0, h->stream>>>(J.Mc, J.r1, J.ord, J.S, kk, J.r2, G, 0);
        k_gather_cols<C><<<(unsigned)((n2 + 255) / 256), 256, 0, h->stream>>>(J.Y, J.r2, J.ord, J.S, kk, J.r2, Hh, 1);
        HM_CHECK_LAUNCH();
        count_launch(h, 2);
        *Uo = (C *)dalloc(h, sizeof(C) * (size_t)J.m * kk);
        *Vo = (C *)dalloc(h, sizeof(C) * (size_t)J.n * kk);
        zgemm<C>(h, 'N', 'N', J.m, kk, J.r1, cmk<C>(1, 0), J.QU, J.m, G, J.r1, cmk<C>(0, 0), *Uo, J.m);
        zgemm<C>(h, 'N', 'N', J.n, kk, J.r2, cmk<C>(1, 0), J.QV, J.n, Hh, J.r2, cmk<C>(0, 0), *Vo, J.n);
        dfree(h, G);
        dfree(h, Hh);
    }
    dfree(h, J.Ua);
    dfree(h, J.Va);
    dfree(h, J.QU);
    dfree(h, J.QV);
    dfree(h, J.RU);
    dfree(h, J.RV);
    dfree(h, J.Mc);
    dfree(h, J.Y);
    dfree(h, J.bU);
    dfree(h, J.ord);
    return kk;
}

// During an H-LU the zero-pivot flag of the diagonal leaves is read at every
// synchronisation of a recompression batch, so a singular leaf stops the factorisation
// before its non-finite values reach a rank decision.
static void check_pivots(hm_handle_s *h)
{
    if (!h->d_info_cur) return;
    int info = 0;
    HM_CUDA(cudaMemcpy(&info, h->d_info_cur, sizeof(int), cudaMemcpyDeviceToHost));
    if (info) throw HmError{HM_ERR_SINGULAR, "H-LU: zero pivot in a diagonal leaf"};
}

template <class C>
static void fetch_sv(hm_handle_s *h, std::vector<TruncJob<C>> &jobs, std::vector<std::vector<double>> &S,
                     std::vector<std::vector<int>> &ord)
{
    typedef typename CReal<C>::R R;
    S.resize(jobs.size());
    ord.resize(jobs.size());
    if (use_qrcp<C>(h)) {
        // QRCP: only the chosen ranks come back (ord[i][0])
        std::vector<int> rk(jobs.size());
        for (size_t i = 0; i < jobs.size(); ++i)
            HM_CUDA(cudaMemcpyAsync(&rk[i], jobs[i].ord + jobs[i].r2, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
        HM_CUDA(cudaStreamSynchronize(h->stream));
        check_pivots(h);
        for (size_t i = 0; i < jobs.size(); ++i) {
            if (rk[i] < 0 || rk[i] > std::min(jobs[i].r1, jobs[i].r2))
                throw HmError{HM_ERR_NUMERIC, "recompression rank out of range"};
            ord[i].assign(1, rk[i]);
        }
        return;
    }
    std::vector<std::vector<R>> Sr(jobs.size());
    for (size_t i = 0; i < jobs.size(); ++i) {
        Sr[i].resize(jobs[i].r2);
        ord[i].resize(jobs[i].r2);
        HM_CUDA(cudaMemcpyAsync(Sr[i].data(), jobs[i].S, sizeof(R) * jobs[i].r2, cudaMemcpyDeviceToHost, h->stream));
        HM_CUDA(cudaMemcpyAsync(ord[i].data(), jobs[i].ord, sizeof(int) * jobs[i].r2, cudaMemcpyDeviceToHost, h->stream));
    }
    HM_CUDA(cudaStreamSynchronize(h->stream));
    check_pivots(h);
    for (size_t i = 0; i < jobs.size(); ++i) S[i].assign(Sr[i].begin(), Sr[i].end());
}


// Recompress the low-rank leaves blks (U, V with ranks[i] columns) in one batch;
// replaces b->U, b->V, b->k.
template <class C>
void batched_truncate(hm_handle_s *h, std::vector<BlockT<C> *> &blks, const std::vector<int> &ranks, double tol)
{
    const size_t CH = 512;  // jobs per batch (bounds the workspace)
    auto t0 = std::chrono::steady_clock::now();
    for (size_t s = 0; s < blks.size(); s += CH) {
        size_t e = std::min(blks.size(), s + CH);
        std::vector<TruncJob<C>> jobs;
        std::vector<size_t> idx;
        for (size_t i = s; i < e; ++i) {
            BlockT<C> *b = blks[i];
            if (ranks[i] <= 0) continue;
            TruncJob<C> J{};
            J.m = b->nr;
            J.n = b->nc;
            J.K = ranks[i];
            J.U = b->U;
            J.ldu = b->nr;
            J.V = b->V;
            J.ldv = b->nc;
            J.kmax = 0;
            jobs.push_back(J);
            idx.push_back(i);
        }
        if (jobs.empty()) continue;
        auto tb = std::chrono::steady_clock::now();
        h->tr_batches += 1;
        h->tr_jobs += (double)jobs.size();
        double bmm = 0, bmk = 0, bw = 0;
        for (auto &J : jobs) {
            h->tr_maxk = std::max(h->tr_maxk, (double)J.K);
            h->tr_work += ((double)J.m + J.n) * J.K * J.K;
            bmm = std::max(bmm, (double)std::max(J.m, J.n));
            bmk = std::max(bmk, (double)J.K);
            bw += ((double)J.m + J.n) * J.K * J.K;
        }
        const double q0 = h->kqr_s, c0 = h->kcore_s;
        double saved = h->cur_tol;
        h->cur_tol = tol;
        trunc_stage1(h, jobs);
        h->cur_tol = saved;
        std::vector<std::vector<double>> S;
        std::vector<std::vector<int>> ord;
        fetch_sv(h, jobs, S, ord);
        account_kernels(h);
        if (use_qrcp<C>(h))
            for (size_t t = 0; t < jobs.size(); ++t) h->kcore_flops += householder_flops(jobs[t].r1, jobs[t].r2, ord[t][0]);
        for (size_t t = 0; t < jobs.size(); ++t) {
            BlockT<C> *b = blks[idx[t]];
            C *Uo, *Vo;
            int kk = use_qrcp<C>(h) ? trunc_stage2_qrcp(h, jobs[t], ord[t][0], &Uo, &Vo)
                                                : trunc_stage2(h, jobs[t], S[t], ord[t], tol, &Uo, &Vo);
            dfree(h, b->U);
            dfree(h, b->V);
            b->U = Uo;
            b->V = Vo;
            b->k = kk;
        }
        const double wall = std::chrono::duration<double>(std::chrono::steady_clock::now() - tb).count();
        const double rec[7] = {(double)jobs.size(), bmm, bmk, bw, h->kqr_s - q0, h->kcore_s - c0, wall};
        h->trunc_log.insert(h->trunc_log.end(), rec, rec + 7);
    }
    h->tr_seconds += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

// ---------------------------------------------------------------------------
// Explicit instantiations: complex128 (the FP64 method) and complex64 (the FP32
// factor used as a preconditioner).
// ---------------------------------------------------------------------------
#define HM_INST_LINALG(C)                                                                                         \
    template void zgemm<C>(hm_handle_s *, char, char, int, int, int, C, const C *, int, const C *, int, C, C *, int); \
    template void zgetrf<C>(hm_handle_s *, int, C *, int, int *, int *);                                          \
    template void zlaswp<C>(hm_handle_s *, MVT<C>, const int *, int);                                             \
    template void ztrsm_lln<C>(hm_handle_s *, const C *, int, int, MVT<C>);                                       \
    template void ztrsm_lun<C>(hm_handle_s *, const C *, int, int, MVT<C>);                                       \
    template void ztrsm_luh<C>(hm_handle_s *, const C *, int, int, MVT<C>);                                       \
    template void ztrsm_run<C>(hm_handle_s *, const C *, int, int, MVT<C>);                                       \
    template void ztri_inverses<C>(hm_handle_s *, const C *, int, int, C *, C *);                                 \
    template void zcopy2d<C>(hm_handle_s *, MVT<C>, MVT<C>);                                                      \
    template void zscale_cols<C>(hm_handle_s *, MVT<C>, const typename CReal<C>::R *);                            \
    template void batched_truncate<C>(hm_handle_s *, std::vector<BlockT<C> *> &, const std::vector<int> &, double);
HM_INST_LINALG(zc)
HM_INST_LINALG(cf)
