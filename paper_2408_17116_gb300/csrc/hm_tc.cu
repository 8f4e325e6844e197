// Complex64 GEMM on the 5th-generation tensor cores (tcgen05, sm_103a) for the dense
// products of the FP32 H-LU: the Schur-complement updates A22 -= L21 U12 of the merged
// dense blocks and of the blocked LU (Sec. III, Eq. 23, formatted arithmetic on the
// dense leaves).
//
// Precision: each FP32 operand is split into two BF16 parts, a = a_hi + a_lo
// (a_hi = bf16(a), a_lo = bf16(a - a_hi)), and the product is taken as
// a_hi b_hi + a_hi b_lo + a_lo b_hi with FP32 accumulation (the split-BF16 scheme of
// Ootomo & Yokota, 2022): the dropped term a_lo b_lo and the rounding of the parts leave
// a relative error of about 2^-16 per product, below the truncation tolerance of the
// FP32 factor; FP64 iterative refinement removes it from the solution.
//
// Complex arithmetic as one real product: op(A) (m x k complex, column-major) is the
// real matrix Ar (2m x k) whose rows alternate real and imaginary parts; op(B)^T gives
// Br (2n x k) the same way.  P = Ar Br^T (2m x 2n) holds the four real products
// P[2i + a][2j + b] = (A_a B_b)[i][j], a, b in {re, im}, and the epilogue forms
// C[i][j] = alpha ((P_rr - P_ii) + i (P_ri + P_ir)) + beta C[i][j].  8 m n k real
// multiply-adds as in the 4-real-product form, in one contraction of depth k.
//
// Data path: a pack kernel writes the BF16 parts of both operands K-major
// ([rows][hi k | lo k], k padded to 64); the GEMM kernel streams 128 x 64 tiles of Ar and
// 256 x 64 tiles of Br with TMA (128-byte swizzle) through a 4-stage mbarrier pipeline,
// one thread issues tcgen05.mma (M = 128, N = 256, K = 16, BF16 in, FP32 accumulator in
// TMEM), and four warps read the accumulator back with tcgen05.ld for the complex
// epilogue.  Every mbarrier wait is bounded (2 s of globaltimer); on expiry the kernel
// records HM_ERR_TIMEOUT in a device flag, skips its stores, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "hm_internal.h"

#define TC_BM 128  // real rows of Ar per tile (64 complex rows)
#define TC_BN 256  // real rows of Br per tile (128 complex columns of C)
#define TC_BK 64   // BF16 elements of K per stage: one 128-byte swizzle row
#define TC_T 128   // four warps: one per TMEM lane quarter
#define TC_KC 2048 // complex K per packed chunk (bounds the workspace)

static constexpr int TC_A_BYTES = TC_BM * TC_BK * 2;
static constexpr int TC_B_BYTES = TC_BN * TC_BK * 2;
static constexpr int TC_STAGE_BYTES = TC_A_BYTES + TC_B_BYTES;
// pipeline stages: 4 (one CTA per SM) for deep products, 2 for shallow ones (K <= 512), where
// two CTAs per SM let one CTA's epilogue overlap the other's main loop
template <int ST>
constexpr int tc_smem() { return ST * TC_STAGE_BYTES + 1024 /* alignment */ + 256 /* barriers */; }

// ---------------------------------------------------------------------------
// pack: out[(2r + c) * 2kp + p] = hi part, out[(2r + c) * 2kp + kp + p] = lo part of
// component c of op(X)[r][p]; op(X)[r][p] = X[r + p ld] (rc) or X[p + r ld], conjugated
// when cj.  Columns p in [k, kp) are zero.  32 x 32 tiles transposed through shared memory.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_tc_pack(const float2 *__restrict__ X, int ld, int rows, int k, int kp, int rc,
                                                 int cj, __nv_bfloat16 *__restrict__ out)
{
    __shared__ float2 t[32][33];
    const int r0 = blockIdx.y * 32, p0 = blockIdx.x * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;
    for (int q = ty; q < 32; q += 8) {
        const int a = rc ? tx : q, b = rc ? q : tx;  // lanes along the contiguous index
        const int r = r0 + a, p = p0 + b;
        float2 v = make_float2(0.f, 0.f);
        if (r < rows && p < k) v = rc ? X[(size_t)p * ld + r] : X[(size_t)r * ld + p];
        if (cj) v.y = -v.y;
        t[a][b] = v;
    }
    __syncthreads();
    const size_t row = 2 * (size_t)kp;
    for (int a = ty; a < 32; a += 8) {
        const int r = r0 + a;
        if (r >= rows) continue;
        const int p = p0 + tx;
        const float2 v = t[a][tx];
        const __nv_bfloat16 hr = __float2bfloat16_rn(v.x), hi = __float2bfloat16_rn(v.y);
        const __nv_bfloat16 lr = __float2bfloat16_rn(v.x - __bfloat162float(hr));
        const __nv_bfloat16 li = __float2bfloat16_rn(v.y - __bfloat162float(hi));
        __nv_bfloat16 *o = out + (size_t)(2 * r) * row;
        o[p] = hr;
        o[kp + p] = lr;
        o[row + p] = hi;
        o[row + kp + p] = li;
    }
}

// ---------------------------------------------------------------------------
// PTX wrappers (tcgen05, TMA, mbarrier)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ uint64_t globaltimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait until the phase of parity `parity` of the barrier has completed; false (and the
// flag set) when 2 s pass first.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int *err)
{
    uint64_t t0 = 0;
    for (uint32_t it = 0;; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
        if ((it & 255) == 0) {
            const uint64_t now = globaltimer();
            if (it == 0)
                t0 = now;
            else if (now - t0 > 2000000000ull) {
                atomicCAS(err, 0, (int)HM_ERR_TIMEOUT);
                return false;
            }
        }
    }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor of a K-major tile with 128-byte rows, 128-byte swizzle:
// 8-row groups 1024 bytes apart (stride byte offset), descriptor version 1 (sm_100 family).
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)1 << 16;             // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;   // stride byte offset
    d |= (uint64_t)1 << 46;             // version
    d |= (uint64_t)2 << 61;             // 128-byte swizzle
    return d;
}

// Instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both K-major,
// N = TC_BN, M = TC_BM.
__host__ __device__ constexpr uint32_t tc_idesc()
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TC_BN >> 3) << 17) | ((uint32_t)(TC_BM >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Epilogue of one warp: accumulator lanes of real rows R (this lane) of a 128 x 256 tile whose
// TMEM lane quarter starts at taddr, accumulator columns [cbeg, cend); C = alpha P + beta C
// for the tile's complex columns from n0 / 2.  Warp-collective (tcgen05.ld): all 32 lanes,
// converged.
__device__ __forceinline__ void tc_store_rows(uint32_t taddr, int R, int m, int n, int n0, float2 alpha, float2 beta,
                                              float2 *__restrict__ Cm, int ldc, int cbeg = 0, int cend = TC_BN)
{
    const int gi = R >> 1;  // complex row of C
    const bool odd = threadIdx.x & 1;
    for (int c0 = cbeg; c0 < cend; c0 += 32) {
        uint32_t v[32];
        tmem_ld32(taddr + (uint32_t)c0, v);
        // even lane (real part of op(A)): P_r* of complex columns q = 0..15 of this chunk;
        // odd lane: P_i*.  The even lane finishes columns 0..7, the odd lane 8..15.
        float mine[16], other[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const float send = __uint_as_float(odd ? v[q] : v[16 + q]);
            other[q] = __shfl_xor_sync(0xffffffffu, send, 1);
            mine[q] = __uint_as_float(odd ? v[16 + q] : v[q]);
        }
        const int jb = (n0 + c0) / 2 + (odd ? 8 : 0);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const float prr = odd ? other[2 * q] : mine[2 * q];
            const float pri = odd ? other[2 * q + 1] : mine[2 * q + 1];
            const float pir = odd ? mine[2 * q] : other[2 * q];
            const float pii = odd ? mine[2 * q + 1] : other[2 * q + 1];
            const float cr = prr - pii, ci = pri + pir;
            const int j = jb + q;
            if (gi < m && j < n) {
                float2 *cp = Cm + (size_t)j * ldc + gi;
                float2 o = make_float2(alpha.x * cr - alpha.y * ci, alpha.x * ci + alpha.y * cr);
                if (beta.x != 0.f || beta.y != 0.f) {
                    const float2 c = *cp;
                    o.x += beta.x * c.x - beta.y * c.y;
                    o.y += beta.x * c.y + beta.y * c.x;
                }
                *cp = o;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// GEMM: C (m x n complex, ld ldc) = alpha P + beta C for the tile (blockIdx.x, blockIdx.y)
// of P = Ar Br^T, with K = 3 kp (passes hi.hi, hi.lo, lo.hi over the packed operands).
// ---------------------------------------------------------------------------
template <int TC_ST>
__global__ void __launch_bounds__(TC_T, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int m, int n, int kp,
              float2 alpha, float2 beta, float2 *__restrict__ Cm, int ldc, int *err)
{
    extern __shared__ __align__(1024) unsigned char tc_raw[];
    const uint32_t raw = smem_u32(tc_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    unsigned char *gbase = tc_raw + (base - raw);
    const uint32_t sA = base, sB = base + TC_ST * TC_A_BYTES;
    const uint32_t bars = base + TC_ST * TC_STAGE_BYTES;  // full[ST], empty[ST], done
    auto full = [&](int s) { return bars + 8u * s; };
    auto empty = [&](int s) { return bars + 8u * (TC_ST + s); };
    const uint32_t done = bars + 8u * (2 * TC_ST);
    uint32_t *tslot = (uint32_t *)(gbase + TC_ST * TC_STAGE_BYTES + 8 * (2 * TC_ST + 1));

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * TC_BM, n0 = blockIdx.y * TC_BN;
    if (threadIdx.x == 0) {
        for (int s = 0; s < TC_ST; ++s) {
            mbar_init(full(s), 1);
            mbar_init(empty(s), 1);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmA) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmB) : "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(TC_BN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    const int KB = kp / TC_BK, KT = 3 * KB;

    if (warp == 0) {
        if (lane == 0) {
            // producer: stage it % ST of pass it / KB (hi.hi, hi.lo, lo.hi)
            for (int it = 0; it < KT; ++it) {
                const int s = it % TC_ST;
                if (!mbar_wait(empty(s), ((it / TC_ST) & 1) ^ 1, err)) break;
                const int pass = it / KB, kb = it - pass * KB;
                const int xa = (pass == 2 ? kp : 0) + kb * TC_BK;
                const int xb = (pass == 1 ? kp : 0) + kb * TC_BK;
                mbar_expect_tx(full(s), TC_STAGE_BYTES);
                tma_load_2d(sA + s * TC_A_BYTES, &tmA, xa, m0, full(s));
                tma_load_2d(sB + s * TC_B_BYTES, &tmB, xb, n0, full(s));
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            // MMA issuer: four K = 16 steps per stage (32 bytes along the swizzled row)
            constexpr uint32_t idesc = tc_idesc();
            for (int it = 0; it < KT; ++it) {
                const int s = it % TC_ST;
                if (!mbar_wait(full(s), (it / TC_ST) & 1, err)) break;
                tc_fence_after();
                const uint64_t da = sdesc_sw128(sA + s * TC_A_BYTES), db = sdesc_sw128(sB + s * TC_B_BYTES);
#pragma unroll
                for (int kk = 0; kk < TC_BK / 16; ++kk)
                    tc_mma(tmem, da + 2 * kk, db + 2 * kk, idesc, (it | kk) != 0 ? 1u : 0u);
                tc_commit(empty(s));
            }
            tc_commit(done);
        }
        __syncwarp();
    }

    // epilogue: warp w reads accumulator lanes (real rows) 32 w .. 32 w + 31
    const bool mine_ok = mbar_wait(done, 0, err);
    // tcgen05.ld is warp-collective: the decision to read is made once per warp, converged
    const bool ok = __all_sync(0xffffffffu, mine_ok && *(volatile int *)err == 0);
    __syncwarp();
    tc_fence_after();
    if (ok) tc_store_rows(tmem + ((uint32_t)(warp * 32) << 16), m0 + warp * 32 + lane, m, n, n0, alpha, beta, Cm, ldc);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_BN) : "memory");
    }
}

// ---------------------------------------------------------------------------
// Persistent variant: one CTA per SM walks the output tiles (tile c, c + G, c + 2G, ...),
// with two TMEM accumulators (512 columns) so that the epilogue of one tile runs under the
// main loop of the next.  Ten warps: 0 TMA producer, 1 MMA issuer, 2-9 epilogue (TMEM lane
// quarter = warp mod 4, the first or second half of the 256 accumulator columns).  4-stage
// operand ring as above; accumulator hand-off through tfull[b] (MMA -> epilogue,
// tcgen05.commit) and tempty[b] (epilogue -> MMA, 256 arrivals).
// ---------------------------------------------------------------------------
#define TCP_T 320
#define TCP_ST 4

__global__ void __launch_bounds__(TCP_T, 1)
    k_tc_gemm_p(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int m, int n, int kp,
                int tiles_x, int ntiles, float2 alpha, float2 beta, float2 *__restrict__ Cm, int ldc, int *err)
{
    extern __shared__ __align__(1024) unsigned char tc_raw[];
    const uint32_t raw = smem_u32(tc_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    unsigned char *gbase = tc_raw + (base - raw);
    const uint32_t sA = base, sB = base + TCP_ST * TC_A_BYTES;
    const uint32_t bars = base + TCP_ST * TC_STAGE_BYTES;  // full[ST], empty[ST], tfull[2], tempty[2]
    auto full = [&](int s) { return bars + 8u * s; };
    auto empty = [&](int s) { return bars + 8u * (TCP_ST + s); };
    auto tfull = [&](int b) { return bars + 8u * (2 * TCP_ST + b); };
    auto tempty = [&](int b) { return bars + 8u * (2 * TCP_ST + 2 + b); };
    uint32_t *tslot = (uint32_t *)(gbase + TCP_ST * TC_STAGE_BYTES + 8 * (2 * TCP_ST + 4));

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < TCP_ST; ++s) {
            mbar_init(full(s), 1);
            mbar_init(empty(s), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(tfull(b), 1);
            mbar_init(tempty(b), TCP_T - 64);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmA) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmB) : "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(2 * TC_BN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    const int KB = kp / TC_BK, KT = 3 * KB;

    if (warp == 0) {
        if (lane == 0) {
            uint32_t g = 0;
            bool alive = true;
            for (int t = blockIdx.x; t < ntiles && alive; t += gridDim.x) {
                const int m0 = (t % tiles_x) * TC_BM, n0 = (t / tiles_x) * TC_BN;
                for (int it = 0; it < KT; ++it, ++g) {
                    const int s = g % TCP_ST;
                    if (!mbar_wait(empty(s), ((g / TCP_ST) & 1) ^ 1, err)) {
                        alive = false;
                        break;
                    }
                    const int pass = it / KB, kb = it - pass * KB;
                    mbar_expect_tx(full(s), TC_STAGE_BYTES);
                    tma_load_2d(sA + s * TC_A_BYTES, &tmA, (pass == 2 ? kp : 0) + kb * TC_BK, m0, full(s));
                    tma_load_2d(sB + s * TC_B_BYTES, &tmB, (pass == 1 ? kp : 0) + kb * TC_BK, n0, full(s));
                }
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = tc_idesc();
            uint32_t g = 0;
            bool alive = true;
            int j = 0;
            for (int t = blockIdx.x; t < ntiles && alive; t += gridDim.x, ++j) {
                const int ab = j & 1;
                if (!mbar_wait(tempty(ab), ((j >> 1) & 1) ^ 1, err)) break;
                tc_fence_after();
                const uint32_t acc = tmem + (uint32_t)(ab * TC_BN);
                for (int it = 0; it < KT; ++it, ++g) {
                    const int s = g % TCP_ST;
                    if (!mbar_wait(full(s), (g / TCP_ST) & 1, err)) {
                        alive = false;
                        break;
                    }
                    tc_fence_after();
                    const uint64_t da = sdesc_sw128(sA + s * TC_A_BYTES), db = sdesc_sw128(sB + s * TC_B_BYTES);
#pragma unroll
                    for (int kk = 0; kk < TC_BK / 16; ++kk)
                        tc_mma(acc, da + 2 * kk, db + 2 * kk, idesc, (it | kk) != 0 ? 1u : 0u);
                    tc_commit(empty(s));
                }
                tc_commit(tfull(ab));
            }
        }
        __syncwarp();
    } else {
        const int q = warp & 3;                // TMEM lane quarter of this warp
        const int half = (warp - 2) >> 2;      // accumulator columns [128 half, 128 half + 128)
        int j = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++j) {
            const int ab = j & 1;
            const bool mine_ok = mbar_wait(tfull(ab), (j >> 1) & 1, err);
            const bool ok = __all_sync(0xffffffffu, mine_ok && *(volatile int *)err == 0);
            __syncwarp();
            if (!ok) break;
            tc_fence_after();
            const int m0 = (t % tiles_x) * TC_BM, n0 = (t / tiles_x) * TC_BN;
            tc_store_rows(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(ab * TC_BN), m0 + q * 32 + lane, m, n, n0,
                          alpha, beta, Cm, ldc, half * (TC_BN / 2), (half + 1) * (TC_BN / 2));
            tc_fence_before();
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tempty(ab)) : "memory");
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TC_BN) : "memory");
    }
}

constexpr int tcp_smem() { return TCP_ST * TC_STAGE_BYTES + 1024 + 256; }

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        HM_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
        if (q != cudaDriverEntryPointSuccess || !p) throw HmError{HM_ERR_CUDA, "cuTensorMapEncodeTiled unavailable"};
        fn = (EncodeTiledFn)p;
    }
    return fn;
}

// 2-D BF16 tensor map of a packed operand: `rows` rows of 2 kp elements, box 64 x box_rows.
static void make_map(CUtensorMap *map, const void *ptr, int rows, int kp, int box_rows)
{
    const cuuint64_t dims[2] = {(cuuint64_t)(2 * (size_t)kp), (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)(2 * (size_t)kp * sizeof(__nv_bfloat16))};
    const cuuint32_t box[2] = {TC_BK, (cuuint32_t)box_rows};
    const cuuint32_t es[2] = {1, 1};
    const CUresult r = encode_fn()(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides,
                                   box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) throw HmError{HM_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")"};
}

// Variants: 2 = 2-stage ring, two CTAs per SM; 4 = 4-stage ring, one CTA per SM; 1 =
// persistent (one CTA per SM over all tiles, double-buffered accumulators).
static void launch_tc(int st, dim3 grid, cudaStream_t stream, const CUtensorMap &ma, const CUtensorMap &mb, int m,
                      int n, int kp, cf alpha, cf beta, cf *Cm, int ldc, int *err)
{
    if (st == 2) {
        k_tc_gemm<2><<<grid, TC_T, tc_smem<2>(), stream>>>(ma, mb, m, n, kp, alpha, beta, Cm, ldc, err);
    } else if (st == 4) {
        k_tc_gemm<4><<<grid, TC_T, tc_smem<4>(), stream>>>(ma, mb, m, n, kp, alpha, beta, Cm, ldc, err);
    } else {
        static int nsm = 0;
        if (!nsm) {
            int dev = 0;
            HM_CUDA(cudaGetDevice(&dev));
            HM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        }
        const int ntiles = (int)(grid.x * grid.y);
        k_tc_gemm_p<<<std::min(ntiles, nsm), TCP_T, tcp_smem(), stream>>>(ma, mb, m, n, kp, (int)grid.x, ntiles, alpha,
                                                                          beta, Cm, ldc, err);
    }
    HM_CHECK_LAUNCH();
}

// Variant autotuner.  Per depth class (kp = 64 .. 4096 by powers of two) the first product
// with m, n >= 2048 times the three kernel variants (2 stages, two CTAs per SM; 4 stages, one
// CTA per SM; persistent with double-buffered accumulators) on its leading block of at most
// 2^28 outputs, accumulating (beta = 1, so the epilogue reads and writes as in the H-LU's
// updates) into scratch memory, twice each, and keeps the fastest for every later product of
// that class.  Until a class is tuned: 2 stages for kp <= 512, else 4.
static int g_tc_stages[8] = {0, 0, 0, 0, 0, 0, 0, 0};
static float g_tc_tune_ms[8][3];

static std::mutex g_tc_tune_mutex;  // handles on different host threads share the record

static int tc_stages(hm_handle_s *h, const CUtensorMap &ma, const CUtensorMap &mb, int m, int n, int kp, int *err)
{
    int cls = 0;
    while ((TC_BK << cls) < kp && cls < 7) ++cls;
    std::lock_guard<std::mutex> lock(g_tc_tune_mutex);
    if (g_tc_stages[cls]) return g_tc_stages[cls];
    const int dflt = kp <= 512 ? 2 : 4;
    if (m < 2048 || n < 2048) return dflt;
    const int ms = m, ns = (int)std::min<long long>(n, std::max<long long>(256, (1LL << 28) / m));
    cf *scratch = nullptr;
    try {
        scratch = (cf *)dalloc(h, sizeof(cf) * (size_t)ms * ns);
    } catch (const HmError &) {
        return dflt;  // no room for the timing block: the default variant, tuned later
    }
    const dim3 grid((2 * ms + TC_BM - 1) / TC_BM, (2 * ns + TC_BN - 1) / TC_BN);
    cudaEvent_t e0 = gemm_event(h), e1 = gemm_event(h);
    float best[3] = {1e30f, 1e30f, 1e30f};
    const int sts[3] = {2, 4, 1};
    HM_CUDA(cudaMemsetAsync(scratch, 0, sizeof(cf) * (size_t)ms * ns, h->stream));
    for (int rep = 0; rep < 2; ++rep)
        for (int v = 0; v < 3; ++v) {
            HM_CUDA(cudaEventRecord(e0, h->stream));
            launch_tc(sts[v], grid, h->stream, ma, mb, ms, ns, kp, cmk<cf>(1, 0), cmk<cf>(1, 0), scratch, ms, err);
            HM_CUDA(cudaEventRecord(e1, h->stream));
            HM_CUDA(cudaEventSynchronize(e1));
            float t = 0;
            HM_CUDA(cudaEventElapsedTime(&t, e0, e1));
            best[v] = std::min(best[v], t);
        }
    count_launch(h, 6);
    h->gemm_free.push_back(e0);
    h->gemm_free.push_back(e1);
    dfree(h, scratch);
    int bv = 0;
    for (int v = 0; v < 3; ++v) {
        g_tc_tune_ms[cls][v] = best[v];
        if (best[v] < best[bv]) bv = v;
    }
    g_tc_stages[cls] = sts[bv];
    return g_tc_stages[cls];
}

// The autotuner's record: per depth class kp = 64 << c (c = 0..7) the chosen variant
// (2, 4 or 1 = persistent; 0: not tuned) and the three measured times (ms).
void tc_tune_record(int *stages, float *ms3)
{
    std::lock_guard<std::mutex> lock(g_tc_tune_mutex);
    for (int c = 0; c < 8; ++c) {
        stages[c] = g_tc_stages[c];
        for (int v = 0; v < 3; ++v) ms3[3 * c + v] = g_tc_tune_ms[c][v];
    }
}

bool tc_eligible(const hm_handle_s *h, int m, int n, int k)
{
    if (h->prm.simt_gemm) return false;
    return m >= 64 && n >= 64 && k >= 16 && 8.0 * m * n * k >= 2.0e8;
}

int *tc_err_flag(hm_handle_s *h)
{
    if (!h->d_tc_err) {
        HM_CUDA(cudaMalloc(&h->d_tc_err, sizeof(int)));
        HM_CUDA(cudaMemsetAsync(h->d_tc_err, 0, sizeof(int), h->stream));
    }
    return h->d_tc_err;
}

void tc_gemm(hm_handle_s *h, char opA, char opB, int m, int n, int k, cf alpha, const cf *A, int lda, const cf *B,
             int ldb, cf beta, cf *Cm, int ldc, int variant)
{
    if (m <= 0 || n <= 0 || k <= 0) throw HmError{HM_ERR_ARG, "tc_gemm: empty product"};
    static bool attr = false;
    if (!attr) {
        HM_CUDA(cudaFuncSetAttribute(k_tc_gemm<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc_smem<4>()));
        HM_CUDA(cudaFuncSetAttribute(k_tc_gemm<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc_smem<2>()));
        HM_CUDA(cudaFuncSetAttribute(k_tc_gemm_p, cudaFuncAttributeMaxDynamicSharedMemorySize, tcp_smem()));
        attr = true;
    }
    int *err = tc_err_flag(h);
    const int kc_max = std::min(k, TC_KC);
    const int kp_max = (kc_max + TC_BK - 1) / TC_BK * TC_BK;
    const size_t abytes = (size_t)2 * m * 2 * kp_max * sizeof(__nv_bfloat16);
    const size_t bbytes = (size_t)2 * n * 2 * kp_max * sizeof(__nv_bfloat16);
    const size_t need = ((abytes + 1023) & ~(size_t)1023) + bbytes;
    // the packed operands of this stream (products on other streams have their own)
    hm_handle_s::TcWs *ws = nullptr;
    for (auto &w : h->tc_ws)
        if (w.s == h->stream) ws = &w;
    if (!ws) {
        h->tc_ws.push_back(hm_handle_s::TcWs{h->stream, nullptr, 0});
        ws = &h->tc_ws.back();
    }
    if (need > ws->bytes) {
        if (ws->p) dfree(h, ws->p);
        ws->p = nullptr;
        ws->bytes = 0;
        ws->p = dalloc(h, need);
        ws->bytes = need;
    }
    __nv_bfloat16 *pa = (__nv_bfloat16 *)ws->p;
    __nv_bfloat16 *pb = (__nv_bfloat16 *)((char *)ws->p + ((abytes + 1023) & ~(size_t)1023));
    const bool ca = opA == 'C', cb = opB == 'C';
    for (int k0 = 0; k0 < k; k0 += TC_KC) {
        const int kc = std::min(TC_KC, k - k0);
        const int kp = (kc + TC_BK - 1) / TC_BK * TC_BK;
        // op(A)[i][p]: 'N' A[i + p lda] (rows contiguous), 'C' conj(A[p + i lda])
        const cf *xa = ca ? A + k0 : A + (size_t)k0 * lda;
        // op(B)^T[j][p] = op(B)[p][j]: 'N' B[p + j ldb], 'C' conj(B[j + p ldb])
        const cf *xb = cb ? B + (size_t)k0 * ldb : B + k0;
        k_tc_pack<<<dim3(kp / 32, (m + 31) / 32), dim3(32, 8), 0, h->stream>>>(xa, lda, m, kc, kp, ca ? 0 : 1,
                                                                               ca ? 1 : 0, pa);
        HM_CHECK_LAUNCH();
        k_tc_pack<<<dim3(kp / 32, (n + 31) / 32), dim3(32, 8), 0, h->stream>>>(xb, ldb, n, kc, kp, cb ? 1 : 0,
                                                                               cb ? 1 : 0, pb);
        HM_CHECK_LAUNCH();
        CUtensorMap ma, mb;
        make_map(&ma, pa, 2 * m, kp, TC_BM);
        make_map(&mb, pb, 2 * n, kp, TC_BN);
        const cf bet = k0 == 0 ? beta : cmk<cf>(1, 0);
        const dim3 grid((2 * m + TC_BM - 1) / TC_BM, (2 * n + TC_BN - 1) / TC_BN);
        const double fl = 24.0 * m * n * (double)kc;  // BF16 tensor flops: 3 split products of 8 m n kc
        const bool timed = fl >= 1e9;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (timed) {
            e0 = gemm_event(h);
            e1 = gemm_event(h);
        }
        const int st = variant ? variant : tc_stages(h, ma, mb, m, n, kp, err);
        if (timed) HM_CUDA(cudaEventRecord(e0, h->stream));  // after any tuning launches
        launch_tc(st, grid, h->stream, ma, mb, m, n, kp, alpha, bet, Cm, ldc, err);
        if (timed) {
            HM_CUDA(cudaEventRecord(e1, h->stream));
            h->gemm_pending.push_back(GemmTiming{e0, e1, fl, 1});
        }
        count_launch(h, 3);
    }
    h->flops_factor += 8.0 * m * n * (double)k;
}

// Reads and clears the flag of the tensor-core products (the stream is synchronised by the
// caller); a set flag means a bounded wait inside k_tc_gemm expired.
void tc_check(hm_handle_s *h)
{
    if (!h->d_tc_err) return;
    int e = 0;
    HM_CUDA(cudaMemcpy(&e, h->d_tc_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (e) {
        HM_CUDA(cudaMemset(h->d_tc_err, 0, sizeof(int)));
        throw HmError{HM_ERR_TIMEOUT, "tensor-core GEMM: a bounded pipeline wait expired"};
    }
}
