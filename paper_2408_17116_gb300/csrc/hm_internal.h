// Host-side structures of libhm: handle, cluster tree, block tree, error
// handling, device memory, and the launch wrappers each translation unit exports.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/hm.h"
#include "hm_device.cuh"

struct HmError {
    hm_status st;
    std::string msg;
};

#define HM_CUDA(x)                                                                              \
    do {                                                                                        \
        cudaError_t e_ = (x);                                                                   \
        if (e_ != cudaSuccess)                                                                  \
            throw HmError{e_ == cudaErrorMemoryAllocation ? HM_ERR_OOM : HM_ERR_CUDA,           \
                          std::string(#x) + ": " + cudaGetErrorString(e_)};                     \
    } while (0)

#define HM_CHECK_LAUNCH()                                                                       \
    do {                                                                                        \
        cudaError_t e_ = cudaGetLastError();                                                    \
        if (e_ != cudaSuccess)                                                                  \
            throw HmError{HM_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e_)}; \
    } while (0)

// Quadrature constants of the near-field rule (the GPU method; see hm_near.cu).
struct NearRule {
    int qd, qi, qo;     // Duffy points per direction, inner sinh panel points, outer panel points
    double t0;          // inner panel length (parameter units)
};

struct Cluster {
    int off, cnt;       // nodes [off, off+cnt) in tree order
    double bmin[3], bmax[3];
    int child[2];
    int level;
    int b0 = 0, b1 = 0;      // bodies of its nodes: [b0, b1] (independent bodies: contiguous)
    bool body_root = false;  // independent bodies: the cluster of one whole body
};

enum BType { B_DENSE = 0, B_LR = 1, B_HIER = 2 };

// One node of the block cluster tree; C = complex128 (the FP64 H-matrix) or
// complex64 (the FP32 copy that is factored as a preconditioner).
template <class C>
struct BlockT {
    BType type = B_DENSE;
    int r0 = 0, nr = 0, c0 = 0, nc = 0;  // tree-ordered unknown ranges
    int t = -1, s = -1;                  // clusters
    BlockT *ch[4] = {nullptr, nullptr, nullptr, nullptr};  // (0,0) (0,1) (1,0) (1,1)
    C *D = nullptr;                      // dense, column-major, ld = nr
    int *piv = nullptr;                  // diagonal dense leaf after LU (device, nr entries)
    C *U = nullptr, *V = nullptr;        // low rank: A = U V^H, U nr x k, V nc x k
    int k = 0;
    int leaf_id = -1;
    // low-rank updates not yet recompressed: sum_i Up_i Vp_i^H (owned buffers)
    std::vector<C *> pu, pv;
    std::vector<int> pk;
    int pend_k = 0;
    bool zero = false;      // independent bodies: a block between two bodies (identically zero)
    bool dirty = false;     // queued for the next batched recompression
    bool in_batch = false;  // scratch flag while a batch is assembled
};
typedef BlockT<zc> Block;
typedef BlockT<cf> Block32;

// A dense column-major view in device memory.
template <class C>
struct MVT {
    C *p;
    int rows, cols, ld;
};
typedef MVT<zc> MV;

template <class C>
struct TileOp;

// A product timed with CUDA events (hm_linalg.cu), read after the next synchronisation.
// Named phases timed with CUDA events on the handle's stream (PhaseScope), summed by
// phase_collect at the next synchronisation point.
enum PhaseId { PH_LU_PANEL = 0, PH_LU_U12, PH_TILE_BUILD, PH_SOLVE_SWEEP, PH_SOLVE_MATVEC, PH_COUNT };
struct PhaseMark {
    int id;
    cudaEvent_t e0, e1;
};

struct GemmTiming {
    cudaEvent_t e0, e1;
    double flops;
    int kind = 0;  // 0: CUDA-core k_zgemm (complex flops), 1: tensor-core k_tc_gemm (BF16 tensor flops)
};

struct hm_handle_s {
    cudaStream_t stream = nullptr;
    int device = 0;
    int state = 0;  // 0 created, 1 geometry, 2 filled, 3 factored
    std::string err;
    hm_params prm{};
    NearRule rule{24, 24, 16, 0.5};
    // geometry
    int nc = 0, nbodies = 0, npatch = 0, nnode = 0, N = 0;
    int dof = 2;  // unknowns per node, kept together and interleaved (2: J^u, J^v)
    std::vector<DevBody> bodies;
    std::vector<DevPatch> patches;
    DevBody *d_bodies = nullptr;
    DevPatch *d_patches = nullptr;
    double *d_nodes = nullptr;  // SoA [14][nnode]
    std::vector<double> h_nodes;  // SoA copy
    // near pairs (CSR by target patch) and store
    std::vector<int> pair_q, pair_p;  // per pair
    int *d_pair_q = nullptr, *d_pair_p = nullptr;
    int *d_nearidx = nullptr;  // [P][P] -> pair index or -1
    int *d_patch_body = nullptr;  // independent bodies: body of each patch (device), else null
    std::vector<int> node_body;   // body of each node (natural order, host)
    zc *d_near = nullptr;      // [npairs][dof nc^2][dof nc^2]
    double *d_d1 = nullptr;    // [nc][nc] derivatives of the cardinal functions at the nodes (N-Mueller)
    unsigned long long *d_counter = nullptr;  // device counters (quadrature points)
    // tree
    std::vector<Cluster> clusters;
    std::vector<int> perm_node;  // tree position -> natural node
    int *d_perm = nullptr;       // tree unknown -> natural unknown
    int *d_iperm = nullptr;      // natural unknown -> tree unknown
    Block *root = nullptr;
    std::vector<Block *> blocks;  // all blocks (owned)
    std::vector<Block *> leaves;
    Block *copy_root = nullptr;   // unfactored copy (keep_matrix)
    std::vector<Block *> copy_blocks;
    // low-rank leaves whose pending updates reached the recompression threshold; they are
    // recompressed together with the next batch that has to run
    std::vector<Block *> dirty64;
    std::vector<Block32 *> dirty32;
    Block32 *root32 = nullptr;    // FP32 factor (precision HM_FP32_REFINED)
    std::vector<Block32 *> blocks32;
    // rank model (learned ACA-rank predictor) and the samples of the last fill
    hm_mlp rank_model = nullptr;
    std::vector<float> rank_feat, rank_target;  // [n][HM_RANK_NFEAT], log(1 + rank)
    double aca_prealloc = 0;      // complex words allocated for ACA factors by the last fill
    int aca_reruns = 0;           // blocks re-run because the predicted rank was too low
    int aca_skipped = 0;          // attempts skipped because the model predicted failure
    double rank_pred_err = 0;     // mean |predicted - achieved| log(1 + rank) of the last fill
    double factor_tol = 1e-5;     // truncation tolerance of the FP32 factor
    int refine_iters = 0;         // refinement steps taken by the last solve
    double refine_res = 0;        // final relative residual of the last solve (max over RHS)
    // statistics
    double t_geom = 0, t_near = 0, t_dense = 0, t_aca = 0, t_trunc = 0, t_factor = 0, t_solve = 0;
    double flops_factor = 0;
    // recompression statistics (reset by hm_fill and hm_factor)
    double tr_batches = 0, tr_jobs = 0, tr_maxk = 0, tr_work = 0, tr_seconds = 0;
    // device time (CUDA events around each launch) and algorithmic real flops of the
    // recompression kernels: Householder QR of the factors, and the core factorisation
    // (pivoted QR for complex64, Jacobi SVD for complex128); reset with the statistics
    double kqr_s = 0, kqr_flops = 0, kqr_n = 0, kcore_s = 0, kcore_flops = 0, kcore_n = 0;
    // one record per recompression batch (reset with the statistics): jobs, largest m or n,
    // largest K, sum of (m + n) K^2, device seconds of the QR and of the core kernel, host
    // wall seconds of the whole batch
    std::vector<double> trunc_log;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    long long launches = 0;
    int aca_nonconv = 0;
    unsigned long long near_points = 0;
    double tol = 1e-7;
    double trunc_tol = 1e-7;     // truncation tolerance of the FP64 recompressions and H-LU
    double cur_tol = 1e-7;       // truncation tolerance of the factorisation in progress
    int fault = 0;               // host-side fault injection armed by hm_inject_fault (HM_FAULT_*)
    int *d_info_cur = nullptr;   // zero-pivot flag of the H-LU in progress (device), else null
    int dense_lev = -1;          // cluster level from which the last factor stored dense blocks
    // products of at least 1e9 real flops, timed with CUDA events (reset with the statistics)
    std::vector<GemmTiming> gemm_pending;
    std::vector<cudaEvent_t> gemm_free;
    double kgemm_s = 0, kgemm_flops = 0, kgemm_n = 0;
    double ktc_s = 0, ktc_flops = 0, ktc_n = 0;
    std::vector<PhaseMark> phase_pending;
    double phase_s[PH_COUNT] = {0, 0, 0, 0, 0};
    // tensor-core products (hm_tc.cu): packed-operand workspace (grow-only) and the
    // device flag of an expired pipeline wait
    struct TcWs {
        cudaStream_t s;
        void *p;
        size_t bytes;
    };
    std::vector<TcWs> tc_ws;  // one grow-only workspace per stream that runs products
    int *d_tc_err = nullptr;
    // streams for independent work (the LUs of independent bodies, the inverses of the
    // diagonal tiles): forked from and joined back into `stream` with events
    std::vector<cudaStream_t> pool;
    std::vector<cudaEvent_t> pool_ev;
    // block-row plans (hm_tiles.cu): product with the FP64 H-matrix, sweeps of the factors
    TileOp<zc> *tmat64 = nullptr, *tmatcopy = nullptr, *tfac64 = nullptr;
    TileOp<cf> *tfac32 = nullptr;
};

// ---- hm_mlp.cu ----
#define HM_RANK_NFEAT 8
void mlp_predict_host(hm_mlp m, int n, const float *feat_host, float *pred_host);
int mlp_nin(hm_mlp m);
void rank_features(hm_handle_s *h, const Block *b, float *f);  // hm_api.cu

// ---- device memory (stream-ordered pool) ----
void *dalloc(hm_handle_s *h, size_t bytes);
void dfree(hm_handle_s *h, void *p);

// ---- hm_geometry.cu ----
void launch_nodes(hm_handle_s *h, const double *d_x1d, const double *d_w1d);
void launch_patch_grid(hm_handle_s *h, const double *d_g, int ng, double *d_out);
void launch_near(hm_handle_s *h, const double *d_tabs, const double *d_C);
// ---- hm_muller_dev.cu (N-Mueller: near quadrature, right-hand sides, far field) ----
void launch_near_muller(hm_handle_s *h, const double *d_tabs, const double *d_C);
void launch_rhs_muller(hm_handle_s *h, int nrhs, const double *d_dirs, zc *d_b);  // tree order
void launch_farfield_muller(hm_handle_s *h, int nrhs, const zc *d_x, int nang, const double *d_dirs, zc *d_efar,
                            double *d_rcs);

// ---- hm_fill.cu ----
struct DenseDesc {
    int r0, nr, c0, ncol;
    zc *D;
};
struct LRDesc {
    int r0, nr, c0, ncol;
    zc *U, *V;
    int kmax;
};
void launch_dense_fill(hm_handle_s *h, const std::vector<DenseDesc> &descs);
void launch_aca(hm_handle_s *h, const std::vector<LRDesc> &descs, int *d_rank, int *d_flag);
void launch_entries(hm_handle_s *h, int n, const int *d_rows, const int *d_cols, zc *d_out);

// ---- hm_linalg.cu (complex dense kernels, instantiated for complex128 and complex64) ----
cudaEvent_t gemm_event(hm_handle_s *h);
void gemm_timing_collect(hm_handle_s *h);
// C = alpha op(A) op(B) + beta C, op: 'N' or 'C' (conjugate transpose)
template <class C>
void zgemm(hm_handle_s *h, char opA, char opB, int m, int n, int k, C alpha, const C *A, int lda, const C *B, int ldb,
           C beta, C *Cm, int ldc);
template <class C>
void zgetrf(hm_handle_s *h, int n, C *A, int lda, int *piv, int *d_info);
template <class C>
void zlaswp(hm_handle_s *h, MVT<C> X, const int *piv, int n);  // apply piv[0..n) forward to rows
template <class C>
void ztrsm_lln(hm_handle_s *h, const C *L, int ldl, int n, MVT<C> X);  // X = L^-1 X, unit lower
template <class C>
void ztrsm_lun(hm_handle_s *h, const C *U, int ldu, int n, MVT<C> X);  // X = U^-1 X, upper
template <class C>
void ztrsm_luh(hm_handle_s *h, const C *U, int ldu, int n, MVT<C> X);  // X = U^-H X
template <class C>
void ztrsm_run(hm_handle_s *h, const C *U, int ldu, int n, MVT<C> X);  // X = X U^-1 (X rows x n)
// Li = L^-1, Ui = U^-1 (n x n, ld n) of the LU factors stored in T (unit lower L, upper U)
template <class C>
void ztri_inverses(hm_handle_s *h, const C *T, int ldt, int n, C *Li, C *Ui);
template <class C>
void zcopy2d(hm_handle_s *h, MVT<C> dst, MVT<C> src);
template <class C>
void zscale_cols(hm_handle_s *h, MVT<C> X, const typename CReal<C>::R *d_s);  // X[:,j] *= s[j]
// Householder QR of many matrices in one cooperative launch (hm_qr.cu): A (m x K, ld m)
// is overwritten; Q (m x r, ld m) and R (r x K, ld r) with r = min(m, K) are written.
template <class C>
struct QRJob {
    C *A;
    int m, K;
    C *Q, *R;
};
template <class C>
void batched_qr(hm_handle_s *h, const std::vector<QRJob<C>> &jobs);
template <class C>
void batched_truncate(hm_handle_s *h, std::vector<BlockT<C> *> &blks, const std::vector<int> &ranks, double tol);

void phase_collect(hm_handle_s *h);
// The first n streams of the pool start after the work issued so far on h->stream (fork), and
// h->stream waits for everything they were given (join).
void pool_fork(hm_handle_s *h, int n);
void pool_join(hm_handle_s *h, int n);
#define HM_POOL_STREAMS 8
struct PhaseScope {
    hm_handle_s *h;
    int id;
    cudaEvent_t e0;
    bool open = true;
    PhaseScope(hm_handle_s *h_, int id_) : h(h_), id(id_)
    {
        e0 = gemm_event(h);
        HM_CUDA(cudaEventRecord(e0, h->stream));
    }
    void end()
    {
        if (!open) return;
        open = false;
        cudaEvent_t e1 = gemm_event(h);
        if (cudaEventRecord(e1, h->stream) == cudaSuccess) {
            h->phase_pending.push_back(PhaseMark{id, e0, e1});
        } else {
            h->gemm_free.push_back(e0);
            h->gemm_free.push_back(e1);
        }
    }
    ~PhaseScope() { end(); }
};

// ---- hm_tc.cu (complex64 GEMM on the tensor cores, split-BF16) ----
bool tc_eligible(const hm_handle_s *h, int m, int n, int k);
// variant: 0 = autotuned, 2 / 4 = 2- / 4-stage ring, 1 = persistent
void tc_gemm(hm_handle_s *h, char opA, char opB, int m, int n, int k, cf alpha, const cf *A, int lda, const cf *B,
             int ldb, cf beta, cf *Cm, int ldc, int variant = 0);
void tc_check(hm_handle_s *h);  // after a synchronisation: HM_ERR_TIMEOUT if a pipeline wait expired
void tc_tune_record(int *stages, float *ms3);  // the variant autotuner's choices and timings

// ---- hm_io.cu ----
void launch_rhs(hm_handle_s *h, int nrhs, const double *d_dirs, zc *d_b);  // tree order
void launch_permute(hm_handle_s *h, int nrhs, const zc *src, zc *dst, const int *map);
void launch_farfield(hm_handle_s *h, int nrhs, const zc *d_x, int nang, const double *d_dirs, zc *d_efar,
                     double *d_rcs);

// ---- hm_hlu.cu (instantiated for complex128 and complex64) ----
template <class C>
void hlu_factor(hm_handle_s *h, BlockT<C> *root, double tol);
template <class C>
void hmatvec(hm_handle_s *h, BlockT<C> *A, MVT<C> X, MVT<C> Y, C alpha, bool conjtrans);  // Y += alpha op(A) X
// Deep copy of a block tree, converting the storage precision (complex128 -> C).
template <class C>
BlockT<C> *clone_tree(hm_handle_s *h, Block *b, std::vector<BlockT<C> *> &owned);
template <class C>
void free_tree(hm_handle_s *h, std::vector<BlockT<C> *> &owned);
// Complex64 copy of the FP64 tree with every hierarchical block on cluster level `level` or
// deeper already merged into one dense block (one batched expansion launch).
Block32 *clone_tree_merged(hm_handle_s *h, Block *root, int level, std::vector<Block32 *> &owned);
// Merge every hierarchical block on cluster level `level` or deeper into one dense block.
template <class C>
void coarsen_tree(hm_handle_s *h, BlockT<C> *root, int level);
// level value of coarsen_tree / clone_tree_merged: merge the diagonal block of every body
// (independent bodies)
#define HM_MERGE_BODIES (-2)
template <class C>
bool merges_at(const hm_handle_s *h, const BlockT<C> *b, int level);
// Coarsest level of clusters of at most cap unknowns whose non-low-rank blocks store at
// least theta of their dense size (-1: none).
template <class C>
int dense_level_by_storage(hm_handle_s *h, BlockT<C> *root, int cap, double theta);
// Coarsest level whose merge keeps the tree's storage within budget_words (-1: none).
template <class C>
int dense_level_by_memory(hm_handle_s *h, BlockT<C> *root, double budget_words);
// y[i] = (To) x[i] for n complex values
template <class Ti, class To>
void convert_vec(hm_handle_s *h, const Ti *x, To *y, size_t n);

// ---- hm_tiles.cu (block-row product and substitution sweeps, complex128 and complex64) ----
template <class C>
struct TileOp;
// Plan over the leaves of a block tree; factored: also the sweeps of its H-LU factors
// (explicit inverses of the diagonal factors are formed here).  The plan points at the
// leaves' data: it is valid while the tree's storage is unchanged.
template <class C>
TileOp<C> *tile_build(hm_handle_s *h, BlockT<C> *root, bool factored);
template <class C>
void tile_free(hm_handle_s *h, TileOp<C> *T);
template <class C>
void tile_matvec(hm_handle_s *h, TileOp<C> *T, const C *X, C *Y, int nrhs, C alpha);  // Y += alpha A X
template <class C>
void tile_solve(hm_handle_s *h, TileOp<C> *T, C *X, int nrhs);  // X <- A^-1 X (factored plan)

// ---- hm_planner.cpp ----
void plan_geometry(hm_handle_s *h);  // nodes, near pairs, cluster tree, block tree
void rebuild_block_tree(hm_handle_s *h);  // block tree from the cluster tree (discards blocks)
void build_cluster_tree(hm_handle_s *h);  // cluster tree from h->h_nodes (host only)
void cheb_nodes_host(int n, double *x);
void fejer_weights_host(int n, double *w);
void gauss_legendre_host(int q, double *x, double *w);

static inline void count_launch(hm_handle_s *h, int n = 1) { h->launches += n; }
