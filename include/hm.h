/*
 * hm.h -- C ABI of the GB300 (sm_103a) H-matrix accelerated CBIE direct solver.
 *
 * Method: arXiv 2408.17116, "H-Matrix Accelerated Direct Matrix Solver for
 * Maxwell's Equations using the Chebyshev-based Nystrom Boundary Integral
 * Equation Method".  The solver discretises the MFIE of a PEC body (Sec. II.A,
 * Eq. 10, second row) with the CBIE (Sec. II.B, Eqs. 11-20), compresses the
 * system as an H-matrix (Sec. III, Eq. 21, ACA), factors it by H-LU and solves
 * by H-forward/back substitution (Sec. III.A, Eqs. 23-28) on the entire-matrix
 * ordering (Sec. III.B).
 *
 * Conventions shared by every call
 *   - Complex numbers are two IEEE doubles (re, im); "complex128" below.
 *   - Unknowns: N = 2 * nnode.  Node n = patch * Nc^2 + kv * Nc + lu (lu: index of
 *     the u Chebyshev node, kv: index of the v node); unknown 2n + a, a = 0 for
 *     F^u, a = 1 for F^v (contravariant components scaled by sqrt|G|, Eq. 11).
 *     Patch p of body b: p = offset(b) + (face * m + i) * m + j.
 *   - Time convention exp(j w t); Green's function exp(-jkR) / (4 pi R) (Eq. 4).
 *   - All device work is issued on the stream given to hm_create (NULL = the
 *     legacy default stream).  Calls return after enqueuing unless stated
 *     otherwise; hm_query, hm_farfield's host output and every "_host" getter
 *     synchronise the stream.
 *   - Every call returns an hm_status; on failure hm_last_error() holds a
 *     message.  No C++ exception crosses this boundary.  One handle must not
 *     be used from two host threads at once.
 *   - Pointers named *_dev are device pointers owned by the caller; every other
 *     pointer is host memory owned by the caller and is only read during the
 *     call (inputs are copied).  The library owns all of its internal device
 *     memory and frees it in hm_destroy.
 */
#ifndef HM_H
#define HM_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hm_handle_s *hm_handle;
typedef struct hm_mlp_s *hm_mlp;

typedef enum {
    HM_OK = 0,
    HM_ERR_ARG = 1,           /* invalid argument (null pointer, bad size, bad enum) */
    HM_ERR_STATE = 2,         /* call out of order (geometry -> fill -> factor -> solve) */
    HM_ERR_CUDA = 3,          /* a CUDA runtime call failed */
    HM_ERR_OOM = 4,           /* device allocation failed */
    HM_ERR_SINGULAR = 5,      /* a zero pivot in a diagonal leaf of the H-LU */
    HM_ERR_NOT_CONVERGED = 6, /* an iteration hit its limit (reported, not fatal for ACA) */
    HM_ERR_TIMEOUT = 7,       /* a bounded device wait expired */
    HM_ERR_NUMERIC = 8        /* NaN/Inf in the solution (hm_solve scans its output) */
} hm_status;

/* Integral equation.  HM_PEC_MFIE: the magnetic-field equation of a PEC body (Sec. II.A,
 * Eq. 10, second row), the formulation the paper solves for every PEC case.
 * HM_PEC_CFIE: the combined field equation alpha EFIE / eta0 + (1 - alpha) MFIE of a PEC
 * body (Eq. 10, both rows; the paper does not combine them).  HM_DIEL_MULLER: the
 * N-Mueller equations of a penetrable body (Eqs. 7-9).  hm_build_geometry returns
 * HM_ERR_ARG for a formulation this library was built without (hm_version lists them). */
typedef enum { HM_PEC_MFIE = 0, HM_PEC_CFIE = 1, HM_DIEL_MULLER = 2 } hm_formulation;
/* HM_FP64: the plain FP64 method (complex128 H-matrix, FP64 H-LU and H-solve).
 * HM_FP32_REFINED: the same FP64 fill; hm_factor builds a complex64 copy of the
 * H-matrix and factors it by H-LU in FP32 (truncation tolerance factor_tol); hm_solve
 * uses that factor as a preconditioner inside FP64 iterative refinement, with the
 * residual b - A x taken with the FP64 H-matrix, until the relative residual is at
 * most refine_tol.  The paper has no FP32 mode; this is the GB300-side choice that
 * keeps FP64 only in the fill and the residual. */
typedef enum { HM_FP64 = 0, HM_FP32_REFINED = 1 } hm_precision;

/* Solver parameters.  Paper: eta and n_leaf (Sec. III, Eq. 21 and the text that
 * follows it), ACA tolerance (Sec. IV), wavenumber from the wavelength. */
typedef struct {
    double k0;            /* wavenumber (rad/m) of the exterior medium */
    int formulation;      /* hm_formulation */
    int leaf;             /* n_leaf: clusters with at most this many unknowns are leaves */
    double eta;           /* admissibility parameter of Eq. 21 */
    double aca_tol;       /* ACA stopping tolerance, also the truncation tolerance */
    double near_delta;    /* near pair: dist(bbox_q, bbox_p) < near_delta * max(diam_q, diam_p) */
    int aca_max_rank;     /* ACA rank bound before a block is split (0 = 160) */
    int precision;        /* hm_precision */
    int keep_matrix;      /* nonzero: keep an unfactored copy for hm_matvec after hm_factor */
    double factor_tol;    /* HM_FP32_REFINED: truncation tolerance of the FP32 H-LU (0 = 1e-4) */
    double refine_tol;    /* HM_FP32_REFINED: target relative residual per RHS (0 = 1e-10) */
    int refine_max_iter;  /* HM_FP32_REFINED: refinement step limit (0 = 30) */
    double cfie_alpha;    /* HM_PEC_CFIE: weight alpha of the EFIE row, 0 < alpha <= 1 */
    double eps_r_re;      /* HM_DIEL_MULLER: relative permittivity of the interior, real part (> 0) */
    double eps_r_im;      /* HM_DIEL_MULLER: imaginary part (<= 0 for a lossy medium, exp(j w t)) */
    double mu_r;          /* HM_DIEL_MULLER: relative permeability of the interior (0 = 1; only 1 is supported) */
    double trunc_tol;     /* truncation tolerance of the QR+SVD recompressions of the FP64 H-matrix and its
                             H-LU (0 = aca_tol) */
    int quad_order;       /* Gauss points per direction of the self/near rule's inner panels and Duffy squares
                             (0 = 24; 4..36; the outer panels take ceil(2 quad_order / 3)) */
    int factor_leaf;      /* the H-LU stores, as one dense block each (an exact merge), the hierarchical
                             blocks of one cluster level and of every level below it: > 0, the first
                             level whose clusters hold at most factor_leaf unknowns; 0 (adaptive):
                             the coarsest level whose merged storage fits in 40 % of the free device
                             memory (the whole matrix, when it fits), for products on the CUDA cores
                             (complex128, or simt_gemm) no coarser than clusters of 24,576 unknowns;
                             when no level fits, the coarsest level of clusters of at most 4096
                             (complex64) / 1280 (complex128) unknowns whose non-low-rank blocks store at
                             least 35 % of their dense size, else the level of 640-unknown clusters; negative, the
                             fill's block structure.  HM_FP64: applies to the H-matrix factored in
                             place; HM_FP32_REFINED: to the complex64 copy (the FP64 H-matrix is kept). */
    int simt_gemm;        /* HM_FP32_REFINED: nonzero keeps every complex64 product of the H-LU on the
                             CUDA cores; 0 runs the large ones on the tensor cores (tcgen05, operands
                             split into two BF16 parts, three products accumulated in FP32) */
    int independent;      /* nonzero: the bodies do not interact -- each scatters the incident waves alone
                             (a batch of scatterers).  The system is block diagonal, one block per body:
                             clusters never mix bodies, blocks between bodies are zero (no ACA), near pairs
                             stay within a body, and the factor stores each body's diagonal block dense
                             (factor_leaf 0).  One fill, factor and solve serve the whole batch. */
} hm_params;

/* One cube-mapped ellipsoid: 6 m^2 curvilinear patches r = center + rot diag(semi) c/|c|,
 * c = e_f + tan(pi s/4) e1 + tan(pi t/4) e2 on each cube face (equiangular map). */
typedef struct {
    int family;           /* 0 = cube-mapped ellipsoid (the only family) */
    int m;                /* patches per cube-face edge */
    double center[3];
    double semi_axes[3];
    double rot[9];        /* row-major rotation */
} hm_body;

/* hm_query keys */
enum {
    HM_Q_N = 0,            /* number of unknowns */
    HM_Q_NNODE = 1,
    HM_Q_NPATCH = 2,
    HM_Q_NEAR_PAIRS = 3,   /* near patch pairs (incl. self) */
    HM_Q_DENSE_BLOCKS = 4,
    HM_Q_LR_BLOCKS = 5,
    HM_Q_CR = 6,           /* compression rate 1 - storage(H)/N^2 (Sec. IV.A) */
    HM_Q_MAX_RANK = 7,
    HM_Q_T_GEOMETRY = 8,   /* seconds, measured with CUDA events (last call) */
    HM_Q_T_NEAR = 9,
    HM_Q_T_DENSE = 10,
    HM_Q_T_ACA = 11,
    HM_Q_T_FACTOR = 12,
    HM_Q_T_SOLVE = 13,
    HM_Q_FLOPS_FACTOR = 14,/* real flops performed by the H-LU (host-side ledger) */
    HM_Q_STORAGE = 15,     /* complex words stored by the H-matrix */
    HM_Q_ACA_NONCONV = 16, /* admissible blocks whose ACA hit the rank bound (stored dense) */
    HM_Q_LAUNCHES = 17,    /* kernels launched by the library since hm_create */
    HM_Q_NEAR_QPOINTS = 18,/* kernel evaluations performed by the near-field quadrature */
    HM_Q_MEAN_RANK = 19,
    HM_Q_STORAGE_FACTOR = 20,/* complex words of the factored H-matrix */
    HM_Q_T_RECOMPRESS = 21,/* seconds in the QR+SVD recompression after ACA */
    HM_Q_REFINE_ITERS = 22,/* refinement steps of the last hm_solve (HM_FP32_REFINED; 0 otherwise) */
    HM_Q_REFINE_RES = 23,  /* largest relative residual |b - A x| / |b| (FP64 H-matrix) after the last
                              hm_solve in HM_FP32_REFINED mode */
    HM_Q_STORAGE32 = 24,   /* complex64 words of the FP32 factor (HM_FP32_REFINED) */
    HM_Q_ACA_PREALLOC = 25,/* complex words allocated for ACA factors by the last hm_fill (all attempts) */
    HM_Q_ACA_RERUNS = 26,  /* blocks whose ACA was re-run because the rank model predicted too low */
    HM_Q_RANK_PRED_ERR = 27,/* mean |predicted - achieved| of log(1 + ACA rank) in the last hm_fill */
    /* QR + SVD recompressions since the last hm_fill or hm_factor began: */
    HM_Q_TRUNC_BATCHES = 28,/* batched launches */
    HM_Q_TRUNC_JOBS = 29,  /* low-rank sums recompressed */
    HM_Q_TRUNC_MAXK = 30,  /* largest number of columns K of one sum */
    HM_Q_TRUNC_WORK = 31,  /* sum of (m + n) K^2 over the sums */
    HM_Q_T_TRUNC = 32,     /* wall seconds spent in them (they synchronise) */
    HM_Q_ACA_SKIPPED = 33, /* ACA attempts the rank model skipped (predicted rank >= 1.25 x bound) */
    /* recompression kernels since the last hm_fill or hm_factor began, device time from
     * CUDA events around each launch and algorithmic real flops: */
    HM_Q_KQR_SECONDS = 34, /* Householder QR of the factors (one launch per batch) */
    HM_Q_KQR_FLOPS = 35,
    HM_Q_KQR_LAUNCHES = 36,
    HM_Q_KCORE_SECONDS = 37,  /* core factorisation: pivoted QR (complex64) or Jacobi SVD (complex128) */
    HM_Q_KCORE_FLOPS = 38,    /* counted for the pivoted QR only (the Jacobi sweep count varies) */
    HM_Q_KCORE_LAUNCHES = 39,
    HM_Q_DENSE_LEVEL = 40, /* cluster level from which the last hm_factor stored dense blocks (-1: none;
                              -2: each body's diagonal block, independent bodies) */
    /* products of at least 1e9 real flops in the last hm_factor (the dense Schur updates), device
     * time from CUDA events around each launch, their algorithmic real flops and count: */
    HM_Q_KGEMM_SECONDS = 41,
    HM_Q_KGEMM_FLOPS = 42,
    HM_Q_KGEMM_LAUNCHES = 43,
    /* the same for the tensor-core products (k_tc_gemm) of the last hm_factor, flops counted
     * as BF16 tensor flops: three split products of 8 m n k each */
    HM_Q_KTC_SECONDS = 44,
    HM_Q_KTC_FLOPS = 45,
    HM_Q_KTC_LAUNCHES = 46,
    /* device seconds (CUDA events) of phases of the last hm_factor: the column panels of the
     * blocked dense LU (panel LU, interchanges, updates inside the panel), the row blocks
     * U12 = L11^-1 A12 with their interchanges, and the block-row plans with the explicit
     * inverses of the diagonal tiles; of the last hm_solve: the substitution sweeps and the
     * FP64 H-matrix products of the refinement */
    HM_Q_T_LU_PANEL = 47,
    HM_Q_T_LU_U12 = 48,
    HM_Q_T_TILE_BUILD = 49,
    HM_Q_T_SOLVE_SWEEP = 50,
    HM_Q_T_SOLVE_MATVEC = 51
};

const char *hm_version(void);

/* Create a handle bound to a CUDA stream (cudaStream_t passed as void*; may be NULL)
 * on the current device.  The library allocates its internal buffers with
 * cudaMallocAsync from the device's default memory pool and sets that pool's release
 * threshold to keep freed memory cached (a process-wide setting of that pool). */
hm_status hm_create(hm_handle *h, void *cuda_stream);

/* Build the discretisation: node geometry at first-kind Chebyshev nodes (Sec. II.B,
 * Eqs. 11, 14, 17-18; Fejer weights), cluster tree and block cluster tree with the
 * admissibility of Eq. 21 (Sec. III), near patch pairs (Eq. 20).
 * bodies[nbodies] are copied; nodes_per_dir = Nc (2..16). */
hm_status hm_build_geometry(hm_handle h, const hm_body *bodies, int nbodies, int nodes_per_dir,
                            const hm_params *p);

/* Fill the H-matrix: self/near CBIE quadrature (Eq. 20, singularity-cancelling
 * change of variables), dense inadmissible leaves, ACA of admissible leaves and
 * QR+SVD recompression (Sec. III).  An admissible block whose ACA reaches the rank
 * bound min(aca_max_rank, |t||s|/(|t|+|s|)) is split into its four children and
 * retried; on the leaf level it is stored dense. */
hm_status hm_fill(hm_handle h);

/* H-LU factorisation (Sec. III, Eq. 23), partial pivoting inside the diagonal
 * dense leaves.  HM_FP64: in place.  HM_FP32_REFINED: on a complex64 copy; the FP64
 * H-matrix is kept for the refinement residual (and hm_matvec). */
hm_status hm_factor(hm_handle h);

/* Solve for nrhs plane waves E = pol exp(-jk khat.r): right-hand sides of Eq. 22
 * (b1 = -a_v.H_inc, b2 = a_u.H_inc), H-forward substitution (Eqs. 24, 26, 27) and
 * back substitution (Eqs. 25, 28).  inc_dirs, pols: host [nrhs][3] unit vectors.
 * x_dev: device complex128 [nrhs][N], natural unknown order.  In HM_FP32_REFINED mode
 * the substitutions run with the FP32 factor inside FP64 iterative refinement;
 * HM_ERR_NOT_CONVERGED (x_dev still holds the last iterate) when refine_tol is not
 * reached within refine_max_iter steps.  Synchronises in HM_FP32_REFINED mode (the
 * residual norms decide the next step on the host). */
hm_status hm_solve(hm_handle h, int nrhs, const double *inc_dirs, const double *pols, void *x_dev);

/* As hm_solve with host buffers: x_host receives complex128 [nrhs][N].  Copies in and
 * out are part of the call; returns after the result is in x_host. */
hm_status hm_solve_host(hm_handle h, int nrhs, const double *inc_dirs, const double *pols, void *x_host);

/* Far field of solutions x_dev [nrhs][N] at unit directions obs_dirs (host [nang][3]):
 * efar_dev (device complex128 [nrhs][nang][3], may be NULL) = -jk eta0/(4 pi) (I - r r)
 * sum_j w_j (F^u a_u + F^v a_v)_j exp(jk r.r_j); rcs_host (host [nrhs][nang], may be
 * NULL) = 4 pi |E_far|^2 in m^2.  Always synchronises before returning (obs_dirs is read
 * during the call). */
hm_status hm_farfield(hm_handle h, int nrhs, const void *x_dev, int nang, const double *obs_dirs,
                      void *efar_dev, double *rcs_host);

/* hm_farfield without device allocation.  The paper has no counterpart: this entry
 * point exists for callers that cannot let the library allocate device memory during
 * a call (their device memory belongs to their own pool or allocator, or their loop
 * forbids allocation after start-up).  Same arguments and results as hm_farfield, and
 * like it always synchronises before returning, but the observation directions and the RCS values are staged in one
 * static device array of HM_FARFIELD_STATIC_DOUBLES doubles (512 KiB, held by every
 * GPU that loads the library until the process exits) instead of buffers allocated
 * per call.  Limit: 3 nang + nrhs nang (nrhs nang only when rcs_host is given) must
 * not exceed HM_FARFIELD_STATIC_DOUBLES, otherwise HM_ERR_ARG and nothing runs.
 * The first call on a device looks up the array's device address (once per device,
 * with that device current); make that first call before any stream capture.  All
 * calls share the array, which keeps the last call's contents: calls that overlap on
 * the GPU (other streams or other host threads) race on it.  The current device must be
 * the one the handle was created on (HM_ERR_STATE otherwise, before anything is copied). */
#define HM_FARFIELD_STATIC_DOUBLES 65536
hm_status hm_farfield_static(hm_handle h, int nrhs, const void *x_dev, int nang, const double *obs_dirs,
                             void *efar_dev, double *rcs_host);

/* y_dev = A x_dev for nrhs vectors [nrhs][N] (natural order) with the FP64 H-matrix
 * (available after hm_fill; after hm_factor only with keep_matrix). */
hm_status hm_matvec(hm_handle h, int nrhs, const void *x_dev, void *y_dev);

hm_status hm_query(hm_handle h, int what, double *out);
const char *hm_last_error(hm_handle h);

/* Recompression batches since the last hm_fill or hm_factor began: *nbatches receives the
 * count; out (may be NULL) receives [nbatches][7] = jobs, largest m or n, largest K, sum of
 * (m + n) K^2, device seconds of the QR launch, device seconds of the core launch, host wall
 * seconds of the batch.  Diagnostics for the recompression kernels; synchronises. */
hm_status hm_get_trunc_log_host(hm_handle h, int *nbatches, double *out);

/* The complex64 GEMM of the FP32 H-LU on caller-owned device memory (Sec. III, Eq. 23: the
 * Schur-complement products of the factorisation): C = alpha op(A) op(B) + beta C with
 * op 'N' (as stored) or 'C' (conjugate transpose); A, B, C column-major complex64
 * (interleaved real/imaginary float pairs) with leading dimensions lda, ldb, ldc; op(A) is
 * m x k, op(B) k x n.  alpha and beta point at two floats (real, imaginary) on the host.
 * path 0: the dispatch hm_factor uses (tensor cores for products of at least 2e8 real
 * flops with m, n >= 64 and k >= 16, unless simt_gemm was set); 1: CUDA cores; 2: tensor
 * cores, autotuned kernel variant; 3, 4, 5: tensor cores with the 2-stage, 4-stage or
 * persistent variant (HM_ERR_ARG for 2..5 when m or n < 64 or k < 16).  Runs on the handle's stream and
 * synchronises it; HM_ERR_TIMEOUT when a bounded pipeline wait of the tensor-core kernel
 * expired (C is then unspecified).  Any handle state. */
hm_status hm_cgemm(hm_handle h, char opA, char opB, int m, int n, int k, const float *alpha, const void *A, int lda,
                   const void *B, int ldb, const float *beta, void *C, int ldc, int path);

/* The kernel-variant autotuner of the tensor-core products (process-wide): for each depth
 * class c = 0..7 (packed depth 64 << c), stages[c] = the variant chosen (2: 2-stage ring, two
 * CTAs per SM; 4: 4-stage ring, one CTA per SM; 1: persistent, double-buffered accumulators;
 * 0: not tuned yet) and ms[3c .. 3c + 2] the best of three timed launches of the 2-stage,
 * 4-stage and persistent variants on the class's first large product (a leading block of at
 * most 4096 x 4096 complex outputs, into scratch memory).  No GPU work. */
hm_status hm_tc_tuning(int *stages, float *ms);

/* Host-side fault injection for tests of the error paths (the paper has no counterpart).
 * Arms one fault for the next call that reaches it; no GPU fault, trap or hang is caused.
 *   HM_FAULT_ZERO_PIVOT: hm_factor zeroes the first column of the first diagonal leaf before
 *                        the H-LU, which must report HM_ERR_SINGULAR;
 *   HM_FAULT_NAN_RHS:    hm_solve sets one right-hand-side entry to NaN; the scan of the
 *                        solution reports HM_ERR_NUMERIC;
 *   HM_FAULT_ALLOC:      the next internal device allocation reports failure: HM_ERR_OOM.
 * HM_FAULT_NONE disarms. */
enum { HM_FAULT_NONE = 0, HM_FAULT_ZERO_PIVOT = 1, HM_FAULT_NAN_RHS = 2, HM_FAULT_ALLOC = 3 };
hm_status hm_inject_fault(hm_handle h, int what);

/* ---- learned ACA-rank predictor ---------------------------------------------
 * The paper has no learned component.  A small MLP predicts, from the geometry of
 * an admissible block, the rank ACA (Sec. III, ref. [22]) will reach.  The fill
 * splits (or, on the leaf level, stores dense) without an attempt every block whose
 * prediction is at least 1.25 times its rank bound, uses the prediction to size the
 * other blocks' ACA buffers and to order the launch, and re-runs plain adaptive ACA
 * with the full bound for every block whose prediction was too low.  Every low-rank
 * block therefore still meets the ACA tolerance; only a wrongly skipped block changes
 * the partition (it is split where plain ACA would have kept it).
 *
 * Features (HM_RANK_NFEAT = 8, float): log2|t|/10, log2|s|/10, diam(t)/(8 lambda),
 * diam(s)/(8 lambda), dist(t,s)/(8 lambda), max(diam)/dist/4, Nc/10, -log10(tol)/10,
 * with bounding-box diameters and distance (Eq. 21).  Target: log(1 + rank), with
 * rank = twice the bound for an attempt that reached its bound (only a lower bound is known).
 *
 * Network: h1 = tanh(W1 x + b1), h2 = tanh(W2 h1 + b2), y = w3.h2 + b3 (FP32).
 * Packed parameters (host float[hm_mlp_num_params]): W1 [nh][nin] row-major, b1 [nh],
 * W2 [nh][nh], b2 [nh], w3 [nh], b3.  Loss (1/n) sum (y - t)^2; training is
 * full-batch Adam (beta1 0.9, beta2 0.999, eps 1e-8) on the device. */

/* Samples of the last hm_fill: every conclusive ACA attempt (converged, or stopped at
 * the block's real bound).  *n receives the count; feat_host [n][8] and target_host [n]
 * may be NULL. */
hm_status hm_rank_samples(hm_handle h, int *n, float *feat_host, float *target_host);
/* Use model m (nin = 8) in the next hm_fill calls; NULL switches it off.  The handle
 * does not own m. */
hm_status hm_set_rank_model(hm_handle h, hm_mlp m);

/* nin in 1..16, nh in 1..64; parameters start at zero (set them with hm_mlp_set_params). */
hm_status hm_mlp_create(hm_mlp *m, int nin, int nh, void *cuda_stream);
int hm_mlp_num_params(hm_mlp m);
/* Copy parameters in (resets the Adam state) or out; host float arrays. */
hm_status hm_mlp_set_params(hm_mlp m, const float *params);
hm_status hm_mlp_get_params(hm_mlp m, float *params);
/* y_dev[n] = network(x_dev[n][nin]); device float arrays. */
hm_status hm_mlp_forward(hm_mlp m, int n, const float *x_dev, float *y_dev);
/* Loss and its gradient for targets t_dev[n]; loss_host, grad_host (host, may be NULL).
 * Synchronises. */
hm_status hm_mlp_loss_grad(hm_mlp m, int n, const float *x_dev, const float *t_dev, double *loss_host,
                           float *grad_host);
/* steps full-batch Adam steps with learning rate lr; loss_host (may be NULL) receives the
 * loss after the last step (synchronises). */
hm_status hm_mlp_train(hm_mlp m, int n, const float *x_dev, const float *t_dev, int steps, float lr,
                       double *loss_host);
const char *hm_mlp_last_error(hm_mlp m);
void hm_mlp_destroy(hm_mlp m);
void hm_destroy(hm_handle h);

/* ---- host-only planning (no GPU needed) ------------------------------------ */

/* The cluster tree and block cluster tree that hm_build_geometry builds (Sec. III:
 * balanced median bisection along the widest bounding-box axis, leaf clusters of at
 * most `leaf` unknowns; admissibility of Eq. 21, min(diam) <= eta dist of the
 * bounding boxes, dist > 0), computed on the host from node positions xyz [nnode][3]
 * with dof unknowns per node kept together and interleaved (2: the MFIE's J^u, J^v;
 * 4: the N-Mueller system's J^u, J^v, M^u, M^v).  *nblocks receives the number of leaves;
 * blocks (may be NULL) receives [nblocks][5] = type (0 dense, 1 admissible), row0,
 * nrow, col0, ncol in tree-ordered unknowns; perm_node (may be NULL) [nnode] receives
 * the natural node at each tree position.  Blocks are those before ACA, which may
 * split an admissible block further. */
hm_status hm_plan_host(const double *xyz, int nnode, int dof, int leaf, double eta, int *nblocks, int *blocks,
                       int *perm_node);

/* hm_plan_host for a batch of independent bodies (hm_params.independent): node_body
 * [nnode] gives each node's body, nodes of one body contiguous and bodies in increasing
 * order.  Clusters are split by bodies first, then bisected geometrically down to `leaf`
 * unknowns; a block whose clusters share no body is a zero block, reported with type 2. */
hm_status hm_plan_bodies_host(const double *xyz, const int *node_body, int nnode, int dof, int leaf, double eta,
                              int *nblocks, int *blocks, int *perm_node);

/* N-Mueller formulation of a dielectric body (Sec. II.A, Eqs. 7-9 with
 * alpha = -eps_r, beta = -1, mu_r = 1): the far (Nystrom) entries of target node tn
 * over every node of source patch p, evaluated on the host with the library's geometry
 * and the entry generator its device fill uses.  out: host complex128 [16][Nc^2],
 * index (row * 4 + col) * Nc^2 + j; rows E-u, E-v, H-u, H-v (tested with sqrt|G| a^b),
 * columns eta0 J^u, eta0 J^v, M^u, M^v of source node j; relative permittivity
 * eps_re + j eps_im of the interior (Im <= 0 for a lossy medium with exp(j w t)).  The
 * identity terms of the jump relations (Eq. 6) are not included. */
hm_status hm_muller_far_block_host(const hm_body *bodies, int nbodies, int nodes_per_dir, double k0,
                                   double eps_re, double eps_im, int tn, int p, void *out);
/* The self/near N-Mueller integrals of target node tn over source patch p (Eq. 20: the
 * integrand against the patch's Chebyshev interpolant), by the near-field rule of the
 * device quadrature (singular point split, graded tensor panels for near targets, Duffy
 * squares and graded strips for self targets) evaluated on the host; same layout as
 * hm_muller_far_block_host.  qd, qi, qo: Gauss points of the Duffy, inner graded and
 * outer panels (0: 24, 24, 16); t0: inner panel length (0: 0.5). */
hm_status hm_muller_near_block_host(const hm_body *bodies, int nbodies, int nodes_per_dir, double k0,
                                    double eps_re, double eps_im, int tn, int p, int qd, int qi, int qo, double t0,
                                    void *out);
/* N-Mueller right-hand side and far field on the host: rhs_out (may be NULL) receives
 * complex128 [4 nnode] for the plane wave E = pol exp(-jk khat.r) (khat, pol: [3]),
 * rows (E-u, E-v, H-u, H-v) per node = (t_b.E_inc, t_b.(khat x pol) exp(-jk khat.r));
 * efar_out (may be NULL) receives complex128 [nang][3] = -jk/(4 pi) [(I - r r) N_J - r x N_M]
 * for the solution x [4 nnode] (eta0 J^u, eta0 J^v, M^u, M^v per node). */
hm_status hm_muller_rhs_farfield_host(const hm_body *bodies, int nbodies, int nodes_per_dir, double k0,
                                      const double *khat, const double *pol, void *rhs_out, const void *x,
                                      int nang, const double *obs, void *efar_out);

/* ---- inspection (tests and diagnostics; all synchronise) ------------------- */

/* Node table, host double [nnode][14]: r[3], a_u[3], a_v[3], n[3], sqrtG, w. */
hm_status hm_get_nodes_host(hm_handle h, double *out);
/* Near patch pairs: host int [npairs][2] (target patch, source patch). */
hm_status hm_get_near_pairs_host(hm_handle h, int *out);
/* Near weights of target node tn over source patch p (must be a near pair):
 * host complex128 [d^2][Nc^2], index (d b + a) * Nc^2 + j (tested rows b, source components a;
 * d = 2 unknowns per node for the MFIE, 4 for the N-Mueller system). */
hm_status hm_get_near_block_host(hm_handle h, int tn, int p, void *out);
/* Matrix entries A[rows[i], cols[i]] (natural unknown indices) from the fill's entry
 * rule (near store + Nystrom far rule + identity term): host complex128 [n]. */
hm_status hm_entries_host(hm_handle h, int n, const int *rows, const int *cols, void *out);
/* Permutation of unknowns: perm[i] = natural index of tree-ordered unknown i (host int [N]). */
hm_status hm_get_perm_host(hm_handle h, int *perm);
/* Leaf blocks: host int [nblocks][6] = type (0 dense, 1 low-rank), row0, nrow, col0, ncol,
 * rank (tree-ordered unknowns).  Pass out = NULL to get only the count in *nblocks. */
hm_status hm_get_blocks_host(hm_handle h, int *nblocks, int *out);
/* Dense content of leaf block b after hm_fill (dense block, or U V^H of a low-rank one):
 * host complex128 column-major [nrow][ncol]. */
hm_status hm_get_block_dense_host(hm_handle h, int b, void *out);

#ifdef __cplusplus
}
#endif
#endif /* HM_H */
