/*
 * hsolve.h -- C-ABI of the GB300 (sm_103a) hierarchical solver with deferred
 * compression.
 *
 * The method: Chen, Cambier, Boman, Rajamanickam, Tuminaro, Darve, "A Robust
 * Hierarchical Solver for Ill-conditioned Systems with Applications to Ice
 * Sheet Modeling".  The library solves A x = b for a sparse SPD matrix A
 * (Sec. 3, Eq. ax=b) with a hierarchical factorization (Algorithm 1) used as
 * a preconditioner (Algorithm 2) inside PCG or right-preconditioned GMRES
 * (Sec. 5).
 *
 * Conventions for every entry point:
 *   - CSR input: rowptr[n+1] (int64), col[nnz] (int32), val[nnz] (double);
 *     both triangles stored, columns of a row in any order, A symmetric
 *     positive definite.  The library copies what it needs during the call;
 *     the caller keeps ownership of every pointer it passes.
 *   - Vectors and CSR arrays live where options.mem says (HS_MEM_HOST: host
 *     memory, HS_MEM_DEVICE: device memory of the current CUDA device).
 *     hs_apply and hs_krylov always take device vectors.
 *   - All device work is ordered on options.stream (a cudaStream_t, NULL =
 *     legacy default stream); calls return after their work has completed,
 *     except hs_apply, which is stream-ordered and returns immediately.
 *   - Every function returns an hs_status; no exception crosses the ABI.
 *     On error, output handles are set to NULL and nothing is leaked.
 */
#ifndef HSOLVE_H
#define HSOLVE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HS_OK = 0,
    HS_ERR_ARG = 1,         /* invalid argument (sizes, pointers, options)       */
    HS_ERR_NOT_SPD = 2,     /* a diagonal block lost definiteness (Sec. 2, after
                               Prop. 1): hs_info.fail_level / fail_cluster      */
    HS_ERR_NOCONV = 3,      /* Krylov did not reach rtol within maxit            */
    HS_ERR_CUDA = 4,        /* a CUDA call failed                                */
    HS_ERR_OOM = 5,         /* device allocation failed                          */
    HS_ERR_UNSUPPORTED = 6, /* a block is larger than the kernels support        */
    HS_ERR_TIMEOUT = 7      /* a bounded device wait gave up                     */
} hs_status;

enum { HS_MEM_HOST = 0, HS_MEM_DEVICE = 1 };
enum { HS_PREC_FP64 = 0, HS_PREC_MIXED = 1 };
enum { HS_KRYLOV_PCG = 0, HS_KRYLOV_GMRES = 1 };
enum { HS_PRODUCTS_FP32 = 0, HS_PRODUCTS_TF32X3 = 1, HS_PRODUCTS_TF32 = 2, HS_PRODUCTS_BF16 = 3 };
enum { HS_PART_AUTO = 0, HS_PART_MULTILEVEL = 1 };

/* Partition tree: leaf c owns the DOFs perm[leaf_ptr[c] .. leaf_ptr[c+1]);
 * siblings 2c, 2c+1 merge at the next level (Sec. 4.2, Sec. 5).  n_leaf must
 * be divisible by 2^depth. */
typedef struct {
    int32_t n_leaf;
    int32_t* perm;      /* n entries, host memory */
    int32_t* leaf_ptr;  /* n_leaf + 1 entries, host memory */
    int32_t depth;      /* elimination levels before the dense top */
} hs_tree;

typedef struct {
    double tol;          /* compression tolerance eps (absolute on the scaled
                            block G^-1 A_sw, Eq. offdiag_new); default 1e-2  */
    int32_t depth;       /* levels; -1 = log2(n_leaf) - 2 (top of 8 clusters) */
    int32_t leaf_lines;  /* partitioner: vertical lines per leaf (default 4)   */
    double theta;        /* partitioner: strong-coupling threshold (0.5)       */
    int32_t precision;   /* HS_PREC_FP64 or HS_PREC_MIXED                      */
    int32_t krylov;      /* HS_KRYLOV_PCG or HS_KRYLOV_GMRES                   */
    int32_t restart;     /* GMRES restart length (default 50)                  */
    double rtol;         /* Krylov stop: ||b - A x|| / ||b|| (default 1e-8)    */
    int32_t maxit;       /* Krylov iteration cap (default 1000)                */
    int32_t mem;         /* HS_MEM_HOST or HS_MEM_DEVICE                       */
    int32_t profile;     /* nonzero: CUDA-event timing of every kernel class   */
    void* stream;        /* cudaStream_t for all device work                   */
    const double* coords; /* host n x 2 horizontal DOF positions for the
                            partitioner when no tree is given (NULL: BFS)     */
    int32_t coarse_dense; /* solve phase: the levels from one with at most
                            this many DOFs (and the top) are applied as one
                            explicit dense operator formed at setup; the
                            level is picked by a cost model of forming it
                            plus ten applies; 0 = never; default 4096         */
    int32_t fused_levels; /* nonzero (default): levels whose clusters have at
                            most 32 DOFs run all their phases in one launch   */
    int32_t record_ranks; /* nonzero: keep the rank predictor's features and
                            the rank of every eliminated cluster for
                            hs_rank_samples (default 0)                       */
    const float* rank_model; /* NULL (default), or a trained rank predictor
                            (host, HS_MLP_MODEL floats: feature means (8),
                            deviations (8), network parameters).  Mixed form
                            only, for clusters of at least 16 DOFs with
                            dense fill columns on the per-cluster kernel: a
                            cluster predicted to have rank 0 scales those
                            columns in FP32 only; if the FP32 result plus a
                            forward-error bound of the FP32 substitution
                            (from ||G^-1||_F, the input norm and
                            || |G| |result| ||_F) proves ||G^-1 A_sw||_F <=
                            eps, its rank is 0 and the FP64 scaling of those
                            columns and the QR are skipped; otherwise they
                            are scaled again in FP64 and the column-pivoted
                            QR decides as usual.  Copied during hs_setup.   */
    int32_t no_dc;       /* 0 (default): deferred compression (Sec. 2: A_sw
                            scaled by G_s^-1 before it is compressed, Eq.
                            offdiag_new).  1: without it, the original
                            LoRaSp step that Sec. 2 compares against: the
                            unscaled A_sw compressed (Eq. offdiag) at the
                            threshold eps * sqrt(max_i (A_ss)_ii), the row
                            rotated and the fine DOFs eliminated by Cholesky
                            of the rotated fine block, which also updates the
                            coarse DOFs.  For comparing the two schemes;
                            every level runs the per-phase kernel (FP64
                            compression in both precision forms); not with
                            rank_model or record_ranks (HS_ERR_UNSUPPORTED). */
    int32_t wait_polls;  /* bounded device waits (the grid barrier between the
                            phases of a level factored in one launch): polls
                            before the launch gives up with HS_ERR_TIMEOUT.
                            0 (default): about a second; > 0: that many;
                            < 0: none, the first wait gives up at once (for
                            testing the timeout path).  A launch that gives
                            up returns at once, and the call returns
                            HS_ERR_TIMEOUT without a handle.                 */
    int32_t schur_products; /* mixed form, Schur update X_nn -= C^T C (Eq.
                            elim) of the per-phase levels (default
                            HS_PRODUCTS_TF32X3): HS_PRODUCTS_FP32
                            (FP32 products on the CUDA cores),
                            HS_PRODUCTS_TF32X3 (tensor cores: each FP32
                            entry split into two TF32 parts, three products,
                            about 2^-21 relative error per product) or
                            HS_PRODUCTS_TF32 (tensor cores, one TF32
                            product, about 2^-11) or HS_PRODUCTS_BF16
                            (tensor cores, BF16 products, about 2^-8); FP32
                            accumulation and an FP64 block store in every
                            case.  Ignored by the FP64 form.                 */
    int32_t partitioner;  /* when no tree is given: HS_PART_AUTO (default:
                            coordinate bisection with coords, else BFS
                            graph growing) or HS_PART_MULTILEVEL (the
                            multilevel graph bisection of
                            hs_partition_multilevel; coords ignored)         */
} hs_options;

typedef struct {
    int32_t iters;        /* Krylov iterations (PCG steps / GMRES inner steps) */
    double rel_resid;     /* final true relative residual                      */
    double setup_s;       /* partition + symbolic + numeric factorization      */
    double solve_s;       /* Krylov solve                                      */
    int32_t fail_level;   /* where HS_ERR_NOT_SPD happened, else -1            */
    int32_t fail_cluster;
    int64_t factor_bytes; /* device bytes held by the factor                   */
} hs_info;

typedef struct hs_factor_s* hs_handle;

/* Fill *opt with the defaults listed above. */
int hs_default_options(hs_options* opt);

/* Column-preserving partition (Sec. 4.2): strongly coupled vertical lines
 * (|a_ij| >= theta * max_k!=i |a_ik|) stay in one cluster; the line graph is
 * bisected recursively (coords: n x 2 horizontal positions, or NULL for BFS
 * graph growing) into 2^L leaves of at most leaf_lines lines.  Host pointers.
 * out->perm / out->leaf_ptr are allocated by the library; release them with
 * hs_tree_free. */
int hs_partition_extruded(int64_t n, const int64_t* rowptr, const int32_t* col,
                          const double* val, const double* coords, int32_t leaf_lines,
                          double theta, hs_tree* out);

/* The same partition from the matrix alone (Sec. 4.2 with a graph
 * partitioner in place of coordinates; Sec. 6 on black-box use): the lines
 * are found as above, then the weighted line graph (an edge per pair of
 * lines sharing a nonzero, weight = sum of |a_ij| over those nonzeros) is
 * bisected recursively by a multilevel method (heavy-edge matching,
 * graph growing on the coarsest graph, Fiduccia-Mattheyses refinement on
 * the way back up) into ceil(k/2) and floor(k/2) lines at every split.  The
 * result depends only on the matrix (not on the thread count).  Arguments,
 * ownership and errors as for hs_partition_extruded. */
int hs_partition_multilevel(int64_t n, const int64_t* rowptr, const int32_t* col,
                            const double* val, int32_t leaf_lines, double theta, hs_tree* out);
int hs_tree_free(hs_tree* t);

/* Phase plan of one level (host only, no device work; the same code the
 * setup runs).  Input: the level's block graph over nc clusters as CSR
 * (adj_ptr[nc+1] int64, adj sorted per row, symmetric, no self loops) and
 * each cluster's size (a cluster of size 0 has no blocks and no phase).
 * Algorithm 1 eliminates the clusters one at a time in an order it leaves
 * open; here phases are repeated greedy maximal independent sets (ascending
 * cluster index) of the unprocessed clusters in the current block graph.
 * Eliminating a cluster couples every pair of its neighbours in the level's
 * input graph (Sec. 3.1, Eq. elim), and a cluster none of whose blocks is
 * fill leaves the graph (rank 0).  ranges: nranges pairs [lo, hi) of
 * consecutive clusters covering [0, nc) with no block between two ranges
 * (independent problems, planned on separate threads), or nranges = 0.
 * Output (caller-owned host arrays): phase[nc] (-1 for size 0), vanished[nc]
 * (1 = left the graph), end_ptr[nc+1] and, when end_adj is not NULL,
 * end_adj[end_cap] with each cluster's blocks at the level's end (sorted,
 * including itself unless it left or has size 0); all_ptr[nc+1] and, when
 * all_adj is not NULL, all_adj[all_cap] with every block that existed at
 * some point of the level (sorted, with the cluster itself unless it has
 * size 0: the level's block store).  HS_ERR_ARG on malformed input or a
 * capacity below end_ptr[nc] / all_ptr[nc] (the pointer arrays are filled
 * first, so a call with NULL lists queries the sizes). */
int hs_plan_level(int32_t nc, const int64_t* adj_ptr, const int32_t* adj, const int32_t* size0, int32_t nranges,
                  const int32_t* ranges, int32_t* phase, int32_t* vanished, int64_t* end_ptr, int32_t* end_adj,
                  int64_t end_cap, int64_t* all_ptr, int32_t* all_adj, int64_t all_cap);

/* Hierarchical_Factor (Algorithm 1): scaled low-rank elimination of every
 * cluster, level by level, then dense Cholesky of the top.  tree may be NULL
 * (then hs_partition_extruded, or hs_partition_multilevel when
 * options->partitioner says so, runs on options->coords, options->leaf_lines,
 * options->theta, and options->depth applies).  CSR in options->mem.  On HS_ERR_NOT_SPD the
 * failing (level, cluster) is written to *info when info is not NULL.
 * With device inputs the pattern (and, for the partitioner, the values) is
 * read back into a pinned host buffer that the calling thread keeps for
 * later calls (freed when the thread exits). */
int hs_setup(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val,
             const hs_tree* tree, const hs_options* opt, hs_handle* out, hs_info* info);

/* Hierarchical_Solve (Algorithm 2): z = M^-1 r, device pointers, n doubles
 * each, stream-ordered on the handle's stream; r and z may not alias. */
int hs_apply(hs_handle h, const double* r, double* z);

/* Preconditioned Krylov solve with the factored handle (PCG, or GMRES(restart)
 * with FP64 true-residual restarts): x0 = 0, stops at rel. residual <= rtol.
 * b, x device pointers. */
int hs_krylov(hs_handle h, const double* b, double* x, hs_info* info);

/* Allocation-free PCG solve with an existing handle.  No counterpart in the
 * paper: it is for callers that cannot allocate device memory when they
 * solve, for example a time-stepping loop inside a host application whose own
 * allocator owns all device memory, or code that must not call
 * cudaMalloc/cudaFree (which synchronise the device) after initialisation.
 * It runs the same PCG as hs_krylov, but the four work vectors and the
 * dot-product partial sums live in a fixed array compiled into the library
 * (static __device__, 256-byte aligned, 4 * 262144 + 1040 doubles, about
 * 8.4 MB, held on every GPU that loads the library until the process exits).
 * Limits: n <= 262144 (else HS_ERR_ARG); a handle from hs_setup with
 * HS_KRYLOV_PCG (a GMRES handle or a batched handle from hs_setup_batched,
 * whose problems each stop on their own residual, gives HS_ERR_UNSUPPORTED);
 * the current CUDA device must be the one the handle was set up on (else
 * HS_ERR_ARG, before any device work).  The first call on a device looks
 * up the array's device address and caches it; make that first call before
 * any stream capture.  All calls share the one array and it keeps the last
 * call's contents (this call zeroes or writes everything it reads): calls
 * whose device work overlaps in time (several streams, threads or handles at
 * once) race and return wrong results.  b, x: device pointers, n doubles.
 * Allocates nothing: no cudaMalloc / cudaFree and no allocating library call. */
int hs_krylov_noalloc(hs_handle h, const double* b, double* x, hs_info* info);

/* Batched setup: nprob independent problems in one handle (no counterpart in
 * the paper, which factors one operator; each problem gets exactly the
 * factorization hs_setup would give it alone).  The problems come as one
 * block-diagonal CSR of order n: problem p owns rows and columns
 * prob_ptr[p] .. prob_ptr[p+1] (host array, nprob + 1 entries, prob_ptr[0] = 0,
 * prob_ptr[nprob] = n, every problem non-empty) and no entry may couple two
 * problems (else HS_ERR_ARG).  Each problem is partitioned on its own
 * (options->coords rows of that problem, leaf_lines, theta) with its own
 * default depth (or options->depth for all); every problem needs at least two
 * leaves.  Level l of the handle holds level l of every problem that still
 * has one (problem after problem), so each level of all problems is factored
 * by the same launches, and a problem whose levels are done gets its own
 * dense top.  hs_apply works on the whole block-diagonal system;
 * hs_krylov / hs_krylov_batched run one PCG per problem (only
 * HS_KRYLOV_PCG); hs_top_size gives the sum of the tops.  nprob <= 65535. */
int hs_setup_batched(int32_t nprob, const int64_t* prob_ptr, int64_t n, const int64_t* rowptr,
                     const int32_t* col, const double* val, const hs_options* opt, hs_handle* out,
                     hs_info* info);

/* PCG on every problem of a batched handle (x0 = 0; problem p stops when its
 * own ||b_p - A_p x_p|| / ||b_p|| <= rtol, checked on the true residual).  All
 * problems share each preconditioner apply and SpMV; the rest is per problem.
 * b, x: device, n doubles.  iters, rel_resid: host arrays of nprob entries
 * (may be NULL).  info: the largest count and residual over the problems.
 * HS_ERR_NOCONV if some problem is still above rtol after maxit iterations;
 * HS_ERR_UNSUPPORTED for a handle from hs_setup. */
int hs_krylov_batched(hs_handle h, const double* b, double* x, int32_t* iters, double* rel_resid,
                      hs_info* info);

/* Problems in the handle (1 for hs_setup handles) and, for problem prob, its
 * leaf range in the level-0 cluster numbering, its depth and its top size. */
int hs_num_problems(hs_handle h, int32_t* nprob);
int hs_problem_info(hs_handle h, int32_t prob, int32_t* leaf_lo, int32_t* leaf_hi, int32_t* depth,
                    int32_t* ntop);

/* Partition + setup + Krylov in one call; pointers in opt->mem. */
int hs_solve(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val,
             const double* b, double* x, const hs_options* opt, hs_info* info);

/* Release the handle and all device memory it owns (NULL is accepted). */
int hs_destroy(hs_handle h);

/* Introspection (host outputs): levels, per-cluster start size / final
 * size (rank, 0 if eliminated) / phase of level l, dense top size. */
int hs_num_levels(hs_handle h, int32_t* levels);
int hs_level_clusters(hs_handle h, int32_t level, int32_t* nc);
int hs_level_info(hs_handle h, int32_t level, int32_t* size0, int32_t* final_size,
                  int32_t* phase);
int hs_top_size(hs_handle h, int32_t* ntop);

/* Kernel classes: 0 factor phase (Cholesky + scaling + CPQR + write-back,
 * one launch per phase), 1 Schur update, 2 level assembly, 3 dense top (and
 * forming the dense coarse operator), 4 preconditioner apply, 5 Krylov
 * vector kernels (dots, updates), 6 fused coarse-level factor kernel (all
 * phases of a level in one launch), 7 SpMV.  For each class k < nclasses
 * (host arrays, any may be NULL): device milliseconds summed over its
 * launches since setup (CUDA events on the handle's stream; only when
 * options.profile was set), the number of launch sites used, and the
 * algorithmic work of the paper's dense counts, split into the flops done in
 * FP64 (flops64) and in FP32 (flops32: the mixed form's compression and
 * Schur products): POTRF s^3/3 and scaling s^2 (n+w) in FP64; CPQR
 * sum_k 4 (s-k)(w-k) + 4 s r n and Schur n^2 f in the form's compression /
 * product precision; and bytes (assembly 20 per nonzero; apply: the stored
 * factor twice, three vectors per level, the dense coarse operator or top,
 * the two permutations; SpMV 12 nnz + 24 n per product). */
int hs_kernel_stats(hs_handle h, int32_t nclasses, double* times_ms, int64_t* launches, double* flops64,
                    double* flops32, double* bytes);
int hs_reset_kernel_stats(hs_handle h);

/* Number of this library's kernels launched by the process so far (a kernel
 * inside the solve-phase CUDA graph counts once per graph launch). */
int hs_launch_count(int64_t* count);

/* Self-check of the reciprocals the factor kernels use for their Cholesky
 * pivots (Sec. 2: G_s with A_ss = G_s G_s^T) and Householder scalars:
 * rsqrt_out[i] = 1 / sqrt(x[i]) and rcp_out[i] = 1 / x[i], each an FP32
 * estimate refined by two Newton-Raphson steps in FP64 (the FP64 square root
 * and division outside 1e-30 < x < 1e30).  x, rsqrt_out, rcp_out: device
 * arrays of n doubles, caller-owned; x > 0.  Returns after completion. */
int hs_eval_pivot_reciprocals(int64_t n, const double* x, double* rsqrt_out, double* rcp_out, void* stream);

/* Measures the FP64 FMA throughput of the current device with a chain of
 * independent fma() operations (8 per thread, 8 CTAs per SM); TFLOP/s out. */
int hs_measure_fp64_peak(void* stream, double* tflops);

/* The same probe on the FP32 pipe (fmaf chains), TFLOP/s out: the peak that
 * the mixed form's FP32 compression and Schur products are measured against. */
int hs_measure_fp32_peak(void* stream, double* tflops);

/* ---- Rank predictor ----
 * No counterpart in the paper.  A three-layer perceptron of width 64 maps 8
 * features of a scaled block row (the block G^-1 [A_sn A_sw] whose
 * column-pivoted QR decides the rank, Sec. 3.1) to the fraction r / s of its
 * numerical rank; the factorization can record (features, rank) pairs of
 * every cluster it eliminates (hs_rank_samples) to train it on.  FP32.
 * Parameter vector (HS_MLP_NPARAM floats): W1 (64 x 8, row-major), b1 (64),
 * W2 (64 x 64, row-major), b2 (64), w3 (64), b3 (1);
 * h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), y = w3 . h2 + b3; loss over a
 * batch (1/B) sum (y - t)^2; Adam with beta1 0.9, beta2 0.999, eps 1e-8. */
#define HS_MLP_NIN 8
#define HS_MLP_NPARAM 4801
#define HS_MLP_MAX_BATCH 256
#define HS_MLP_MODEL (2 * HS_MLP_NIN + HS_MLP_NPARAM)

/* y[i] = network(x[i * 8 .. i * 8 + 8)) for i < n.  Device pointers; stream-ordered. */
int hs_mlp_forward(const float* params, const float* x, int64_t n, float* y, void* stream);

/* Loss and gradient of one minibatch: rows idx[0..batch) of x (n x 8) and t
 * (idx may be NULL: rows 0..batch).  batch in 1..HS_MLP_MAX_BATCH.  grad:
 * HS_MLP_NPARAM floats, loss: 1 float.  Device pointers; stream-ordered;
 * deterministic (fixed summation order). */
int hs_mlp_grad(const float* params, const float* x, const float* t, const int32_t* idx, int32_t batch,
                float* grad, float* loss, void* stream);

/* One Adam update of params with grad (step counts from 1); m, v: moment
 * vectors (HS_MLP_NPARAM floats, zero before step 1).  Device pointers. */
int hs_mlp_adam(float* params, const float* grad, float* m, float* v, int32_t step, float lr, void* stream);

/* Minibatch training on the GPU: step k (k < nsteps) takes the samples
 * order[k * batch .. (k + 1) * batch) of x (n x 8) / t (n) and applies
 * hs_mlp_grad + hs_mlp_adam.  Host arrays: params (in: initial, out:
 * trained), x, t, order (nsteps * batch indices < n), losses (nsteps floats,
 * the loss before each update; may be NULL).  Returns after completion. */
int hs_mlp_train(float* params, const float* x, const float* t, int64_t n, const int32_t* order, int64_t nsteps,
                 int32_t batch, float lr, float* losses, void* stream);

/* (features, rank, size) of every cluster the factorization eliminated, in
 * level order and, within a level, in elimination order; the handle must
 * have been set up with options.record_ranks.  Host arrays: feat count x 8
 * floats, rank and size count int32 each; pass feat = NULL to query *count.
 * Features (all known before the scaling step): 0 s (rows of the block
 * row), 1 n columns (neighbour blocks of the level input), 2 fill columns,
 * 3 level, 4 blocks in the row, 5 log10 of ||D^-1 A_sw||_F / eps with D the
 * diagonal of the Cholesky factor G, 6 log10 of max |A_ss| off its diagonal
 * over max |[A_sn A_sw]|, 7 log10 of the largest column norm of D^-1 A_sw
 * over eps (5 and 7 are -30 when the cluster has no fill columns or a zero
 * fill block, and at least -30 otherwise; 6 is clamped to [-30, 30]).  The
 * norms are formed in FP32 from the entries' magnitudes truncated to 20
 * mantissa bits, and the logarithms are FP32. */
int hs_rank_samples(hs_handle h, float* feat, int32_t* rank, int32_t* size, int64_t* count);

/* Static string for a status code. */
const char* hs_status_str(int status);

#ifdef __cplusplus
}
#endif

#endif /* HSOLVE_H */
