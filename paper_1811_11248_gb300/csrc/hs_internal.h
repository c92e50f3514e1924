// hs_internal.h -- records shared by the host planner (hs_host.cpp) and the
// sm_103a kernels (hs_kernels.cu).  All records are plain int32/int64 so the
// host builds them once per level and uploads them with one copy.
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

namespace hs {

// One cluster elimination ("scaled low-rank elimination", Sec. 3.1) of a
// phase.  Column blocks of the cluster's row are listed n-neighbours first,
// then fill ("w") blocks, each with its current width read on the device.
// Vector slice copy (coarse parts between levels).  to_top: the destination is
// the top vector (the cluster's problem ends at this level) instead of the next
// level's vector.
struct VCopyDev {
    int64_t src, dst;
    int32_t len, to_top;
};

// Dense top of one problem: L (n x n, row-major, lower after factorization)
// and the offset of its vector in the top vector.
struct TopDev {
    double* L;
    int64_t vec_off;
    int32_t n, pad;
};

struct TaskDev {
    int32_t c;         // cluster id at this level
    int32_t s;         // its size when processed (= size at level start)
    int32_t nn, nw;    // neighbour / fill block counts
    int32_t list;      // first ListDev entry
    int32_t diag_blk;  // block index of (c, c)
    int32_t ncap;      // sum of level-start sizes of the n-neighbours (ld of C)
    int32_t wcap;      // same over n and w (capacity of the block row)
    int32_t meta;      // first int of: rank, then (col offset, width) per n-neighbour
    int32_t pad;
    int64_t w_off;     // W = U^T G^-1 (s x s, row-major) in the factor array
    int64_t c_off;     // C = fine rows of U^T G^-1 A_sn ((s - r) x ncap)
    int64_t m_off;     // block-row workspace (s x (wcap + s)) in the workspace array
};

// ---- solve phase (Algorithm 2), records built on the host after a level is
// factored, with every offset resolved so that a kernel reads each operand in
// one round of loads.
struct ApTask {
    int64_t y;        // slot of the cluster in the level vector
    int64_t w;        // W = U^T G^-1 (s x s, row-major) in the factor array
    int64_t cm;       // C ((s - r) x ncap) in the factor array
    int64_t stg;      // staged update C^T y_fine (ncols) in the stage array
    int32_t s, r, ncols, ncap;
    int32_t pull0, pull1;  // staged updates subtracted before the transform
    int32_t nb0, nb1;      // neighbour slices read by the backward step
};
// A staged update y_q -= C_t(:, q)^T y_t(fine) of task t's neighbour q: its
// offset in the stage array (its length is q's width when t was processed).
struct ApPull {
    int64_t off;
};
struct ApNb {
    int64_t y;       // neighbour's slot in the level vector
    int32_t col, m;  // its first column in C and its width
};
// End-of-level forward step of a cluster with a coarse part: subtract the
// updates of tasks processed after it, copy the coarse part to the parent slot.
struct ApFin {
    int64_t y, dst;
    int32_t len, pull0, pull1, to_top;
};
// One level of the single-CTA coarse-levels kernel.
struct ApLevel {
    const ApTask* tasks;
    const int32_t* ph;  // phase ranges (nph + 1)
    const ApPull* pulls;
    const ApNb* nbs;
    const ApFin* fins;
    const VCopyDev* vcopy;
    const void* fac;  // double, or float in the mixed-precision form
    double* stage;
    double* y;
    double* ynext;
    int32_t nph, nfin, nvcopy, pad;
};

struct ListDev {
    int32_t q;       // neighbour / fill cluster
    int32_t blk_cq;  // block index of (c, q)
    int32_t blk_qc;  // block index of (q, c)
    int32_t pad;
};

// Schur target: block (p, q), p <= q, of one phase; contributions from the
// phase's tasks that have both p and q as n-neighbours, in ascending task order.
struct TargetDev {
    int32_t p, q, blk_pq, blk_qp, c_begin, c_end;
};

struct ContribDev {
    int32_t task, kp, kq;  // task index (in the level's task array), positions of p, q in its n-list
};

// Dense copy of a rows x cols sub-block (level assembly, top assembly).
struct CopyDev {
    int64_t src, dst;   // element offsets
    int32_t src_ld, dst_ld, rows, cols;
};


// status word written by kernels (0 = ok)
enum : int32_t { ST_OK = 0, ST_NOT_SPD = 1, ST_TOO_BIG = 2, ST_TIMEOUT = 3 };

// ---- kernel launchers (hs_kernels.cu) -------------------------------------
// *bad |= 1 unless rowptr[0] == 0, rowptr is non-decreasing over [0, n] and
// every col[e], e < nnz, lies in [0, n)
cudaError_t launch_check_csr(cudaStream_t st, int64_t n, int64_t nnz, const int64_t* rowptr, const int32_t* col,
                             int32_t* bad);
cudaError_t launch_scatter_csr(cudaStream_t st, int64_t n, const int64_t* rowptr, const int32_t* col,
                               const double* val, const int32_t* dof_cluster, const int32_t* dof_local,
                               const int32_t* blk_ptr, const int32_t* blk_col, const int64_t* blk_off,
                               const int32_t* blk_ld, double* blocks);
cudaError_t launch_factor_phase(cudaStream_t st, const TaskDev* tasks, int t0, int ntasks, int smax,
                                int wmax, int lmax, const ListDev* lists, double* blocks, const int64_t* blk_off,
                                const int32_t* blk_ld, int32_t* cur, void* fac, int fp32, int32_t* meta,
                                double* ws, double eps2, int32_t* status, int32_t level, float* feat,
                                const float* model);
// the elimination step without deferred compression (hs_nodc.cu): one CTA
// per task, same records and outputs as launch_factor_phase
size_t factor_nodc_smem_bytes(int smax, int wmax, int lmax);
cudaError_t launch_factor_nodc(cudaStream_t st, const TaskDev* tasks, int t0, int ntasks, int smax, int wmax,
                               int lmax, const ListDev* lists, double* blocks, const int64_t* blk_off,
                               const int32_t* blk_ld, int32_t* cur, void* fac, int fp32, int32_t* meta, double* ws,
                               double eps2, int32_t* status, int32_t level);
// products of the mixed form's Schur update: FP32 on the CUDA cores, or
// tensor-core products: TF32 (one pass, or three with the hi/lo split), BF16
enum { kProductsFp32 = 0, kProductsTf32x3 = 1, kProductsTf32 = 2, kProductsBf16 = 3 };
cudaError_t launch_schur_phase(cudaStream_t st, const TargetDev* targets, int g0, int ntargets,
                               const ContribDev* contribs, const TaskDev* tasks, const void* fac,
                               const int32_t* meta, double* blocks, const int64_t* blk_off,
                               const int32_t* blk_ld, const int32_t* cur, int fp32, int products);
cudaError_t launch_copy_blocks(cudaStream_t st, const CopyDev* cps, int ncps, const double* src,
                               double* dst);
cudaError_t launch_dense_cholesky(cudaStream_t st, int n, double* a, int32_t* status);
cudaError_t launch_ap_fwd(cudaStream_t st, const ApTask* tasks, int t0, int ntasks, int smax,
                          const ApPull* pulls, const void* fac, int fp32, double* stage, double* y);
cudaError_t launch_ap_fin(cudaStream_t st, const ApFin* fins, int nfin, const ApPull* pulls, const double* stage,
                          double* y, double* ynext, double* ytop);
cudaError_t launch_ap_bwd(cudaStream_t st, const ApTask* tasks, int t0, int ntasks, int smax, int nmax,
                          const ApNb* nbs, const void* fac, int fp32, double* y);
// levels lvl[0..nlev) forward, dense top, then backward, in one CTA
constexpr int kCoarseThreads = 1024;
constexpr int kCoarseSmax = 64;   // largest cluster the coarse kernel handles
constexpr int kCoarseNmax = 320;  // largest neighbour width (ncols) it handles
cudaError_t launch_ap_coarse(cudaStream_t st, const ApLevel* lvl, int nlev, int ntop, const double* L,
                             double* ytop, int fp32);
// explicit coarse operator (one CTA per unit vector) and its application
cudaError_t launch_ap_coarse_batch(cudaStream_t st, const ApLevel* lvl, int nlev, int ntop, const double* L,
                                   double* ytop0, double* yin0, int n, int64_t stride, double* Mc, int fp32);
cudaError_t launch_dense_gemv(cudaStream_t st, int n, const double* Mc, const double* x, double* y);
cudaError_t launch_vcopy(cudaStream_t st, const VCopyDev* cps, int ncps, const double* src, double* dst,
                         int reverse, const double* ytop);
// dense tops of several problems: Cholesky / forward+backward solve, one CTA each
cudaError_t launch_tops_cholesky(cudaStream_t st, const TopDev* tops, int ntops, int32_t* status);
cudaError_t launch_tops_solve(cudaStream_t st, const TopDev* tops, int ntops, double* ytop);
cudaError_t launch_top_solve(cudaStream_t st, int n, const double* L, double* y);
cudaError_t launch_permute(cudaStream_t st, int64_t n, const int32_t* perm, const double* src, double* dst,
                           int inverse);
cudaError_t launch_spmv(cudaStream_t st, int64_t n, const int64_t* rowptr, const int32_t* col,
                        const double* val, const double* x, double* y);
// partial sums for dot products: out[k] for k < nparts, then a final pass
cudaError_t launch_dot(cudaStream_t st, int64_t n, const double* a, const double* b, double* partial,
                       double* out);
// y = a*x + y with device scalar alpha = num/den (sign), etc.
// fused PCG steps (*count: a zeroed counter, left zeroed; partial: kDotParts doubles)
cudaError_t launch_spmv_dot(cudaStream_t st, int64_t n, const int64_t* rowptr, const int32_t* col, const double* val,
                            const double* x, double* y, double* partial, unsigned* count, double* out);
cudaError_t launch_pcg_xr_dot(cudaStream_t st, int64_t n, const double* rz, const double* pq, const double* p,
                              const double* q, double* x, double* r, double* partial, unsigned* count, double* out);
cudaError_t launch_dot_fused(cudaStream_t st, int64_t n, const double* a, const double* b, double* partial,
                             unsigned* count, double* out);
cudaError_t launch_pcg_update_xr(cudaStream_t st, int64_t n, const double* rz, const double* pq,
                                 const double* p, const double* q, double* x, double* r);
cudaError_t launch_pcg_update_p(cudaStream_t st, int64_t n, const double* rz_new, const double* rz_old,
                                const double* z, double* p);
cudaError_t launch_axpby(cudaStream_t st, int64_t n, double a, const double* x, double b, double* y);
// batched PCG over independent problems (segments pp[p] .. pp[p+1])
constexpr int kBScal = 8;  // per-problem scalars
enum { BS_RZ = 0, BS_PQ = 1, BS_RZN = 2, BS_RR = 3, BS_BB = 4, BS_RRT = 5, BS_REL = 6 };
constexpr int kBFlag = 4;  // per-problem flags
enum { BF_ACTIVE = 0, BF_RESTART = 1, BF_CAND = 2, BF_ITERS = 3 };
cudaError_t launch_seg_dot(cudaStream_t st, int nprob, const int64_t* pp, const double* a, const double* b,
                           double* sc, int slot);
// op 0: x(c) += alpha p(a), r(d) -= alpha q(b); op 1: p(c) = z(a) + beta p(c);
// op 2: r(c) = q(a) where restarted.  Grid: (maxlen / 256, nprob).
cudaError_t launch_bpcg_vec(cudaStream_t st, int op, int nprob, int64_t maxlen, const int64_t* pp, const double* sc,
                            const int32_t* fl, const double* a, const double* b, double* c, double* d);
cudaError_t launch_bpcg_book(cudaStream_t st, int nprob, int mode, double rtol, double* sc, int32_t* fl,
                             int32_t* cnt);

cudaError_t launch_gmres_update(cudaStream_t st, int64_t n, int k, const double* coef, const double* V,
                                int64_t ldv, double* y, double sign);
cudaError_t launch_gemv_t(cudaStream_t st, int64_t n, int k, const double* V, int64_t ldv,
                          const double* w, double* partial, double* out);

size_t factor_smem_bytes(int smax, int wmax, int lmax, bool xsh = false);
// coarse levels: all phases of a level in one single-CTA launch (warp per task)
constexpr int kFusedWarps = 16, kFusedSmax = 32;
// A fused level runs in one thread-block cluster of kClusterCtas CTAs when
// every phase's tasks fit its warps in one round and its Schur targets take
// at most kClusterTargetRounds rounds per phase on average.
constexpr int kClusterCtas = 16, kClusterWarps = kClusterCtas * kFusedWarps, kClusterTargetRounds = 2;
size_t fused_smem_bytes(int smax, int wmax, int lmax, int64_t mcap);
cudaError_t launch_factor_level_fused(cudaStream_t st, const TaskDev* tasks, const int32_t* ph_task,
                                      const TargetDev* targets, const int32_t* ph_target, const ContribDev* contribs,
                                      int nph, const ListDev* lists, double* blocks, const int64_t* blk_off,
                                      const int32_t* blk_ld, int32_t* cur, void* fac, int fp32, int32_t* meta,
                                      double* ws, double eps2, int32_t* status, int32_t level, int smax, int wmax,
                                      int lmax, int64_t mcap, int max_items, unsigned* bar, float* feat,
                                      const float* model, int wait_polls, int cluster_ok);
// process-wide count of this library's kernel launches
// rank predictor (hs_mlp.cu): 8 -> 64 -> 64 -> 1 perceptron, FP32
constexpr int kMlpIn = 8, kMlpHidden = 64;
constexpr int kFeat = kMlpIn;  // features recorded per eliminated cluster
constexpr int kSparseNz = 4;   // scaling: columns with at most this many nonzeros use the columns of G^-1
constexpr int kMlpParams = kMlpHidden * kMlpIn + kMlpHidden + kMlpHidden * kMlpHidden + kMlpHidden + kMlpHidden + 1;
constexpr int kMlpMaxBatch = 256, kMlpThreads = 512;
constexpr int kModelFloats = 2 * kMlpIn + kMlpParams;  // mu, sd, network
constexpr float kAdamBeta1 = 0.9f, kAdamBeta2 = 0.999f, kAdamEps = 1e-8f;
size_t mlp_grad_smem_bytes();
cudaError_t launch_mlp_forward(cudaStream_t st, const float* theta, const float* x, int64_t n, float* y);
cudaError_t launch_mlp_grad(cudaStream_t st, const float* theta, const float* x, const float* t, const int32_t* idx,
                            int B, float* grad, float* loss);
cudaError_t launch_mlp_adam(cudaStream_t st, float* theta, const float* grad, float* m, float* v, int step,
                            float lr);
int64_t launch_count();
void launch_count_add(int64_t k);
cudaError_t launch_fp64_peak(cudaStream_t st, int nblocks, int iters, double* sink);
cudaError_t launch_fp32_peak(cudaStream_t st, int nblocks, int iters, double* sink);
// rs[i] = 1 / sqrt(x[i]) and rc[i] = 1 / x[i] by the Cholesky pivot helpers
cudaError_t launch_eval_recip(cudaStream_t st, int64_t n, const double* x, double* rs, double* rc);

constexpr int kDotParts = 1024;
// allocation-free PCG: largest n, scratch layout r | z | p | q | partials | scalars
constexpr int64_t kNoAllocMaxN = 262144;
constexpr int64_t kNoAllocDoubles = 4 * kNoAllocMaxN + kDotParts + 16;
constexpr int kNoAllocMaxDevices = 64;
// device address of the static scratch on the current device (looked up once per device)
cudaError_t noalloc_scratch(double** ptr);
constexpr int kFactorMaxSmem = 226 * 1024;  // dynamic part; static shared adds a few bytes

// Multilevel bisection (hs_mlpart.cpp) of a weighted graph: CSR ptr[n+1],
// adj, w (symmetric, no self loops, w > 0).  part[v] = 0 for exactly na
// vertices (0 <= na <= n), 1 for the rest, chosen for a small edge cut.
void ml_bisect(int n, const int* ptr, const int* adj, const double* w, int na, std::vector<char>& part);
// partitioner methods of partition_impl
enum { kPartAuto = 0, kPartMultilevel = 1 };

}  // namespace hs
