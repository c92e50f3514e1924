// hs_kernels.cu -- sm_103a kernels of the hierarchical solver.
//
// Factorization (Algorithm 1), per phase of independent clusters:
//   k_factor_phase       : one CTA per cluster (512 threads, or 1024 when a
//                          phase has no more clusters than SMs): Cholesky of
//                          A_ss together with G^-1 (Sec. 2), scaling
//                          G^-1 [A_sn A_sw] (Eq. scaling; sparse level-0
//                          columns as combinations of columns of G^-1),
//                          column-pivoted QR of the scaled fill block with
//                          every reflector applied to the whole row (Eq.
//                          offdiag_new, Eq. sparse; FP32 in the mixed form),
//                          write-back of the coarse row (Eq. perm) and of the
//                          factor {W = U^T G^-1, C, r}.
//   k_factor_level_fused : all phases of a coarse level in one launch, one
//                          warp per cluster (clusters of at most 8 DOFs with
//                          the block row in registers): one thread-block
//                          cluster with the hardware cluster barrier between
//                          phases, else a cooperative launch with a bounded
//                          grid barrier.
//   k_schur_phase(_tc)   : one CTA per target block: X_nn = A_nn - C^T C (Eq.
//                          elim), contributions summed in ascending cluster
//                          order; the mixed form's products on the tensor
//                          cores (mma.sync, TF32 x3 split or BF16).
//   k_dense_cholesky / k_tops_cholesky : the dense top(s).
// Solve (Algorithm 2): k_ap_fwd / k_ap_bwd per stage with the explicit
// per-cluster operator W = U^T G^-1, k_ap_fin / k_vcopy between levels,
// k_ap_coarse (single-CTA chain) or k_dense_gemv (explicit coarse operator
// formed by k_ap_coarse_batch), k_tops_solve for batched tops; captured in
// one CUDA graph, each kernel launched with programmatic dependent launch.
// Krylov: CSR SpMV fused with p^T q, the x/r update fused with r^T r, dot
// products in one launch (block partials added in index order by the last
// block), per-problem (segmented) PCG kernels for batched handles.
//
// Decisions that must agree with any other implementation of the method:
// rank = smallest k with sum of squared trailing column norms <= eps^2;
// pivot = lowest unpivoted column index with squared norm >= (1 - 1e-6) *
// the largest; Householder beta = -sign(alpha) * norm, v_k = 1,
// tau = (beta - alpha) / beta.
//
// On this GPU an SM completes about one warp-wide FP64 instruction every 16
// cycles, and conversions between FP64 and FP32 run on the same pipe; the
// kernels keep FP64 instructions full-warp and convert each value once.
#include <atomic>
#include <cfloat>
#include <climits>
#include <cstdint>
#include <mutex>

#include "hs_internal.h"

namespace hs {

namespace {

constexpr double kPivotTie = 1e-6;

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialisation may be scheduled while its predecessor in the stream is still
// running.  griddep_wait() blocks until every predecessor grid has completed
// and its memory writes are visible; griddep_release() lets the successor's
// CTAs be scheduled once every CTA of this grid has issued it or exited.
// Without the launch attribute both are no-ops.  Every kernel launched
// through launch_chained calls griddep_wait() before its first global access,
// so it is ordered after the whole chain before it.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ int warp_min_int(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Block-wide reductions; scratch holds >= 32 doubles.  Every thread returns
// the same value.  Fixed reduction tree => deterministic.
__device__ double block_sum(double v, double* scratch) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) scratch[wid] = v;
    __syncthreads();
    double t = (lane < nw) ? scratch[lane] : 0.0;
    t = warp_sum(t);
    return t;
}
__device__ double block_max(double v, double* scratch) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_max(v);
    __syncthreads();
    if (lane == 0) scratch[wid] = v;
    __syncthreads();
    double t = (lane < nw) ? scratch[lane] : -DBL_MAX;
    return warp_max(t);
}
__device__ int block_min_int(int v, int* scratch) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_min_int(v);
    __syncthreads();
    if (lane == 0) scratch[wid] = v;
    __syncthreads();
    int t = (lane < nw) ? scratch[lane] : INT_MAX;
    return warp_min_int(t);
}

// ---------------------------------------------------------------------------
// Level-0 assembly: scatter CSR entries into the dense blocks.
// ---------------------------------------------------------------------------
__global__ void k_scatter_csr(int64_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                              const double* __restrict__ val, const int32_t* __restrict__ dof_cluster,
                              const int32_t* __restrict__ dof_local, const int32_t* __restrict__ blk_ptr,
                              const int32_t* __restrict__ blk_col, const int64_t* __restrict__ blk_off,
                              const int32_t* __restrict__ blk_ld, double* __restrict__ blocks) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int p = dof_cluster[i], li = dof_local[i];
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; e++) {
        const int j = col[e];
        const int q = dof_cluster[j], lj = dof_local[j];
        int lo = blk_ptr[p], hi = blk_ptr[p + 1] - 1, b = -1;
        while (lo <= hi) {
            const int mid = (lo + hi) >> 1, cm = blk_col[mid];
            if (cm == q) { b = mid; break; }
            if (cm < q) lo = mid + 1; else hi = mid - 1;
        }
        if (b >= 0) blocks[blk_off[b] + (int64_t)li * blk_ld[b] + lj] += val[e];
    }
}

// Validity of a CSR pattern on the device (inputs already in device memory):
// rowptr[0] == 0, non-decreasing row pointers, every column index in [0, n).
// Any violation sets *bad (never cleared here).
__global__ void k_check_csr(int64_t n, int64_t nnz, const int64_t* __restrict__ rowptr,
                            const int32_t* __restrict__ col, int32_t* __restrict__ bad) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int v = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        v |= rowptr[i + 1] < rowptr[i];
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += stride) {
        const int32_t c = col[e];
        v |= (c < 0) | ((int64_t)c >= n);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) v |= rowptr[0] != 0;
    if (__any_sync(0xffffffffu, v) && (threadIdx.x & 31) == 0) atomicOr(bad, 1);
}

// ---------------------------------------------------------------------------
// Factor one phase: one CTA per cluster.
// Shared memory: G (s*s) | rdiag (s) | v (s) | cn (wmax) | red (64) | ioff (lmax+1 ints) | flags
// ---------------------------------------------------------------------------
constexpr int kFactorThreads = 512;

// Block-wide sum and maximum for the factor kernels (scratch holds >= 33
// doubles), with the same reduction tree as block_sum / block_max and so the
// same results, built for GB300's small FP64 rate: a warp whose values are
// all zero skips its shuffle tree (its partial is exactly 0, which a sum or a
// maximum over such partials takes as the tree would), and the second level
// runs on warp 0 alone and is broadcast through scratch[32].  In the
// factorization most warps hold no column at a given step, and every FP64
// add of a tree run by all 32 warps competes for the same pipe.
__device__ double block_sum_sparse(double v, double* scratch) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (__any_sync(0xffffffffu, v != 0.0)) v = warp_sum(v);
    __syncthreads();
    if (lane == 0) scratch[wid] = v;
    __syncthreads();
    if (wid == 0) {
        const double t = warp_sum((lane < nw) ? scratch[lane] : 0.0);
        if (lane == 0) scratch[32] = t;
    }
    __syncthreads();
    return scratch[32];
}
__device__ double block_max_sparse(double v, double* scratch) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (__any_sync(0xffffffffu, v != 0.0)) v = warp_max(v);
    __syncthreads();
    if (lane == 0) scratch[wid] = v;
    __syncthreads();
    if (wid == 0) {
        const double t = warp_max((lane < nw) ? scratch[lane] : -DBL_MAX);
        if (lane == 0) scratch[32] = t;
    }
    __syncthreads();
    return scratch[32];
}

// Thread groups that run one cluster elimination: a whole CTA (fine levels)
// or one warp (coarse levels).  Reductions return the same value to every
// member and use a fixed tree (deterministic).
struct CtaGroup {
    int rank, size;
    __device__ CtaGroup() : rank(threadIdx.x), size(blockDim.x) {}
    __device__ void sync() const { __syncthreads(); }
    __device__ double sum(double v, double* red) const { return block_sum_sparse(v, red); }
    __device__ double max(double v, double* red) const { return block_max_sparse(v, red); }
    __device__ int minint(int v, double* red) const { return block_min_int(v, reinterpret_cast<int*>(red)); }
    __device__ bool any(bool p) const { return __syncthreads_or(p) != 0; }
};
struct WarpGroup {
    int rank, size;
    __device__ WarpGroup() : rank(threadIdx.x & 31), size(32) {}
    __device__ void sync() const { __syncwarp(); }
    __device__ double sum(double v, double*) const { return warp_sum(v); }
    __device__ double max(double v, double*) const { return warp_max(v); }
    __device__ int minint(int v, double*) const { return warp_min_int(v); }
    // a barrier (with memory ordering, as sync) that also votes
    __device__ bool any(bool p) const {
        __syncwarp();
        return __any_sync(0xffffffffu, p) != 0;
    }
};

// Per list entry of a cluster's row: block offsets / leading dimensions of
// (c, q) and (q, c) and q's current width, staged in shared memory so that the
// entries' chains of dependent loads run in parallel.
struct EntryMeta {
    int64_t cq, qc;
    int32_t ldcq, ldqc, w, pad;
};

constexpr int kNB = 16;  // Cholesky panel width

// 1 / sqrt(d) for the Cholesky pivots: the FP32 estimate refined by two
// Newton-Raphson steps y <- y + y (1 - d y^2) / 2 (each squares the relative
// error: 2^-22 -> 2^-44 -> below FP64 rounding); outside the FP32 range the
// FP64 square root and division.
__device__ __forceinline__ double rsqrt_newton(double d) {
    const float f = (float)d;  // the range test in FP32 (no FP64 compare on the chain)
    if (!(f > 1e-30f && f < 1e30f)) return 1.0 / sqrt(d);
    double y = (double)rsqrtf(f);
    double h = fma(-d * y, y, 1.0);
    y = fma(0.5 * y, h, y);
    h = fma(-d * y, y, 1.0);
    return fma(0.5 * y, h, y);
}

// 1 / x for x > 0: the FP32 reciprocal refined by two Newton-Raphson steps
// y <- y + y (1 - x y); outside the FP32 range the FP64 division.
__device__ __forceinline__ double rcp_newton(double x) {
    if (!(x > 1e-30 && x < 1e30)) return 1.0 / x;
    double y = (double)(1.0f / (float)x);
    double h = fma(-x, y, 1.0);
    y = fma(y, h, y);
    h = fma(-x, y, 1.0);
    return fma(y, h, y);
}

// |a| as a float from the bit pattern alone (integer operations only, so the
// FP64 pipe is not used): the exponent rebiased and the top 20 mantissa bits
// kept, a relative error below 2^-20; magnitudes below 2^-126 give 0 and
// magnitudes above 2^63 (with infinities and NaN) give 2^63.  For the rank
// features, where a squared norm to six digits is plenty.
__device__ __forceinline__ float approx_abs_float(double a) {
    const int hi = __double2hiint(a);
    const int e = ((hi >> 20) & 0x7ff) - 1023;
    if (e < -126) return 0.f;
    if (e > 63) return 9.223372e18f;
    return __int_as_float(((e + 127) << 23) | ((hi & 0xfffff) << 3));
}

// |a| as its bit pattern: for non-negative doubles the integer order is the
// numeric order, so maxima of magnitudes need no FP64 instruction.
__device__ __forceinline__ long long abs_bits(double a) {
    return __double_as_longlong(a) & 0x7fffffffffffffffLL;
}

// In-place FP64 -> FP32 conversion of count elements by the group, in chunks
// of kConvBatch elements per member: float i overwrites bytes of double i / 2,
// which an earlier chunk (or this chunk, before the barrier) has already read.
constexpr int kConvBatch = 8;
template <typename Grp>
__device__ __forceinline__ void to_float_inplace(const Grp& g, double* M, int64_t count) {
    float* F = reinterpret_cast<float*>(M);
    const int64_t chunk = (int64_t)g.size * kConvBatch;
    for (int64_t base = 0; base < count; base += chunk) {
        double x[kConvBatch];
#pragma unroll
        for (int u = 0; u < kConvBatch; u++) {
            const int64_t i = base + (int64_t)u * g.size + g.rank;
            x[u] = i < count ? M[i] : 0.0;
        }
        g.sync();
#pragma unroll
        for (int u = 0; u < kConvBatch; u++) {
            const int64_t i = base + (int64_t)u * g.size + g.rank;
            if (i < count) F[i] = (float)x[u];
        }
    }
    g.sync();
}

// Column-pivoted QR of the fill columns of the scaled block row M (s x Wt,
// row-major: n columns, fill columns, identity columns), every reflector
// applied to the whole row; then the rank, W = U^T G^-1, C and the coarse
// write-back.  CT: arithmetic of this step, double, or float in the mixed
// form (the pivot and Householder scalars are formed in FP64 either way).
template <typename CT, typename FT, typename Grp>
__device__ __forceinline__ void compress_task(const TaskDev& T, const Grp& g, CT* M, int Wt, int W, int ncols, CT* v, CT* cn,
                              double* red, double* s_hh, const EntryMeta* em, const int* ioff,
                              double* __restrict__ blocks, const int64_t* __restrict__ blk_off,
                              const int32_t* __restrict__ blk_ld, int32_t* __restrict__ cur, FT* __restrict__ fac,
                              int32_t* __restrict__ meta, double eps2, bool rank0 = false) {
    const int s = T.s, tid = g.rank, NT = g.size;
    const int L = T.nn + T.nw, Wn = W - ncols;
    // column-pivoted QR of the fill columns, reflectors applied to the whole row
    // rank0: the rank is already known to be 0 (no reflector).  A thread's
    // column is read kRowBatch rows at a time, all loads of a batch issued
    // before any is used (the sums keep their row order).
    constexpr int kRowBatch = 8;
    for (int j = tid; j < (rank0 ? 0 : Wn); j += NT) {
        CT c = 0;
        for (int i0 = 0; i0 < s; i0 += kRowBatch) {
            CT a[kRowBatch];
#pragma unroll
            for (int u = 0; u < kRowBatch; u++) a[u] = i0 + u < s ? M[(int64_t)(i0 + u) * Wt + ncols + j] : CT(0);
#pragma unroll
            for (int u = 0; u < kRowBatch; u++)
                if (i0 + u < s) c += a[u] * a[u];
        }
        cn[j] = c;
    }
    g.sync();
    int k = 0;
    while (k < s && !rank0) {
        double lt = 0.0, lm = 0.0;
        for (int j = tid; j < Wn; j += NT) {
            const double c = (double)cn[j];
            if (c >= 0.0) {
                lt += c;
                lm = fmax(lm, c);
            }
        }
        const double total = g.sum(lt, red);
        const double cmax = g.max(lm, red);
        if (total <= eps2) break;
        const double thr = (1.0 - kPivotTie) * cmax;
        int lp = INT_MAX;
        for (int j = tid; j < Wn; j += NT)
            if (cn[j] >= (CT)0 && (double)cn[j] >= thr) {
                lp = j;
                break;  // lowest of this thread's columns
            }
        const int p = g.minint(lp, red);
        const int pc = ncols + p;
        double ls = 0.0;
        for (int i = k + 1 + tid; i < s; i += NT) {
            const double x = (double)M[(int64_t)i * Wt + pc];
            ls += x * x;
        }
        const double sig = g.sum(ls, red);
        if (tid == 0) {
            // beta = -sign(alpha) nrm, tau = (beta - alpha) / beta and
            // 1 / (alpha - beta) from 1 / nrm and 1 / (|alpha| + nrm) by
            // Newton-Raphson (no FP64 square root or division)
            const double alpha = (double)M[(int64_t)k * Wt + pc];
            const double q = fma(alpha, alpha, sig);
            const double rs = rsqrt_newton(q);
            const double nrm = q * rs;
            const double sg = alpha >= 0.0 ? 1.0 : -1.0;
            const double ra = rcp_newton(fabs(alpha) + nrm);
            s_hh[0] = -sg * nrm;                   // beta
            s_hh[1] = (fabs(alpha) + nrm) * rs;    // tau = (beta - alpha) / beta
            s_hh[2] = sg * ra;                     // 1 / (alpha - beta)
            cn[p] = -1.0;
        }
        g.sync();
        const CT beta = (CT)s_hh[0], tau = (CT)s_hh[1], scal = (CT)s_hh[2];
        for (int i = tid; i < s; i += NT) {
            CT vi = 0;
            if (i == k) vi = 1;
            else if (i > k) vi = M[(int64_t)i * Wt + pc] * scal;
            v[i] = vi;
        }
        g.sync();
        for (int i = k + tid; i < s; i += NT) M[(int64_t)i * Wt + pc] = (i == k) ? beta : (CT)0;
        for (int j = tid; j < Wt; j += NT) {
            if (j == pc) continue;
            const bool cand = (j >= ncols && j < W);
            if (cand && cn[j - ncols] < (CT)0) continue;  // pivoted: zero below its row
            // t = v^T M(k:, j) (rows in order), then M(k:, j) -= tau t v with the
            // new trailing squared norm; loads of a batch before its stores
            // (distinct rows of the thread's own column)
            CT t = M[(int64_t)k * Wt + j];
            for (int i0 = k + 1; i0 < s; i0 += kRowBatch) {
                CT a[kRowBatch];
#pragma unroll
                for (int u = 0; u < kRowBatch; u++) a[u] = i0 + u < s ? M[(int64_t)(i0 + u) * Wt + j] : CT(0);
#pragma unroll
                for (int u = 0; u < kRowBatch; u++)
                    if (i0 + u < s) t += v[i0 + u] * a[u];
            }
            t *= tau;
            M[(int64_t)k * Wt + j] -= t;
            CT c = 0;
            for (int i0 = k + 1; i0 < s; i0 += kRowBatch) {
                CT a[kRowBatch];
#pragma unroll
                for (int u = 0; u < kRowBatch; u++) a[u] = i0 + u < s ? M[(int64_t)(i0 + u) * Wt + j] : CT(0);
#pragma unroll
                for (int u = 0; u < kRowBatch; u++) {
                    if (i0 + u >= s) break;
                    const CT x = a[u] - t * v[i0 + u];
                    M[(int64_t)(i0 + u) * Wt + j] = x;
                    if (cand) c += x * x;
                }
            }
            if (cand) cn[j - ncols] = c;
        }
        g.sync();
        k++;
    }
    const int r = k;

    // factor: rank and n-column layout, W = U^T G^-1, C = rows r.. of the n columns
    int32_t* mt = meta + T.meta;
    if (tid == 0) mt[0] = r;
    for (int e = tid; e < T.nn; e += NT) {
        mt[1 + 2 * e] = ioff[e];
        mt[2 + 2 * e] = ioff[e + 1] - ioff[e];
    }
    {
        FT* Wf = fac + T.w_off;
        for (int idx = tid; idx < s * s; idx += NT) Wf[idx] = (FT)M[(int64_t)(idx / s) * Wt + W + idx % s];
        FT* Cf = fac + T.c_off;
        const int f = s - r;
        for (int idx = tid; idx < f * ncols; idx += NT) {
            const int i = idx / ncols, j = idx % ncols;
            Cf[(int64_t)i * T.ncap + j] = (FT)M[(int64_t)(r + i) * Wt + j];
        }
    }
    // write back the coarse row (identity diagonal, U^T G^-1 A_sn, V1^T)
    if (T.nw > 0 && r > 0) {
        for (int e = 0; e < L; e++) {
            const int wq = ioff[e + 1] - ioff[e], o = ioff[e];
            double* dcq = blocks + em[e].cq;
            const int ldcq = em[e].ldcq;
            double* dqc = blocks + em[e].qc;
            const int ldqc = em[e].ldqc;
            for (int idx = tid; idx < r * wq; idx += NT) {
                const int i = idx / wq, j = idx % wq;
                const double x = (double)M[(int64_t)i * Wt + o + j];
                dcq[(int64_t)i * ldcq + j] = x;
                dqc[(int64_t)j * ldqc + i] = x;
            }
        }
        double* dcc = blocks + blk_off[T.diag_blk];
        const int ld = blk_ld[T.diag_blk];
        for (int idx = tid; idx < r * r; idx += NT) {
            const int i = idx / r, j = idx % r;
            dcc[(int64_t)i * ld + j] = (i == j) ? 1.0 : 0.0;
        }
    }
    if (tid == 0) cur[T.c] = (T.nw > 0) ? r : 0;
}

// Rank predictor inside a factor task: y = w3 . relu(W2 relu(W1 xn + b1) + b2)
// + b3 on the standardised features xn = (f - mu) / sd.  model: mu (8), sd
// (8), the network's parameter vector (kMlpParams floats, the layout of the
// training kernels), then W2 transposed (so that neighbouring threads read
// neighbouring floats).  f: the 8 features, standardised in place; h: 64
// floats; part: kPredChunks * 64 floats.  The 64 x 64 layer is split over
// the group in kPredChunks slices of the inner index (each thread's loads
// independent of one another), then summed per output.  Every thread
// returns y.
constexpr int kPredChunks = 8;
template <typename Grp>
__device__ float predict_fraction(const Grp& g, const float* __restrict__ model, float* f, float* h, float* part,
                                  double* red) {
    const float* mu = model;
    const float* sd = model + kMlpIn;
    const float* W1 = model + 2 * kMlpIn;
    const float* b1 = W1 + kMlpHidden * kMlpIn;
    const float* b2 = b1 + kMlpHidden + kMlpHidden * kMlpHidden;
    const float* w3 = b2 + kMlpHidden;
    const float b3 = w3[kMlpHidden];
    const float* W2t = model + kModelFloats;
    if (g.rank < kMlpIn) f[g.rank] = (f[g.rank] - mu[g.rank]) / sd[g.rank];
    g.sync();
    for (int j = g.rank; j < kMlpHidden; j += g.size) {
        float a = b1[j];
#pragma unroll
        for (int i = 0; i < kMlpIn; i++) a += W1[j * kMlpIn + i] * f[i];
        h[j] = a > 0.f ? a : 0.f;
    }
    g.sync();
    constexpr int kSlice = kMlpHidden / kPredChunks;
    for (int t = g.rank; t < kMlpHidden * kPredChunks; t += g.size) {
        const int j = t % kMlpHidden, k0 = (t / kMlpHidden) * kSlice;
        float a = 0.f;
#pragma unroll
        for (int k = 0; k < kSlice; k++) a += W2t[(k0 + k) * kMlpHidden + j] * h[k0 + k];
        part[t] = a;
    }
    g.sync();
    double out = 0.0;
    for (int j = g.rank; j < kMlpHidden; j += g.size) {
        float a = b2[j];
#pragma unroll
        for (int c = 0; c < kPredChunks; c++) a += part[c * kMlpHidden + j];
        out += (double)(w3[j] * (a > 0.f ? a : 0.f));
    }
    return (float)(g.sum(out, red) + (double)b3);
}

// Column j of M <- G^-1 M(:, j) by forward substitution from its first
// nonzero row i0 (zeros above stay zero), FP64.
__device__ __forceinline__ void scale_dense_column(const double* G, const double* rdiag, double* M, int s,
                                                   int Wt, int j, int i0) {
    for (int i = i0; i < s; i++) {
        double acc = M[(int64_t)i * Wt + j];
        for (int k = i0; k < i; k++) acc = fma(-G[i * s + k], M[(int64_t)k * Wt + j], acc);
        M[(int64_t)i * Wt + j] = acc * rdiag[i];
    }
}

// One scaled low-rank elimination (Sec. 3.1) by the group g.  Shared memory
// of the group: G (s*s), rdiag (s), v (s), cn (fill columns), red (>= 64
// doubles), ioff (list length + 1 ints), flag, hh (3 doubles).
// FT: element type of the stored factor (W, C): double, or float in the
// mixed-precision form.  Cholesky and scaling are FP64; the compression runs
// in FP32 in the mixed form (compress_task).
template <typename FT, typename Grp>
__device__ void factor_task(const TaskDev& T, const Grp& g, double* G, double* rdiag, double* v, double* cn,
                            double* red, int* ioff, int* s_flag, double* s_hh, double* Msh, EntryMeta* em,
                            int64_t* colsrc, const ListDev* __restrict__ lists,
                            double* __restrict__ blocks, const int64_t* __restrict__ blk_off,
                            const int32_t* __restrict__ blk_ld, int32_t* __restrict__ cur, FT* __restrict__ fac,
                            int32_t* __restrict__ meta, double* __restrict__ ws, double eps2, int32_t* status,
                            int32_t level, float* fe, const float* __restrict__ model, float* G32, double* Xsh) {
    const int s = T.s, tid = g.rank, NT = g.size;
    const int L = T.nn + T.nw;
    // features for the caller's record, or for the predictor (mixed form,
    // where the speculation has room for its FP32 copy of G)
    const bool use_model = model != nullptr && G32 != nullptr && sizeof(FT) == sizeof(float);
    const bool want_feat = fe != nullptr || use_model;
    // entry metadata (one round of loads for all entries), then the column
    // offsets of the row blocks (compact, current widths)
    for (int e = tid; e < L; e += NT) {
        const ListDev le = lists[T.list + e];
        EntryMeta m;
        m.cq = blk_off[le.blk_cq];
        m.qc = blk_off[le.blk_qc];
        m.ldcq = blk_ld[le.blk_cq];
        m.ldqc = blk_ld[le.blk_qc];
        m.w = cur[le.q];
        m.pad = 0;
        em[e] = m;
    }
    g.sync();
    if (tid == 0) {
        int o = 0;
        for (int e = 0; e < L; e++) {
            ioff[e] = o;
            o += em[e].w;
        }
        ioff[L] = o;
        *s_flag = 0;
    }
    // A_ss -> shared memory
    long long amax_ss_bits = 0;  // largest |A_ss| off the diagonal (features only)
    {
        const double* A = blocks + blk_off[T.diag_blk];
        const int ld = blk_ld[T.diag_blk];
        for (int idx = tid; idx < s * s; idx += NT) {
            const double a = A[(int64_t)(idx / s) * ld + idx % s];
            G[idx] = a;
            if (want_feat && idx / s != idx % s) amax_ss_bits = max(amax_ss_bits, abs_bits(a));
        }
    }
    g.sync();
    const double amax_ss = want_feat ? g.max(__longlong_as_double(amax_ss_bits), red) : 0.0;
    const int W = ioff[L], ncols = ioff[T.nn], Wn = W - ncols;

    // Cholesky A_ss = G G^T and X = G^-1 together, right-looking, one column
    // per step: with r = 1 / g_jj (pivot), column j of G scaled by r gives
    // l (kept contiguous in v); every row i > j then loses l_i l^T over its
    // columns j < c <= i of G and l_i times row j of X (scaled by r) over its
    // columns c <= j of X.  Rows go to warps, columns to lanes; one FMA per
    // element.  The warp that finishes row j + 1 takes the next pivot.  X
    // lives in Xsh (s x s) when the caller has room, else in the identity
    // columns of the block row.
    const int Wt0 = W + s;
    double* M0 = Msh ? Msh : ws + T.m_off;
    double* X = Xsh ? Xsh : M0 + W;
    const int ldx = Xsh ? s : Wt0;
    double* lcol = v;  // s doubles
    for (int idx = tid; idx < s * s; idx += NT) X[(idx / s) * ldx + idx % s] = (idx / s == idx % s) ? 1.0 : 0.0;
    if (tid == 0) {
        const double d = G[0];
        if (!(d > 0.0)) {
            *s_flag = 1;
        } else {
            const double r = rsqrt_newton(d);
            rdiag[0] = r;
            G[0] = d * r;
        }
    }
    g.sync();
    for (int j = 0; j < s; j++) {
        if (*s_flag) {
            if (tid == 0 && atomicCAS(status, 0, ST_NOT_SPD) == 0) {
                status[1] = level;
                status[2] = T.c;
            }
            return;
        }
        const double r = rdiag[j];
        const int m = s - j - 1;
        for (int idx = tid; idx < m + j + 1; idx += NT) {
            if (idx < m) {
                const int i = j + 1 + idx;
                const double l = G[i * s + j] * r;
                G[i * s + j] = l;
                lcol[i] = l;
            } else {
                X[j * ldx + (idx - m)] *= r;
            }
        }
        g.sync();
        // rows below j: X part (columns c <= j) and G part (j < c <= i), each
        // as one flat index space so that every FP64 instruction is full
        const int nx = m * (j + 1), ngt = m * (m + 1) / 2;
        // with a CTA, the first thread of the last warp takes entry 0 of the
        // triangle, (j+1, j+1), and the next pivot at once, while the other
        // warps update the rest; with a warp, lane 0 takes the pivot after
        // its share of the updates
        const bool pw = NT >= 256;
        const int nup = pw ? NT - 32 : NT;
        if (tid < nup) {
            for (int idx = tid; idx < nx; idx += nup) {
                const int t = idx / (j + 1), i = j + 1 + t, c0 = idx - t * (j + 1);
                X[i * ldx + c0] = fma(-lcol[i], X[j * ldx + c0], X[i * ldx + c0]);
            }
            for (int idx = tid + (pw ? 1 : 0); idx < ngt; idx += nup) {
                // entry idx of the packed trailing triangle: row t has t + 1 entries
                int t = (int)((sqrtf(8.f * (float)idx + 1.f) - 1.f) * 0.5f);
                while (t * (t + 1) / 2 > idx) t--;
                while ((t + 1) * (t + 2) / 2 <= idx) t++;
                const int i = j + 1 + t, c0 = j + 1 + idx - t * (t + 1) / 2;
                G[i * s + c0] = fma(-lcol[i], lcol[c0], G[i * s + c0]);
            }
        }
        if (tid == (pw ? nup : 0) && j + 1 < s) {
            const int i = j + 1;
            const double d = pw ? fma(-lcol[i], lcol[i], G[i * s + i]) : G[i * s + i];
            if (!(d > 0.0)) {
                *s_flag = 1;
            } else {
                const double rr = rsqrt_newton(d);
                rdiag[i] = rr;
                G[i * s + i] = d * rr;
            }
        }
        g.sync();
    }
    for (int idx = tid; idx < s * s; idx += NT)
        if (idx % s > idx / s) G[idx] = 0.0;
    g.sync();

    // gather the block row [A_sn | A_sw | I] into the workspace (row-major, ld Wt);
    // the identity columns come out as W = U^T G^-1, the solve-phase operator
    const int Wt = W + s;
    double* M = Msh ? Msh : ws + T.m_off;  // block row in shared memory when the caller has room
    // source of every column (block offset + column, leading dimension) so that
    // the whole block row is gathered by one loop of independent loads
    for (int e = tid; e < L; e += NT)
        for (int j = 0; j < em[e].w; j++) {
            colsrc[2 * (ioff[e] + j)] = em[e].cq + j;
            colsrc[2 * (ioff[e] + j) + 1] = em[e].ldcq;
        }
    float* rdf = reinterpret_cast<float*>(v);  // D^-1 as floats, for the features
    if (want_feat)
        for (int i = tid; i < s; i += NT) rdf[i] = approx_abs_float(rdiag[i]);
    g.sync();
    // pass 1, one thread per column of [A_sn | A_sw]: stream the column from
    // the blocks (loads in groups of kGatherBatch, all in flight before they
    // are used), store it, note its nonzeros.  Scaling M <- G^-1 M: a column
    // with at most kSparseNz nonzeros (level-0 stencil couplings) is the
    // combination sum_k a_k G^-1 e_{i_k} of columns of X = G^-1 and is
    // finished here; a denser one is forward-substituted in pass 2.
    constexpr int kGatherBatch = 8;
    unsigned char* dense = reinterpret_cast<unsigned char*>(cn);  // per column (W bytes)
    // features (integer and FP32 operations only): max |a|, norms of D^-1 A_sw;
    // a sparse column contributes its few nonzeros here, a dense one once the
    // features are known to be wanted (its values stay in the block row
    // until pass 2)
    long long amax_bits = 0;
    float lt = 0.f, lm = 0.f;
    bool dense_fill = false;  // this thread met a dense fill column
    for (int j = tid; j < W; j += NT) {
        const int64_t src = colsrc[2 * j], ldc = colsrc[2 * j + 1];
        const bool fill = j >= ncols;
        int nz = 0, i0 = s;
        int ri[kSparseNz];
        double rv[kSparseNz];
#pragma unroll
        for (int k = 0; k < kSparseNz; k++) { ri[k] = 0; rv[k] = 0.0; }
        for (int b = 0; b < s; b += kGatherBatch) {
            double a[kGatherBatch];
#pragma unroll
            for (int u = 0; u < kGatherBatch; u++) a[u] = (b + u < s) ? blocks[src + (int64_t)(b + u) * ldc] : 0.0;
#pragma unroll
            for (int u = 0; u < kGatherBatch; u++) {
                const int i = b + u;
                if (i >= s) break;
                M[(int64_t)i * Wt + j] = a[u];
                if ((__double_as_longlong(a[u]) << 1) != 0) {  // nonzero (either sign of zero is zero)
                    if (nz == 0) i0 = i;
#pragma unroll
                    for (int k = 0; k < kSparseNz; k++)
                        if (k == nz) { ri[k] = i; rv[k] = a[u]; }
                    nz++;
                }
            }
        }
        const bool sparse = nz <= kSparseNz && 2 * nz <= s - i0;
        dense[j] = sparse ? 0 : (unsigned char)(1 + i0);  // dense: 1 + its first nonzero row
        dense_fill |= fill && !sparse;
        if (want_feat && sparse) {
            float cj = 0.f;
#pragma unroll
            for (int k = 0; k < kSparseNz; k++)
                if (k < nz) {
                    amax_bits = max(amax_bits, abs_bits(rv[k]));
                    const float x = approx_abs_float(rv[k]) * rdf[ri[k]];
                    cj = fmaf(x, x, cj);
                }
            if (fill) {
                lt += cj;
                lm = fmaxf(lm, cj);
            }
        }
        if (sparse)
            for (int r = i0; r < s; r++) {
                double x = 0.0;
#pragma unroll
                for (int k = 0; k < kSparseNz; k++)
                    if (k < nz && ri[k] <= r) x = fma(rv[k], X[r * ldx + ri[k]], x);
                M[(int64_t)r * Wt + j] = x;
            }
    }
    if (Xsh)  // the identity columns become G^-1
        for (int idx = tid; idx < s * s; idx += NT) M[(int64_t)(idx / s) * Wt + W + idx % s] = Xsh[idx];
    // the predictor runs only where dense fill columns leave FP64 work to
    // spare, and where the space of G^-1 holds its scratch (s >= 16)
    const bool predict = use_model && Wn > 0 && s >= 16 ? g.any(dense_fill) : (g.sync(), false);
    // features of the block row (the column table is free from here on):
    // structure, the coupling ratio, and the fill block scaled by the
    // Cholesky diagonal, D^-1 A_sw (D = diag G), known before the scaling
    float* fsh = reinterpret_cast<float*>(colsrc);  // 8 features, then 64 floats of scratch
    if (fe || predict) {
        for (int j = tid; j < W; j += NT) {
            if (!dense[j]) continue;
            float cj = 0.f;
            for (int i = 0; i < s; i++) {
                const double a = M[(int64_t)i * Wt + j];
                amax_bits = max(amax_bits, abs_bits(a));
                const float x = approx_abs_float(a) * rdf[i];
                cj = fmaf(x, x, cj);
            }
            if (j >= ncols) {
                lt += cj;
                lm = fmaxf(lm, cj);
            }
        }
        const double amax_row = g.max(__longlong_as_double(amax_bits), red);
        const double total = g.sum((double)lt, red), cmax = g.max((double)lm, red);
        if (tid == 0) {  // FP32 logarithms (the features are FP32)
            const float le = 0.5f * log10f(eps2 > 0.0 ? (float)eps2 : 1e-38f);  // log10 eps
            const float lr = log10f(fminf(fmaxf((float)amax_ss, 1e-37f), 1e37f)) -
                             log10f(fminf(fmaxf((float)amax_row, 1e-37f), 1e37f));
            fsh[0] = (float)s;
            fsh[1] = (float)ncols;
            fsh[2] = (float)Wn;
            fsh[3] = (float)level;
            fsh[4] = (float)L;
            fsh[5] = Wn > 0 && total > 0.0 ? fmaxf(0.5f * log10f((float)total) - le, -30.f) : -30.f;
            // coupling inside the cluster against coupling to its neighbours
            fsh[6] = fminf(fmaxf(lr, -30.f), 30.f);
            fsh[7] = Wn > 0 && cmax > 0.0 ? fmaxf(0.5f * log10f((float)cmax) - le, -30.f) : -30.f;
        }
        g.sync();
        if (fe && tid < kFeat) fe[tid] = fsh[tid];
    }
    // learned rank-0 speculation (mixed form): when the predictor says rank 0,
    // dense fill columns are scaled in FP32 only, and the rank is 0 if the
    // FP32 result with its forward-error bound proves ||G^-1 A_sw||_F <= eps;
    // otherwise they are gathered again and scaled in FP64 and the
    // column-pivoted QR decides as usual
    bool spec0 = false;
    if (predict) {
        const float y = predict_fraction(g, model, fsh, fsh + kFeat, G32, red);
        spec0 = y * (float)s < 0.5f;
        if (spec0)
            for (int idx = tid; idx < s * s; idx += NT) G32[idx] = (float)G[idx];
        g.sync();
    }
    // pass 2: dense columns by forward substitution from their first nonzero
    // row (zeros above stay zero); speculated fill columns in FP32 (values in
    // the first float of each slot), with the terms of their error bound:
    // the squared norms of the FP32 inputs (lb) and of |G| |x| (lz)
    float lb = 0.f, lz = 0.f;
    // Few dense columns (at most kXCols, CTA groups): every one becomes
    // X a_j, X = G^-1 (lower triangular).  Its rows are independent sums, so
    // a warp takes the row pair (i, s-1-i) -- s + 1 terms for every pair --
    // with its lanes on 32 columns at a time, from the group's first nonzero
    // row on (the terms above are zero), instead of one thread running a
    // column's whole substitution (a chain of up to s^2 / 2 dependent FMAs,
    // which only many columns keep the FP64 pipe busy with).  Row i is
    // sum_k X_ik a_k in ascending k, accumulated by FMA.
    constexpr int kXCols = 96;
    bool xpath = false;
    if (NT >= 256 && s <= 64) {
        int* dj = reinterpret_cast<int*>(colsrc);  // the column table is free from here on
        int* cnt = reinterpret_cast<int*>(red + 48);
        if (tid == 0) *cnt = 0;
        g.sync();
        for (int j = tid; j < W; j += NT)
            if (dense[j] && !(spec0 && j >= ncols)) {
                const int q = atomicAdd(cnt, 1);
                if (q < kXCols) dj[q] = j;
            }
        g.sync();
        const int nd = *cnt;
        xpath = nd <= kXCols;
        if (xpath && nd > 0) {
            // X: G^-1 in shared memory, unless the predictor used that space;
            // else the identity columns of the block row, which hold G^-1 now
            const bool xs = Xsh != nullptr && !predict;
            const double* Xp = xs ? Xsh : M + W;
            const int64_t ldX = xs ? s : Wt;
            const int lane = tid & 31, wid = tid >> 5, nw = NT >> 5, npair = (s + 1) / 2;
            for (int c0 = 0; c0 < nd; c0 += 32) {
                const int j = c0 + lane < nd ? dj[c0 + lane] : -1;
                const int k0 = (int)__reduce_min_sync(0xffffffffu, j >= 0 ? (unsigned)(dense[j] - 1) : 64u);
                double ya[4], yb[4];
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const int ia = wid + u * nw, ib = s - 1 - ia;
                    ya[u] = 0.0;
                    yb[u] = 0.0;
                    if (ia >= npair || j < 0) continue;
                    for (int k = k0; k <= ib; k++) {
                        const double a = M[(int64_t)k * Wt + j];
                        if (k <= ia) ya[u] = fma(Xp[ia * ldX + k], a, ya[u]);
                        yb[u] = fma(Xp[ib * ldX + k], a, yb[u]);
                    }
                }
                g.sync();  // every warp has read the group's columns
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const int ia = wid + u * nw, ib = s - 1 - ia;
                    if (ia >= npair || j < 0) continue;
                    if (ia >= k0) M[(int64_t)ia * Wt + j] = ya[u];
                    if (ib != ia && ib >= k0) M[(int64_t)ib * Wt + j] = yb[u];
                }
            }
        }
    }
    for (int j = tid; j < W; j += NT) {
        if (!dense[j]) continue;
        if (!(spec0 && j >= ncols)) {
            if (!xpath) scale_dense_column(G, rdiag, M, s, Wt, j, dense[j] - 1);
            continue;
        }
        int i0 = 0;
        while (i0 < s && (__double_as_longlong(M[(int64_t)i0 * Wt + j]) << 1) == 0) i0++;
        {
            float* Mf = reinterpret_cast<float*>(M);
            for (int i = i0; i < s; i++) {
                float acc = (float)M[(int64_t)i * Wt + j];
                lb = fmaf(acc, acc, lb);
                float za = 0.f;
                for (int k = i0; k < i; k++) {
                    const float gk = G32[i * s + k], xk = Mf[2 * ((int64_t)k * Wt + j)];
                    acc -= gk * xk;
                    za = fmaf(fabsf(gk), fabsf(xk), za);
                }
                const float xi = acc * (float)rdiag[i];
                Mf[2 * ((int64_t)i * Wt + j)] = xi;
                za = fmaf(fabsf(G32[i * s + i]), fabsf(xi), za);
                lz = fmaf(za, za, lz);
            }
            for (int i = 0; i < i0; i++) Mf[2 * ((int64_t)i * Wt + j)] = 0.f;
        }
    }
    g.sync();
    bool rank0 = false;
    if (spec0) {
        const float* Mf = reinterpret_cast<const float*>(M);
        double ld = 0.0;  // sparse fill columns (FP64 values)
        float lf = 0.f;   // dense fill columns (FP32 values, summed in FP32)
        for (int j = tid; j < Wn; j += NT) {
            if (dense[ncols + j]) {
                for (int i = 0; i < s; i++) {
                    const float x = Mf[2 * ((int64_t)i * Wt + ncols + j)];
                    lf = fmaf(x, x, lf);
                }
            } else {
                for (int i = 0; i < s; i++) {
                    const double x = M[(int64_t)i * Wt + ncols + j];
                    ld = fma(x, x, ld);
                }
            }
        }
        // Certificate that the exact scaled block B = G^-1 A_sw has
        // ||B||_F <= eps (rank 0 by the rank rule): the FP32 result B' of the
        // substitution solves (G + E) B' = fl32(A_sw) with |E| <= gamma |G|,
        // gamma = (s + 2) u / (1 - (s + 2) u), u = 2^-24 (rounding of G and of
        // the reciprocal pivots, s - 1 products and sums), so
        // ||B - B'||_F <= ||G^-1||_2 (u ||A_sw||_F + gamma || |G| |B'| ||_F)
        // (standard forward-error analysis of triangular substitution).
        // ||G^-1||_2 <= ||X||_F for the FP64 inverse X already formed (doubled
        // to cover X's own error; the FP64 Cholesky is meaningless before
        // that bound is).  Sums of squares in FP32 carry at most a 1e-4
        // relative error here.  Rank 0 only if ||B'||_F + bound <= eps.
        double lx = 0.0;
        for (int idx = tid; idx < s * s; idx += NT) {
            const double x = M[(int64_t)(idx / s) * Wt + W + idx % s];
            lx = fma(x, x, lx);
        }
        const double nb = sqrt(g.sum(ld + (double)lf, red)) * (1.0 + 1e-4);
        const double nin = sqrt(g.sum((double)lb, red)), nz = sqrt(g.sum((double)lz, red));
        const double nx = 2.0 * sqrt(g.sum(lx, red));
        const double u = 5.9604644775390625e-8, gam = (s + 2) * u / (1.0 - (s + 2) * u);
        const double bound = nx * (u * nin + gam * nz) * (1.0 + 1e-4);
        rank0 = (nb + bound) * (nb + bound) <= eps2;
        if (!rank0) {
            // fallback: the fill columns again from the blocks, scaled in FP64
            for (int e = T.nn + tid; e < L; e += NT)
                for (int j = 0; j < em[e].w; j++) {
                    colsrc[2 * (ioff[e] + j)] = em[e].cq + j;
                    colsrc[2 * (ioff[e] + j) + 1] = em[e].ldcq;
                }
            g.sync();
            for (int idx = tid; idx < s * Wn; idx += NT) {
                const int i = idx / Wn, j = ncols + idx % Wn;
                M[(int64_t)i * Wt + j] = blocks[colsrc[2 * j] + (int64_t)i * colsrc[2 * j + 1]];
            }
            g.sync();
            for (int j = ncols + tid; j < W; j += NT) {
                int i0 = 0;
                while (i0 < s && M[(int64_t)i0 * Wt + j] == 0.0) i0++;
                for (int i = i0; i < s; i++) {
                    double acc = M[(int64_t)i * Wt + j];
                    for (int k = i0; k < i; k++) acc -= G[i * s + k] * M[(int64_t)k * Wt + j];
                    M[(int64_t)i * Wt + j] = acc * rdiag[i];
                }
            }
            g.sync();
        }
    }

    if (rank0) {
        compress_task<double, FT>(T, g, M, Wt, W, ncols, v, cn, red, s_hh, em, ioff, blocks, blk_off, blk_ld, cur,
                                  fac, meta, eps2, true);
    } else if constexpr (sizeof(FT) == sizeof(float)) {
        // mixed form: the compression runs on an FP32 copy of the scaled row
        to_float_inplace(g, M, (int64_t)s * Wt);
        compress_task<float, FT>(T, g, reinterpret_cast<float*>(M), Wt, W, ncols, reinterpret_cast<float*>(v),
                                 reinterpret_cast<float*>(cn), red, s_hh, em, ioff, blocks, blk_off, blk_ld, cur,
                                 fac, meta, eps2);
    } else {
        compress_task<double, FT>(T, g, M, Wt, W, ncols, v, cn, red, s_hh, em, ioff, blocks, blk_off, blk_ld, cur,
                                  fac, meta, eps2);
    }
}

// ---------------------------------------------------------------------------
// Coarse-level cluster elimination with the block row in registers.  The same
// steps as factor_task + compress_task (Cholesky of A_ss and FP64 scaling of
// [A_sn | A_sw | I] by G^-1, column-pivoted QR of the fill columns at eps with
// every reflector applied to the whole row, the factor and the coarse write-
// back), for clusters of at most S DOFs whose row has at most 32 K columns:
// lane l owns the block-row columns l, l + 32, ..., so the scaling, each
// reflector and the trailing column norms run without a barrier, and only the
// Cholesky steps, the pivot search and the pivot column's broadcast involve
// the whole warp.  At coarse levels (a few DOFs per cluster, a few phases'
// worth of clusters at a time) the elimination time is this chain of
// dependent steps, not arithmetic.
// ---------------------------------------------------------------------------
template <typename CT, typename FT, int S, int K>
__device__ __forceinline__ void small_compress(const TaskDev& T, CT (&y)[K][S], const int* ecol, int s, int W,
                                               int Wt, int ncols, const EntryMeta* em, const int* ioff,
                                               double* __restrict__ blocks, const int64_t* __restrict__ blk_off,
                                               const int32_t* __restrict__ blk_ld, int32_t* __restrict__ cur,
                                               FT* __restrict__ fac, int32_t* __restrict__ meta, double eps2) {
    const int lane = threadIdx.x & 31;
    CT cn[K];
    bool cand[K];
#pragma unroll
    for (int m = 0; m < K; m++) {
        const int j = lane + 32 * m;
        cand[m] = j >= ncols && j < W;
        CT c = CT(0);
#pragma unroll
        for (int i = 0; i < S; i++)
            if (i < s) c += y[m][i] * y[m][i];
        cn[m] = cand[m] ? c : CT(-1);
    }
    // decisions and Householder scalars in the arithmetic of the step (FP32 in
    // the mixed form, whose compression is FP32 throughout)
    int k = 0;
    while (k < s) {
        CT lt = CT(0), lm = CT(0);
#pragma unroll
        for (int m = 0; m < K; m++)
            if (cn[m] >= CT(0)) {
                lt += cn[m];
                lm = cn[m] > lm ? cn[m] : lm;
            }
        const CT total = warp_sum(lt), cmax = warp_max(lm);
        if (!((double)total > eps2)) break;
        const CT thr = (CT(1) - CT(kPivotTie)) * cmax;
        int lp = INT_MAX;
#pragma unroll
        for (int m = K - 1; m >= 0; m--)
            if (cn[m] >= CT(0) && cn[m] >= thr) lp = lane + 32 * m;  // this lane's lowest column
        const int p = (int)__reduce_min_sync(0xffffffffu, (unsigned)lp);
        if (p >= Wt) break;  // no admissible pivot (non-finite norms)
        // the pivot column, from the lane that owns it
        const int owner = p & 31, slot = p >> 5;
        CT pv[S];
#pragma unroll
        for (int i = 0; i < S; i++) {
            CT val = CT(0);
#pragma unroll
            for (int m = 0; m < K; m++)
                if (m == slot) val = y[m][i];
            pv[i] = __shfl_sync(0xffffffffu, val, owner);
        }
        // Householder scalars, on every lane: beta = -sign(alpha) ||x||,
        // tau = (beta - alpha) / beta, v = x / (alpha - beta) with v_k = 1
        CT sig = CT(0), alpha = CT(0);
#pragma unroll
        for (int i = 0; i < S; i++) {
            if (i == k) alpha = pv[i];
            if (i > k && i < s) sig += pv[i] * pv[i];
        }
        CT beta, tau, scal;
        if constexpr (sizeof(CT) == sizeof(float)) {
            const float q = fmaf(alpha, alpha, sig);
            const float rs = rsqrtf(q);
            const float nrm = q * rs;
            const float sg = alpha >= 0.f ? 1.f : -1.f;
            beta = -sg * nrm;
            tau = (fabsf(alpha) + nrm) * rs;
            scal = sg / (fabsf(alpha) + nrm);
        } else {
            const double q = fma(alpha, alpha, sig);
            const double rs = rsqrt_newton(q);
            const double nrm = q * rs;
            const double sg = alpha >= 0.0 ? 1.0 : -1.0;
            const double ra = rcp_newton(fabs(alpha) + nrm);
            beta = -sg * nrm;
            tau = (fabs(alpha) + nrm) * rs;
            scal = sg * ra;
        }
        CT v[S];
#pragma unroll
        for (int i = 0; i < S; i++) v[i] = (i == k) ? CT(1) : ((i > k && i < s) ? pv[i] * scal : CT(0));
        // the reflector on every owned column (pivoted fill columns are zero
        // from row k down and are skipped); new trailing norms of the fill columns
#pragma unroll
        for (int m = 0; m < K; m++) {
            if (32 * m >= Wt) continue;  // no lane owns a column here
            const int j = lane + 32 * m;
            if (j == p) {
#pragma unroll
                for (int i = 0; i < S; i++) {
                    if (i == k) y[m][i] = beta;
                    else if (i > k) y[m][i] = CT(0);
                }
                cn[m] = CT(-1);
            } else if (j < Wt && !(cand[m] && cn[m] < CT(0))) {
                CT t = CT(0);
#pragma unroll
                for (int i = 0; i < S; i++)
                    if (i == k) t = y[m][i];
#pragma unroll
                for (int i = 0; i < S; i++)
                    if (i > k && i < s) t += v[i] * y[m][i];
                t *= tau;
                CT c = CT(0);
#pragma unroll
                for (int i = 0; i < S; i++) {
                    if (i == k) {
                        y[m][i] -= t;
                    } else if (i > k && i < s) {
                        const CT xx = y[m][i] - t * v[i];
                        y[m][i] = xx;
                        c += xx * xx;
                    }
                }
                if (cand[m]) cn[m] = c;
            }
        }
        k++;
    }
    const int r = k;
    // factor: rank and n-column layout, W = U^T G^-1, C = rows r.. of the n
    // columns; the coarse row (identity diagonal, U^T G^-1 A_sn, V1^T) back
    // into the blocks
    int32_t* mt = meta + T.meta;
    if (lane == 0) mt[0] = r;
    for (int e = lane; e < T.nn; e += 32) {
        mt[1 + 2 * e] = ioff[e];
        mt[2 + 2 * e] = ioff[e + 1] - ioff[e];
    }
    FT* Wf = fac + T.w_off;
    FT* Cf = fac + T.c_off;
    const bool wb = T.nw > 0 && r > 0;
#pragma unroll
    for (int m = 0; m < K; m++) {
        const int j = lane + 32 * m;
        if (j >= W && j < Wt) {
#pragma unroll
            for (int i = 0; i < S; i++)
                if (i < s) Wf[i * s + (j - W)] = (FT)y[m][i];
        } else if (j < ncols) {
#pragma unroll
            for (int i = 0; i < S; i++)
                if (i >= r && i < s) Cf[(int64_t)(i - r) * T.ncap + j] = (FT)y[m][i];
        }
        if (wb && j < W) {
            const EntryMeta& me = em[ecol[m]];
            const int jj = j - ioff[ecol[m]];
#pragma unroll
            for (int i = 0; i < S; i++)
                if (i < r) {
                    const double xx = (double)y[m][i];
                    blocks[me.cq + (int64_t)i * me.ldcq + jj] = xx;
                    blocks[me.qc + (int64_t)jj * me.ldqc + i] = xx;
                }
        }
    }
    if (wb) {
        double* dcc = blocks + blk_off[T.diag_blk];
        const int ld = blk_ld[T.diag_blk];
        for (int idx = lane; idx < r * r; idx += 32) dcc[(int64_t)(idx / r) * ld + idx % r] = (idx / r == idx % r) ? 1.0 : 0.0;
    }
    if (lane == 0) cur[T.c] = (T.nw > 0) ? r : 0;
}

// The body for one (S, K): A_ss, the owned columns of [A_sn | A_sw | I] (all
// loads in flight together), the Cholesky of A_ss in shared memory (one warp
// step per pivot, the trailing update over the packed triangle's pairs), then
// forward substitution of every owned column in FP64.  Returns after recording
// ST_NOT_SPD when a pivot is not positive.
template <typename FT, int S, int K>
__device__ void small_task(const TaskDev& T, int W, int ncols, double* G, double* rdiag, const int* ioff,
                           const EntryMeta* em, double* __restrict__ blocks, const int64_t* __restrict__ blk_off,
                           const int32_t* __restrict__ blk_ld, int32_t* __restrict__ cur, FT* __restrict__ fac,
                           int32_t* __restrict__ meta, double eps2, int32_t* status, int32_t level) {
    const int lane = threadIdx.x & 31;
    const int s = T.s, L = T.nn + T.nw, Wt = W + s;
    {
        const double* A = blocks + blk_off[T.diag_blk];
        const int ld = blk_ld[T.diag_blk];
        for (int idx = lane; idx < s * s; idx += 32) G[idx] = A[(int64_t)(idx / s) * ld + idx % s];
    }
    double x[K][S];
    int ecol[K];
#pragma unroll
    for (int m = 0; m < K; m++) {
        const int j = lane + 32 * m;
        ecol[m] = -1;
        if (j < W) {  // the entry holding column j: the last e with ioff[e] <= j
            int lo = 0, hi = L - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (ioff[mid] <= j) lo = mid;
                else hi = mid - 1;
            }
            ecol[m] = lo;
        }
    }
#pragma unroll
    for (int m = 0; m < K; m++) {
        const int j = lane + 32 * m;
        if (ecol[m] >= 0) {
            const EntryMeta& me = em[ecol[m]];
            const double* src = blocks + me.cq + (j - ioff[ecol[m]]);
#pragma unroll
            for (int i = 0; i < S; i++) x[m][i] = i < s ? src[(int64_t)i * me.ldcq] : 0.0;
        } else {
#pragma unroll
            for (int i = 0; i < S; i++) x[m][i] = (j < Wt && j - W == i) ? 1.0 : 0.0;  // identity columns
        }
    }
    __syncwarp();
    // Cholesky A_ss = G G^T (G strictly below the diagonal scaled, the
    // reciprocal pivots in rdiag)
    for (int j = 0; j < s; j++) {
        const double d = G[j * s + j];
        if (!(d > 0.0)) {
            if (lane == 0 && atomicCAS(status, 0, ST_NOT_SPD) == 0) {
                status[1] = level;
                status[2] = T.c;
            }
            return;
        }
        const double rj = rsqrt_newton(d);
        const int mrow = s - j - 1, npair = mrow * (mrow + 1) / 2;
        double li = 0.0, lc = 0.0, gic = 0.0;
        int pi = 0, pc = 0;
        if (lane < npair) {
            int t = 0;
            while ((t + 1) * (t + 2) / 2 <= lane) t++;
            pi = j + 1 + t;
            pc = j + 1 + lane - t * (t + 1) / 2;
            li = G[pi * s + j] * rj;
            lc = G[pc * s + j] * rj;
            gic = G[pi * s + pc];
        }
        const double lj = lane < mrow ? G[(j + 1 + lane) * s + j] * rj : 0.0;
        __syncwarp();
        if (lane < npair) G[pi * s + pc] = fma(-li, lc, gic);
        if (lane < mrow) G[(j + 1 + lane) * s + j] = lj;
        if (lane == 0) rdiag[j] = rj;
        __syncwarp();
    }
    // scaling G^-1 [A_sn | A_sw | I] (FP64), every owned column by forward substitution
#pragma unroll
    for (int i = 0; i < S; i++) {
        if (i < s) {
            const double ri = rdiag[i];
#pragma unroll
            for (int m = 0; m < K; m++) {
                if (32 * m >= Wt) continue;
                double acc = x[m][i];
#pragma unroll
                for (int k = 0; k < i; k++) acc = fma(-G[i * s + k], x[m][k], acc);
                x[m][i] = acc * ri;
            }
        }
    }
    if constexpr (sizeof(FT) == sizeof(float)) {
        // mixed form: the compression runs in FP32
        float y[K][S];
#pragma unroll
        for (int m = 0; m < K; m++)
#pragma unroll
            for (int i = 0; i < S; i++) y[m][i] = (32 * m < Wt && i < s) ? (float)x[m][i] : 0.f;
        small_compress<float, FT, S, K>(T, y, ecol, s, W, Wt, ncols, em, ioff, blocks, blk_off, blk_ld, cur, fac,
                                        meta, eps2);
    } else {
        small_compress<double, FT, S, K>(T, x, ecol, s, W, Wt, ncols, em, ioff, blocks, blk_off, blk_ld, cur, fac,
                                         meta, eps2);
    }
}

// Entry metadata and column offsets of a task's row (as in factor_task, the
// offsets by a warp scan), then the register path when the row fits one of
// its shapes.  Returns false, having written nothing but its shared scratch,
// when the cluster has more than 8 DOFs or its row more columns than the
// shapes hold; the caller then runs factor_task.
template <typename FT>
__device__ bool small_factor_task(const TaskDev& T, double* G, double* rdiag, int* ioff, EntryMeta* em,
                                  const ListDev* __restrict__ lists, double* __restrict__ blocks,
                                  const int64_t* __restrict__ blk_off, const int32_t* __restrict__ blk_ld,
                                  int32_t* __restrict__ cur, FT* __restrict__ fac, int32_t* __restrict__ meta,
                                  double eps2, int32_t* status, int32_t level) {
    const int lane = threadIdx.x & 31;
    const int s = T.s, L = T.nn + T.nw;
    if (s > 8) return false;
    for (int e = lane; e < L; e += 32) {
        const ListDev le = lists[T.list + e];
        EntryMeta m;
        m.cq = blk_off[le.blk_cq];
        m.qc = blk_off[le.blk_qc];
        m.ldcq = blk_ld[le.blk_cq];
        m.ldqc = blk_ld[le.blk_qc];
        m.w = cur[le.q];
        m.pad = 0;
        em[e] = m;
    }
    __syncwarp();
    // exclusive prefix of the widths: contiguous chunks of entries per lane
    const int ch = (L + 31) / 32;
    int loc = 0;
    for (int u = 0; u < ch; u++) {
        const int e = lane * ch + u;
        if (e < L) loc += em[e].w;
    }
    int inc = loc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    int base = inc - loc;
    for (int u = 0; u < ch; u++) {
        const int e = lane * ch + u;
        if (e < L) {
            ioff[e] = base;
            base += em[e].w;
        }
    }
    const int W = __shfl_sync(0xffffffffu, inc, 31);
    if (lane == 0) ioff[L] = W;
    __syncwarp();
    const int ncols = ioff[T.nn];
    const int Wt = W + s;
    if (s <= 4 && Wt <= 256) {
        small_task<FT, 4, 8>(T, W, ncols, G, rdiag, ioff, em, blocks, blk_off, blk_ld, cur, fac, meta, eps2, status,
                             level);
        return true;
    }
    if (Wt <= 128) {
        small_task<FT, 8, 4>(T, W, ncols, G, rdiag, ioff, em, blocks, blk_off, blk_ld, cur, fac, meta, eps2, status,
                             level);
        return true;
    }
    return false;
}

// NT threads per CTA: 512 (two CTAs per SM) when a phase fills the GPU,
// 1024 (one per SM, twice the threads per cluster) when it has no more
// clusters than SMs
template <typename FT, int NT>
__global__ void __launch_bounds__(NT, 1024 / NT)
k_factor_phase(const TaskDev* __restrict__ tasks, int t0, const ListDev* __restrict__ lists,
               double* __restrict__ blocks, const int64_t* __restrict__ blk_off,
               const int32_t* __restrict__ blk_ld, int32_t* __restrict__ cur, FT* __restrict__ fac,
               int32_t* __restrict__ meta, double* __restrict__ ws, double eps2, int32_t* status,
               int32_t level, int smax, int wmax, int lmax, float* __restrict__ feat,
               const float* __restrict__ model, int use_x) {
    extern __shared__ double sm[];
    __shared__ int s_flag;
    __shared__ double s_hh[3];
    const TaskDev T = tasks[t0 + blockIdx.x];
    double* G = sm;
    double* rdiag = G + (size_t)smax * smax;
    double* v = rdiag + smax;
    double* cn = v + smax;
    double* red = cn + wmax;
    EntryMeta* em = reinterpret_cast<EntryMeta*>(red + 64);
    int64_t* colsrc = reinterpret_cast<int64_t*>(em + lmax);
    int* ioff = reinterpret_cast<int*>(colsrc + 2 * (size_t)wmax);
    // G^-1 (smax x smax doubles) when it fits; the FP32 copy of G for the
    // learned rank-0 speculation (only with a model) reuses that space, free
    // once pass 1 has moved G^-1 into the block row; without it, no
    // speculation (so a model never costs occupancy)
    double* x0 = reinterpret_cast<double*>((reinterpret_cast<uintptr_t>(ioff + lmax + 2) + 15) & ~uintptr_t(15));
    double* Xsh = use_x ? x0 : nullptr;
    float* G32 = model && use_x ? reinterpret_cast<float*>(x0) : nullptr;
    CtaGroup g;
    factor_task<FT>(T, g, G, rdiag, v, cn, red, ioff, &s_flag, s_hh, nullptr, em, colsrc, lists, blocks, blk_off,
                    blk_ld, cur, fac, meta, ws, eps2, status, level,
                    feat ? feat + (size_t)(t0 + blockIdx.x) * kFeat : nullptr, model, G32, Xsh);
}

// ---------------------------------------------------------------------------
// Schur update of one phase: one CTA per target block (p, q), p <= q.
// A(p,q) -= sum over contributions (ascending cluster order) of
// C_t(:, p)^T C_t(:, q), products and their sum in FT (FP64, or FP32 in the
// mixed form), subtracted from the FP64 block; the transpose goes to (q, p).
// 64 x 64 output tiles, 16 x 16 threads with 4 x 4 outputs each, C staged in
// shared memory KC rows at a time.
// ---------------------------------------------------------------------------
constexpr int kSchurTile = 64, kSchurKC = 16;

template <typename FT>
__global__ void __launch_bounds__(256)
k_schur_phase(const TargetDev* __restrict__ targets, int g0, const ContribDev* __restrict__ contribs,
              const TaskDev* __restrict__ tasks, const FT* __restrict__ fac,
              const int32_t* __restrict__ meta, double* __restrict__ blocks,
              const int64_t* __restrict__ blk_off, const int32_t* __restrict__ blk_ld,
              const int32_t* __restrict__ cur) {
    __shared__ FT sp[kSchurKC][kSchurTile];
    __shared__ FT sq[kSchurKC][kSchurTile];
    const TargetDev g = targets[g0 + blockIdx.x];
    const int mp = cur[g.p], mq = cur[g.q];
    double* A = blocks + blk_off[g.blk_pq];
    const int lda = blk_ld[g.blk_pq];
    double* At = blocks + blk_off[g.blk_qp];
    const int ldt = blk_ld[g.blk_qp];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    for (int ti = 0; ti < mp; ti += kSchurTile)
        for (int tj = 0; tj < mq; tj += kSchurTile) {
            FT acc[4][4];
#pragma unroll
            for (int a = 0; a < 4; a++)
#pragma unroll
                for (int b = 0; b < 4; b++) acc[a][b] = FT(0);
            for (int c = g.c_begin; c < g.c_end; c++) {
                const ContribDev cb = contribs[c];
                const TaskDev T = tasks[cb.task];
                const int32_t* mt = meta + T.meta;
                const int f = T.s - mt[0];
                const int op = mt[1 + 2 * cb.kp] + ti, oq = mt[1 + 2 * cb.kq] + tj;
                const FT* C = fac + T.c_off;
                for (int k0 = 0; k0 < f; k0 += kSchurKC) {
                    __syncthreads();
                    for (int idx = tid; idx < kSchurKC * kSchurTile; idx += 256) {
                        const int kk = idx / kSchurTile, jj = idx % kSchurTile;
                        const bool kin = k0 + kk < f;
                        sp[kk][jj] = (kin && ti + jj < mp) ? C[(int64_t)(k0 + kk) * T.ncap + op + jj] : FT(0);
                        sq[kk][jj] = (kin && tj + jj < mq) ? C[(int64_t)(k0 + kk) * T.ncap + oq + jj] : FT(0);
                    }
                    __syncthreads();
#pragma unroll
                    for (int kk = 0; kk < kSchurKC; kk++) {
                        FT a[4], b[4];
#pragma unroll
                        for (int u = 0; u < 4; u++) {
                            a[u] = sp[kk][ty * 4 + u];
                            b[u] = sq[kk][tx * 4 + u];
                        }
#pragma unroll
                        for (int u = 0; u < 4; u++)
#pragma unroll
                            for (int v = 0; v < 4; v++) acc[u][v] += a[u] * b[v];
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < 4; u++)
#pragma unroll
                for (int v = 0; v < 4; v++) {
                    const int i = ti + ty * 4 + u, j = tj + tx * 4 + v;
                    if (i < mp && j < mq) {
                        const double x = A[(int64_t)i * lda + j] - (double)acc[u][v];
                        A[(int64_t)i * lda + j] = x;
                        if (g.p != g.q) At[(int64_t)j * ldt + i] = x;
                    }
                }
        }
}

// ---------------------------------------------------------------------------
// The same Schur update on the tensor cores (mixed form, FP32 factor): the
// products C_t(:, p)^T C_t(:, q) as warp-level TF32 matrix multiply-adds
// (mma.sync m16n8k8) with FP32 accumulation.  passes = 1: each FP32 entry
// rounded to TF32 (10-bit mantissa); passes = 3: each entry split as
// hi + lo (both TF32) and the product formed as hi*hi + hi*lo + lo*hi
// (about 22 significant bits per entry, lo*lo dropped: about 2^-21 relative
// error per product, against 2^-24 for FP32 and 2^-11 for one TF32 pass).  One CTA (8 warps) per target block, 64 x 64
// output tiles, warp w computing rows 16 (w & 3) .. + 16 and columns
// 32 (w >> 2) .. + 32 as four 16 x 8 tiles; C staged k-major in shared memory
// (ld 72: the fragment loads of a warp hit 32 distinct banks).
// ---------------------------------------------------------------------------
constexpr int kTcKC = 32, kTcLd = 72;

__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t u;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x));
    return u;
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

template <int PASSES>
__global__ void __launch_bounds__(256)
k_schur_phase_tc(const TargetDev* __restrict__ targets, int g0, const ContribDev* __restrict__ contribs,
                 const TaskDev* __restrict__ tasks, const float* __restrict__ fac,
                 const int32_t* __restrict__ meta, double* __restrict__ blocks,
                 const int64_t* __restrict__ blk_off, const int32_t* __restrict__ blk_ld,
                 const int32_t* __restrict__ cur) {
    constexpr int NS = PASSES == 1 ? 1 : 2;  // hi (and lo) parts
    __shared__ uint32_t sp[NS][kTcKC][kTcLd];
    __shared__ uint32_t sq[NS][kTcKC][kTcLd];
    const TargetDev g = targets[g0 + blockIdx.x];
    const int mp = cur[g.p], mq = cur[g.q];
    double* A = blocks + blk_off[g.blk_pq];
    const int lda = blk_ld[g.blk_pq];
    double* At = blocks + blk_off[g.blk_qp];
    const int ldt = blk_ld[g.blk_qp];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int gi = lane >> 2, tg = lane & 3;       // fragment row group / thread in group
    const int wi = 16 * (warp & 3), wj = 32 * (warp >> 2);
    for (int ti = 0; ti < mp; ti += kSchurTile)
        for (int tj = 0; tj < mq; tj += kSchurTile) {
            float acc[4][4];
#pragma unroll
            for (int n = 0; n < 4; n++)
#pragma unroll
                for (int r = 0; r < 4; r++) acc[n][r] = 0.f;
            for (int c = g.c_begin; c < g.c_end; c++) {
                const ContribDev cb = contribs[c];
                const TaskDev T = tasks[cb.task];
                const int32_t* mt = meta + T.meta;
                const int f = T.s - mt[0];
                const int op = mt[1 + 2 * cb.kp] + ti, oq = mt[1 + 2 * cb.kq] + tj;
                const float* C = fac + T.c_off;
                for (int k0 = 0; k0 < f; k0 += kTcKC) {
                    __syncthreads();
                    for (int idx = tid; idx < kTcKC * kSchurTile; idx += 256) {
                        const int kk = idx / kSchurTile, jj = idx % kSchurTile;
                        const bool kin = k0 + kk < f;
                        const float xp = (kin && ti + jj < mp) ? C[(int64_t)(k0 + kk) * T.ncap + op + jj] : 0.f;
                        const float xq = (kin && tj + jj < mq) ? C[(int64_t)(k0 + kk) * T.ncap + oq + jj] : 0.f;
                        const uint32_t hp = to_tf32(xp), hq = to_tf32(xq);
                        sp[0][kk][jj] = hp;
                        sq[0][kk][jj] = hq;
                        if (NS == 2) {
                            sp[NS - 1][kk][jj] = to_tf32(xp - __uint_as_float(hp));
                            sq[NS - 1][kk][jj] = to_tf32(xq - __uint_as_float(hq));
                        }
                    }
                    __syncthreads();
                    const int kmax = min(kTcKC, f - k0);
                    for (int k8 = 0; k8 < kmax; k8 += 8) {
                        // A (16 x 8, row-major) = C_p^T: A[i][k] = sp[k][i]
                        uint32_t a[NS][4];
#pragma unroll
                        for (int h = 0; h < NS; h++) {
                            a[h][0] = sp[h][k8 + tg][wi + gi];
                            a[h][1] = sp[h][k8 + tg][wi + gi + 8];
                            a[h][2] = sp[h][k8 + tg + 4][wi + gi];
                            a[h][3] = sp[h][k8 + tg + 4][wi + gi + 8];
                        }
#pragma unroll
                        for (int n = 0; n < 4; n++) {
                            // B (8 x 8, column-major) = C_q: B[k][j] = sq[k][j]
                            uint32_t b[NS][2];
#pragma unroll
                            for (int h = 0; h < NS; h++) {
                                b[h][0] = sq[h][k8 + tg][wj + 8 * n + gi];
                                b[h][1] = sq[h][k8 + tg + 4][wj + 8 * n + gi];
                            }
                            if (PASSES == 3) {
                                mma_tf32(acc[n], a[NS - 1], b[0]);  // lo * hi
                                mma_tf32(acc[n], a[0], b[NS - 1]);  // hi * lo
                            }
                            mma_tf32(acc[n], a[0], b[0]);  // hi * hi
                        }
                    }
                }
            }
            // D fragment: (gi, 2 tg + {0,1}) and (gi + 8, 2 tg + {0,1}) of each 16 x 8 tile
#pragma unroll
            for (int n = 0; n < 4; n++)
#pragma unroll
                for (int r = 0; r < 4; r++) {
                    const int i = ti + wi + gi + 8 * (r >> 1), j = tj + wj + 8 * n + 2 * tg + (r & 1);
                    if (i < mp && j < mq) {
                        const double x = A[(int64_t)i * lda + j] - (double)acc[n][r];
                        A[(int64_t)i * lda + j] = x;
                        if (g.p != g.q) At[(int64_t)j * ldt + i] = x;
                    }
                }
        }
}

// The same update with BF16 products (mma.sync m16n8k16, 8-bit mantissas,
// about 2^-8 relative error per product) and FP32 accumulation: C staged as
// FP32 k-major, pairs of consecutive k packed into bf16x2 fragment registers.
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    uint32_t u;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(u) : "f"(hi), "f"(lo));
    return u;
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__global__ void __launch_bounds__(256)
k_schur_phase_bf16(const TargetDev* __restrict__ targets, int g0, const ContribDev* __restrict__ contribs,
                   const TaskDev* __restrict__ tasks, const float* __restrict__ fac,
                   const int32_t* __restrict__ meta, double* __restrict__ blocks,
                   const int64_t* __restrict__ blk_off, const int32_t* __restrict__ blk_ld,
                   const int32_t* __restrict__ cur) {
    __shared__ float sp[kTcKC][kTcLd];
    __shared__ float sq[kTcKC][kTcLd];
    const TargetDev g = targets[g0 + blockIdx.x];
    const int mp = cur[g.p], mq = cur[g.q];
    double* A = blocks + blk_off[g.blk_pq];
    const int lda = blk_ld[g.blk_pq];
    double* At = blocks + blk_off[g.blk_qp];
    const int ldt = blk_ld[g.blk_qp];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int gi = lane >> 2, tg = lane & 3;
    const int wi = 16 * (warp & 3), wj = 32 * (warp >> 2);
    for (int ti = 0; ti < mp; ti += kSchurTile)
        for (int tj = 0; tj < mq; tj += kSchurTile) {
            float acc[4][4];
#pragma unroll
            for (int n = 0; n < 4; n++)
#pragma unroll
                for (int r = 0; r < 4; r++) acc[n][r] = 0.f;
            for (int c = g.c_begin; c < g.c_end; c++) {
                const ContribDev cb = contribs[c];
                const TaskDev T = tasks[cb.task];
                const int32_t* mt = meta + T.meta;
                const int f = T.s - mt[0];
                const int op = mt[1 + 2 * cb.kp] + ti, oq = mt[1 + 2 * cb.kq] + tj;
                const float* C = fac + T.c_off;
                for (int k0 = 0; k0 < f; k0 += kTcKC) {
                    __syncthreads();
                    for (int idx = tid; idx < kTcKC * kSchurTile; idx += 256) {
                        const int kk = idx / kSchurTile, jj = idx % kSchurTile;
                        const bool kin = k0 + kk < f;
                        sp[kk][jj] = (kin && ti + jj < mp) ? C[(int64_t)(k0 + kk) * T.ncap + op + jj] : 0.f;
                        sq[kk][jj] = (kin && tj + jj < mq) ? C[(int64_t)(k0 + kk) * T.ncap + oq + jj] : 0.f;
                    }
                    __syncthreads();
                    const int kmax = min(kTcKC, f - k0);
                    for (int k16 = 0; k16 < kmax; k16 += 16) {
                        // A (16 x 16, row-major) = C_p^T: register r holds
                        // A[row][col], A[row][col + 1] (low half first)
                        uint32_t a[4];
                        a[0] = pack_bf16(sp[k16 + 2 * tg][wi + gi], sp[k16 + 2 * tg + 1][wi + gi]);
                        a[1] = pack_bf16(sp[k16 + 2 * tg][wi + gi + 8], sp[k16 + 2 * tg + 1][wi + gi + 8]);
                        a[2] = pack_bf16(sp[k16 + 2 * tg + 8][wi + gi], sp[k16 + 2 * tg + 9][wi + gi]);
                        a[3] = pack_bf16(sp[k16 + 2 * tg + 8][wi + gi + 8], sp[k16 + 2 * tg + 9][wi + gi + 8]);
#pragma unroll
                        for (int n = 0; n < 4; n++) {
                            // B (16 x 8, column-major) = C_q: B[k][j], k pairs per register
                            const int j = wj + 8 * n + gi;
                            uint32_t b[2];
                            b[0] = pack_bf16(sq[k16 + 2 * tg][j], sq[k16 + 2 * tg + 1][j]);
                            b[1] = pack_bf16(sq[k16 + 2 * tg + 8][j], sq[k16 + 2 * tg + 9][j]);
                            mma_bf16(acc[n], a, b);
                        }
                    }
                }
            }
#pragma unroll
            for (int n = 0; n < 4; n++)
#pragma unroll
                for (int r = 0; r < 4; r++) {
                    const int i = ti + wi + gi + 8 * (r >> 1), j = tj + wj + 8 * n + 2 * tg + (r & 1);
                    if (i < mp && j < mq) {
                        const double x = A[(int64_t)i * lda + j] - (double)acc[n][r];
                        A[(int64_t)i * lda + j] = x;
                        if (g.p != g.q) At[(int64_t)j * ldt + i] = x;
                    }
                }
        }
}

// ---------------------------------------------------------------------------
// Coarse levels (clusters of at most 32 DOFs): every phase of the level in one
// launch, one warp per cluster elimination and one warp per Schur target,
// __syncthreads() between them.
// ---------------------------------------------------------------------------
// Per-warp shared memory of the fused kernel (doubles): G (smax^2), rdiag and v
// (smax each), cn (wmax), red (64), hh (4), block row (mcap); then ints: ioff
// (lmax + 1) and a flag.
__host__ __device__ inline int64_t fused_warp_doubles(int smax, int wmax, int lmax, int64_t mcap) {
    return (int64_t)smax * smax + 2 * smax + 3 * (int64_t)wmax + 68 + 4 * (int64_t)lmax + mcap;
}
template <typename FT>
__device__ void schur_target_warp(const TargetDev& g, const ContribDev* __restrict__ contribs,
                                  const TaskDev* __restrict__ tasks, const FT* __restrict__ fac,
                                  const int32_t* __restrict__ meta, double* __restrict__ blocks,
                                  const int64_t* __restrict__ blk_off, const int32_t* __restrict__ blk_ld,
                                  const int32_t* __restrict__ cur, int64_t* cm) {
    // cm (shared, 4 per contribution, at most 32 at a time): C of the
    // contribution offset to p's and q's columns, its leading dimension and f
    const int lane = threadIdx.x & 31;
    const int mp = cur[g.p], mq = cur[g.q];
    double* A = blocks + blk_off[g.blk_pq];
    const int lda = blk_ld[g.blk_pq];
    double* At = blocks + blk_off[g.blk_qp];
    const int ldt = blk_ld[g.blk_qp];
    for (int c0 = g.c_begin; c0 < g.c_end; c0 += 32) {
        const int nc = min(32, g.c_end - c0);
        if (lane < nc) {
            const ContribDev cb = contribs[c0 + lane];
            const TaskDev T = tasks[cb.task];
            const int32_t* mt = meta + T.meta;
            cm[4 * lane] = T.c_off + mt[1 + 2 * cb.kp];
            cm[4 * lane + 1] = T.c_off + mt[1 + 2 * cb.kq];
            cm[4 * lane + 2] = T.ncap;
            cm[4 * lane + 3] = T.s - mt[0];
        }
        __syncwarp();
        for (int idx = lane; idx < mp * mq; idx += 32) {
            const int i = idx / mq, j = idx % mq;
            FT acc = FT(0);
            for (int c = 0; c < nc; c++) {
                const FT* Cp = fac + cm[4 * c] + i;
                const FT* Cq = fac + cm[4 * c + 1] + j;
                const int64_t ld = cm[4 * c + 2];
                const int f = (int)cm[4 * c + 3];
                for (int k = 0; k < f; k++) acc += Cp[k * ld] * Cq[k * ld];
            }
            const double x = A[(int64_t)i * lda + j] - (double)acc;
            A[(int64_t)i * lda + j] = x;
            if (g.p != g.q) At[(int64_t)j * ldt + i] = x;
        }
        __syncwarp();
    }
}

// Grid-wide barrier for a cooperative launch (all CTAs co-resident).  bar[0]
// counts arrivals, bar[1] is the generation.  The wait is bounded: after
// `limit` polls (about a second by default) the CTA records ST_TIMEOUT; a
// CTA that sees ST_TIMEOUT recorded by another one while it waits stops
// waiting too.  Returns false (the same value on every thread of the CTA)
// when the launch has timed out: the caller then returns at once instead of
// computing on blocks that other CTAs may not have finished.  limit 0: no
// poll at all (a CTA that has to wait times out at once; for tests).
constexpr long long kBarrierSpins = 1LL << 24;

__device__ bool grid_sync(unsigned* bar, int32_t* status, long long limit) {
    __shared__ int s_ok;
    __threadfence();  // every thread's writes of this phase, device-visible
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* vgen = bar + 1;
        volatile int32_t* vst = status;
        const unsigned gen = *vgen;
        __threadfence();
        const unsigned arrived = atomicAdd(bar, 1u) + 1u;
        int ok = 1;
        if (arrived == gridDim.x) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            long long spins = 0;
            while (*vgen == gen) {
                if (spins++ >= limit) {
                    atomicCAS(status, 0, ST_TIMEOUT);
                    ok = 0;
                    break;
                }
                if (*vst == ST_TIMEOUT) {  // another CTA gave up: this barrier never completes
                    ok = 0;
                    break;
                }
                __nanosleep(40);
            }
        }
        if (*vst == ST_TIMEOUT) ok = 0;
        s_ok = ok;
        __threadfence();
    }
    __syncthreads();
    __threadfence();  // acquire side for every thread
    return s_ok != 0;
}

// Barrier between the steps of a fused level.  kClu false: the bounded grid
// barrier of a cooperative launch.  kClu true: the whole level runs in one
// thread-block cluster (its CTAs are resident together by construction) and
// waits on the cluster's hardware barrier, whose release / acquire pair
// orders one step's global-memory block updates before the next step's
// reads at cluster scope; the fences on either side make the same ordering
// explicit at device scope.
template <bool kClu>
__device__ __forceinline__ bool level_sync(unsigned* bar, int32_t* status, long long limit) {
    if constexpr (kClu) {
        __threadfence();
        asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
        __threadfence();
        return true;
    } else {
        return grid_sync(bar, status, limit);
    }
}

template <typename FT, bool kClu>
__global__ void __launch_bounds__(kFusedWarps * 32)
k_factor_level_fused(const TaskDev* __restrict__ tasks, const int32_t* __restrict__ ph_task,
                     const TargetDev* __restrict__ targets, const int32_t* __restrict__ ph_target,
                     const ContribDev* __restrict__ contribs, int nph, const ListDev* __restrict__ lists,
                     double* __restrict__ blocks, const int64_t* __restrict__ blk_off,
                     const int32_t* __restrict__ blk_ld, int32_t* __restrict__ cur, FT* __restrict__ fac,
                     int32_t* __restrict__ meta, double* __restrict__ ws, double eps2, int32_t* status,
                     int32_t level, int smax, int wmax, int lmax, int64_t mcap, unsigned* bar,
                     float* __restrict__ feat, const float* __restrict__ model, long long wait_limit) {
    extern __shared__ double sm[];
    const int wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    // items go to CTAs round-robin first (item k: CTA k mod grid, warp k /
    // grid), so that a phase's few clusters land on different SMs and do not
    // share an SM's FP64 pipe
    const int gw = wid * gridDim.x + blockIdx.x, GW = gridDim.x * nwarp;
    const int64_t wd = fused_warp_doubles(smax, wmax, lmax, mcap);
    double* d = sm + (size_t)wid * wd;
    int* ii = reinterpret_cast<int*>(sm + (size_t)nwarp * wd) + (size_t)wid * (lmax + 2);
    double* G = d;
    double* rdiag = G + (size_t)smax * smax;
    double* v = rdiag + smax;
    double* cn = v + smax;
    double* red = cn + wmax;
    double* hh = red + 64;
    EntryMeta* em = reinterpret_cast<EntryMeta*>(hh + 4);
    int64_t* colsrc = reinterpret_cast<int64_t*>(hh + 4 + 4 * (size_t)lmax);
    double* Msh = hh + 4 + 4 * (size_t)lmax + 2 * (size_t)wmax;
    int* ioff = ii;
    int* flag = ii + lmax + 1;
    WarpGroup g;
    for (int ph = 0; ph < nph; ph++) {
        for (int t = ph_task[ph] + gw; t < ph_task[ph + 1]; t += GW) {
            const TaskDev T = tasks[t];
            // small clusters take the register path unless features are recorded
            if (feat == nullptr && model == nullptr &&
                small_factor_task<FT>(T, G, rdiag, ioff, em, lists, blocks, blk_off, blk_ld, cur, fac, meta, eps2,
                                      status, level))
                continue;
            factor_task<FT>(T, g, G, rdiag, v, cn, red, ioff, flag, hh, Msh, em, colsrc, lists, blocks,
                            blk_off, blk_ld, cur, fac, meta, ws, eps2, status, level,
                            feat ? feat + (size_t)t * kFeat : nullptr, model, nullptr, nullptr);
        }
        if (!level_sync<kClu>(bar, status, wait_limit)) return;
        for (int k = ph_target[ph] + gw; k < ph_target[ph + 1]; k += GW)
            schur_target_warp<FT>(targets[k], contribs, tasks, fac, meta, blocks, blk_off, blk_ld, cur, colsrc);
        if (!level_sync<kClu>(bar, status, wait_limit)) return;
    }
}

// ---------------------------------------------------------------------------
// Block copies (level assembly and dense top assembly).
// ---------------------------------------------------------------------------
__global__ void k_copy_blocks(const CopyDev* __restrict__ cps, const double* __restrict__ src,
                              double* __restrict__ dst) {
    const CopyDev c = cps[blockIdx.x];
    for (int idx = threadIdx.x; idx < c.rows * c.cols; idx += blockDim.x) {
        const int i = idx / c.cols, j = idx % c.cols;
        dst[c.dst + (int64_t)i * c.dst_ld + j] = src[c.src + (int64_t)i * c.src_ld + j];
    }
}

// Dense Cholesky of the top (lower, row-major, in place), one CTA.
__global__ void __launch_bounds__(1024) k_dense_cholesky(int n, double* a, int32_t* status) {
    __shared__ int flag;
    __shared__ double rd;
    const int tid = threadIdx.x, NT = blockDim.x;
    if (tid == 0) flag = 0;
    for (int j = 0; j < n; j++) {
        __syncthreads();
        if (tid == 0) {
            const double d = a[(int64_t)j * n + j];
            if (!(d > 0.0)) flag = 1;
            else {
                a[(int64_t)j * n + j] = sqrt(d);
                rd = 1.0 / sqrt(d);
            }
        }
        __syncthreads();
        if (flag) {
            if (tid == 0 && atomicCAS(status, 0, ST_NOT_SPD) == 0) {
                status[1] = -1;
                status[2] = j;
            }
            return;
        }
        for (int i = j + 1 + tid; i < n; i += NT) a[(int64_t)i * n + j] *= rd;
        __syncthreads();
        const int m = n - j - 1;
        for (int idx = tid; idx < m * m; idx += NT) {
            const int i = j + 1 + idx / m, k = j + 1 + idx % m;
            if (k <= i) a[(int64_t)i * n + k] -= a[(int64_t)i * n + j] * a[(int64_t)k * n + j];
        }
    }
    __syncthreads();
    for (int idx = tid; idx < n * n; idx += NT)
        if (idx % n > idx / n) a[idx] = 0.0;
}

// ---------------------------------------------------------------------------
// Solve phase (Algorithm 2)
// ---------------------------------------------------------------------------
constexpr int kApplyThreads = 128;

// v - sum of stage[pulls[pi].off + j] over pi in [p0, p1), subtracted in
// ascending pi.  The offsets and values are fetched eight pulls at a time, so
// a task with P pulls waits for 2 ceil(P/8) rounds of loads instead of 2P.
__device__ __forceinline__ double sub_pulls(double v, const ApPull* __restrict__ pulls, int p0, int p1,
                                            const double* __restrict__ stage, int j) {
    constexpr int kB = 8;
    for (int pi = p0; pi < p1; pi += kB) {
        int64_t o[kB];
        double u[kB];
#pragma unroll
        for (int k = 0; k < kB; k++) o[k] = pi + k < p1 ? pulls[pi + k].off : -1;
#pragma unroll
        for (int k = 0; k < kB; k++) u[k] = o[k] >= 0 ? stage[o[k] + j] : 0.0;
#pragma unroll
        for (int k = 0; k < kB; k++)
            if (pi + k < p1) v -= u[k];
    }
    return v;
}

// Gathers the neighbour slices nbs[e0, e1) of y into xnf (converted to FT):
// xnf[nb.col + j] = y[nb.y + j] for j < nb.m, by threads g, g + gs, ...
// Four descriptors, then their first values, are fetched per round of loads.
template <typename FT>
__device__ __forceinline__ void gather_nbs(const ApNb* __restrict__ nbs, int e0, int e1,
                                           const double* __restrict__ y, FT* xnf, int g, int gs) {
    constexpr int kB = 4;
    for (int e = e0; e < e1; e += kB) {
        ApNb nb[kB];
        double u[kB];
#pragma unroll
        for (int k = 0; k < kB; k++) nb[k] = e + k < e1 ? nbs[e + k] : ApNb{0, 0, 0};
#pragma unroll
        for (int k = 0; k < kB; k++) u[k] = g < nb[k].m ? y[nb[k].y + g] : 0.0;
#pragma unroll
        for (int k = 0; k < kB; k++) {
            if (g < nb[k].m) xnf[nb[k].col + g] = (FT)u[k];
            for (int j = g + gs; j < nb[k].m; j += gs) xnf[nb[k].col + j] = (FT)y[nb[k].y + j];
        }
    }
}

// ----- solve phase, fine levels: one CTA per task, one launch per phase -----

// Forward step of one phase:
//   y_c -= staged updates of the tasks of earlier phases that have c as a
//          neighbour (ascending task order);
//   y_c <- W_c y_c with W_c = U^T G^-1;
//   stage d_c = C_c^T y_c(r:), the update of every neighbour of c (Eq. elim
//          applied to the vector), consumed by later tasks or at level end.
template <typename FT>
__global__ void __launch_bounds__(kApplyThreads)
k_ap_fwd(const ApTask* __restrict__ tasks, int t0, const ApPull* __restrict__ pulls,
         const FT* __restrict__ fac, double* __restrict__ stage, double* __restrict__ y, int smax) {
    // vectors in shared memory in the factor's type: each FP64 value is
    // converted once (conversions run on the FP64 pipe)
    extern __shared__ double sh[];
    FT* ys = reinterpret_cast<FT*>(sh);
    FT* yn = ys + smax;
    griddep_wait();
    griddep_release();
    const ApTask T = tasks[t0 + blockIdx.x];
    const int s = T.s, tid = threadIdx.x, NT = blockDim.x;
    double* yg = y + T.y;
    for (int j = tid; j < s; j += NT) {
        double v = yg[j];
        v = sub_pulls(v, pulls, T.pull0, T.pull1, stage, j);
        ys[j] = (FT)v;
    }
    __syncthreads();
    const FT* Wm = fac + T.w;
    const int lane = tid & 31, wid = tid >> 5, nwarp = NT >> 5;
    for (int i0 = 4 * wid; i0 < s; i0 += 4 * nwarp) {
        FT a[4] = {FT(0), FT(0), FT(0), FT(0)};
        for (int j = lane; j < s; j += 32) {
            const FT yj = ys[j];
#pragma unroll
            for (int u = 0; u < 4; u++)
                if (i0 + u < s) a[u] += Wm[(int64_t)(i0 + u) * s + j] * yj;
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const FT t = warp_sum(a[u]);
            if (lane == 0 && i0 + u < s) yn[i0 + u] = t;
        }
    }
    __syncthreads();
    for (int j = tid; j < s; j += NT) yg[j] = (double)yn[j];
    const int f = s - T.r;
    const FT* C = fac + T.cm;
    const FT* yf = yn + T.r;
    int jv = 0;  // columns below jv done with vector loads
    if constexpr (sizeof(FT) == sizeof(float)) {
        // four columns per thread, one aligned float4 per row (C and its
        // leading dimension are multiples of 4 floats)
        jv = T.ncols & ~3;
        const int ncg = jv >> 2;
        int P = 32;  // threads per row chunk: a power of two >= the column groups
        while (P < ncg) P <<= 1;
        if (P <= NT / 2 && f >= 16) {
            // the rows in R = NT / P chunks, eight rows in flight per thread;
            // the chunks' partial sums are added in chunk order through
            // shared memory (behind the two vectors)
            const int R = NT / P, q = tid / P, cg = tid % P;
            const int i0 = q * f / R, i1 = (q + 1) * f / R;
            float4 p0 = make_float4(0.f, 0.f, 0.f, 0.f), p1 = p0;
            if (cg < ncg) {
                const float* cj = reinterpret_cast<const float*>(C) + 4 * cg;
                int i = i0;
                for (; i + 7 < i1; i += 8) {
                    float4 c[8];
#pragma unroll
                    for (int u = 0; u < 8; u++) c[u] = *reinterpret_cast<const float4*>(cj + (int64_t)(i + u) * T.ncap);
#pragma unroll
                    for (int u = 0; u < 8; u += 2) {
                        const float ya = yf[i + u], yb = yf[i + u + 1];
                        p0.x += c[u].x * ya; p0.y += c[u].y * ya; p0.z += c[u].z * ya; p0.w += c[u].w * ya;
                        p1.x += c[u + 1].x * yb; p1.y += c[u + 1].y * yb;
                        p1.z += c[u + 1].z * yb; p1.w += c[u + 1].w * yb;
                    }
                }
                for (; i < i1; i++) {
                    const float4 c0 = *reinterpret_cast<const float4*>(cj + (int64_t)i * T.ncap);
                    const float y0 = yf[i];
                    p0.x += c0.x * y0; p0.y += c0.y * y0; p0.z += c0.z * y0; p0.w += c0.w * y0;
                }
            }
            float4* red = reinterpret_cast<float4*>(sh + 2 * smax);
            red[tid] = make_float4(p0.x + p1.x, p0.y + p1.y, p0.z + p1.z, p0.w + p1.w);
            __syncthreads();
            if (q == 0 && cg < ncg) {
                float4 a = red[cg];
                for (int k = 1; k < R; k++) {
                    const float4 b = red[k * P + cg];
                    a.x += b.x; a.y += b.y; a.z += b.z; a.w += b.w;
                }
                double* st = stage + T.stg + 4 * cg;
                st[0] = (double)a.x;
                st[1] = (double)a.y;
                st[2] = (double)a.z;
                st[3] = (double)a.w;
            }
        } else {
            // more column groups than half the threads: one thread per group
            for (int j4 = 4 * tid; j4 < jv; j4 += 4 * NT) {
                float4 p0 = make_float4(0.f, 0.f, 0.f, 0.f), p1 = p0;
                const float* cj = reinterpret_cast<const float*>(C) + j4;
                int i = 0;
                for (; i + 3 < f; i += 4) {
                    const float4 c0 = *reinterpret_cast<const float4*>(cj + (int64_t)i * T.ncap);
                    const float4 c1 = *reinterpret_cast<const float4*>(cj + (int64_t)(i + 1) * T.ncap);
                    const float4 c2 = *reinterpret_cast<const float4*>(cj + (int64_t)(i + 2) * T.ncap);
                    const float4 c3 = *reinterpret_cast<const float4*>(cj + (int64_t)(i + 3) * T.ncap);
                    const float y0 = yf[i], y1 = yf[i + 1], y2 = yf[i + 2], y3 = yf[i + 3];
                    p0.x += c0.x * y0 + c2.x * y2; p0.y += c0.y * y0 + c2.y * y2;
                    p0.z += c0.z * y0 + c2.z * y2; p0.w += c0.w * y0 + c2.w * y2;
                    p1.x += c1.x * y1 + c3.x * y3; p1.y += c1.y * y1 + c3.y * y3;
                    p1.z += c1.z * y1 + c3.z * y3; p1.w += c1.w * y1 + c3.w * y3;
                }
                for (; i < f; i++) {
                    const float4 c0 = *reinterpret_cast<const float4*>(cj + (int64_t)i * T.ncap);
                    const float y0 = yf[i];
                    p0.x += c0.x * y0; p0.y += c0.y * y0; p0.z += c0.z * y0; p0.w += c0.w * y0;
                }
                double* st = stage + T.stg + j4;
                st[0] = (double)(p0.x + p1.x);
                st[1] = (double)(p0.y + p1.y);
                st[2] = (double)(p0.z + p1.z);
                st[3] = (double)(p0.w + p1.w);
            }
        }
    }
    for (int j = jv + tid; j < T.ncols; j += NT) {
        FT a0 = FT(0), a1 = FT(0), a2 = FT(0), a3 = FT(0);
        const FT* cj = C + j;
        int i = 0;
        for (; i + 3 < f; i += 4) {
            a0 += cj[(int64_t)i * T.ncap] * yf[i];
            a1 += cj[(int64_t)(i + 1) * T.ncap] * yf[i + 1];
            a2 += cj[(int64_t)(i + 2) * T.ncap] * yf[i + 2];
            a3 += cj[(int64_t)(i + 3) * T.ncap] * yf[i + 3];
        }
        for (; i < f; i++) a0 += cj[(int64_t)i * T.ncap] * yf[i];
        stage[T.stg + j] = (double)((a0 + a1) + (a2 + a3));
    }
}

// End of a level's forward solve, one CTA per cluster with a coarse part.
__global__ void __launch_bounds__(kApplyThreads)
k_ap_fin(const ApFin* __restrict__ fins, const ApPull* __restrict__ pulls, const double* __restrict__ stage,
         double* __restrict__ y, double* __restrict__ ynext, double* __restrict__ ytop) {
    griddep_wait();
    griddep_release();
    const ApFin F = fins[blockIdx.x];
    double* dst = (F.to_top ? ytop : ynext) + F.dst;
    for (int j = threadIdx.x; j < F.len; j += blockDim.x) {
        double v = y[F.y + j];
        v = sub_pulls(v, pulls, F.pull0, F.pull1, stage, j);
        y[F.y + j] = v;
        dst[j] = v;
    }
}

// Backward step of one phase: x_c(r:) -= C x_n, then x_c <- W_c^T x_c.
template <typename FT>
__global__ void __launch_bounds__(kApplyThreads)
k_ap_bwd(const ApTask* __restrict__ tasks, int t0, const ApNb* __restrict__ nbs, const FT* __restrict__ fac,
         double* __restrict__ y, int smax, int nmax) {
    // xs in FP64 (it is updated in place), copies of xs and the neighbour
    // values in the factor's type (each converted once)
    extern __shared__ double sh[];
    double* xs = sh;
    double* part = sh + smax;
    FT* xnf = reinterpret_cast<FT*>(part + blockDim.x);
    FT* xsf = xnf + nmax;
    griddep_wait();
    griddep_release();
    const ApTask T = tasks[t0 + blockIdx.x];
    const int s = T.s, r = T.r, f = s - r, tid = threadIdx.x, NT = blockDim.x;
    double* yg = y + T.y;
    for (int i = tid; i < s; i += NT) xs[i] = yg[i];
    gather_nbs<FT>(nbs, T.nb0, T.nb1, y, xnf, tid, NT);
    __syncthreads();
    const FT* C = fac + T.cm;
    const int lane = tid & 31, wid = tid >> 5, nwarp = NT >> 5;
    if constexpr (sizeof(FT) == sizeof(float)) {
        // four rows per warp, four columns per lane (aligned float4 loads)
        const int jv = T.ncols & ~3;
        for (int i0 = 4 * wid; i0 < f; i0 += 4 * nwarp) {
            float a[4] = {0.f, 0.f, 0.f, 0.f};
            for (int j4 = 4 * lane; j4 < jv; j4 += 128) {
                const float x0 = xnf[j4], x1 = xnf[j4 + 1], x2 = xnf[j4 + 2], x3 = xnf[j4 + 3];
#pragma unroll
                for (int u = 0; u < 4; u++)
                    if (i0 + u < f) {
                        const float4 c4 = *reinterpret_cast<const float4*>(reinterpret_cast<const float*>(C) +
                                                                          (int64_t)(i0 + u) * T.ncap + j4);
                        a[u] += c4.x * x0 + c4.y * x1 + c4.z * x2 + c4.w * x3;
                    }
            }
            for (int j = jv + lane; j < T.ncols; j += 32) {
                const float xj = xnf[j];
#pragma unroll
                for (int u = 0; u < 4; u++)
                    if (i0 + u < f) a[u] += (float)C[(int64_t)(i0 + u) * T.ncap + j] * xj;
            }
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const float su = warp_sum(a[u]);
                if (lane == 0 && i0 + u < f) xs[r + i0 + u] -= (double)su;
            }
        }
    } else {
        for (int i0 = 2 * wid; i0 < f; i0 += 2 * nwarp) {
            FT a0 = FT(0), a1 = FT(0);
            const bool two = i0 + 1 < f;
            for (int j = lane; j < T.ncols; j += 32) {
                const FT xj = xnf[j];
                a0 += C[(int64_t)i0 * T.ncap + j] * xj;
                if (two) a1 += C[(int64_t)(i0 + 1) * T.ncap + j] * xj;
            }
            const double s0 = warp_sum((double)a0);
            const double s1 = warp_sum((double)a1);
            if (lane == 0) {
                xs[r + i0] -= s0;
                if (two) xs[r + i0 + 1] -= s1;
            }
        }
    }
    __syncthreads();
    for (int i = tid; i < s; i += NT) xsf[i] = (FT)xs[i];
    __syncthreads();
    const FT* Wm = fac + T.w;
    if (s >= NT) {
        for (int jj = tid; jj < s; jj += NT) {
            FT a0 = FT(0), a1 = FT(0);
            int i = 0;
            for (; i + 1 < s; i += 2) {
                a0 += Wm[(int64_t)i * s + jj] * xsf[i];
                a1 += Wm[(int64_t)(i + 1) * s + jj] * xsf[i + 1];
            }
            if (i < s) a0 += Wm[(int64_t)i * s + jj] * xsf[i];
            yg[jj] = (double)(a0 + a1);
        }
        return;
    }
    const int G = NT / s, g = tid / s, j = tid % s;
    FT a0 = FT(0), a1 = FT(0);
    if (g < G) {
        int i = g;
        for (; i + G < s; i += 2 * G) {
            a0 += Wm[(int64_t)i * s + j] * xsf[i];
            a1 += Wm[(int64_t)(i + G) * s + j] * xsf[i + G];
        }
        if (i < s) a0 += Wm[(int64_t)i * s + j] * xsf[i];
    }
    part[tid] = (double)(a0 + a1);
    __syncthreads();
    if (tid < s) {
        double t = 0.0;
        for (int gg = 0; gg < G; gg++) t += part[gg * s + tid];
        yg[tid] = t;
    }
}

// ----- solve phase, coarse levels: one CTA, one warp per task -----
// Per-warp shared memory: the cluster's vector (kCoarseSmax doubles) and the
// transformed vector / gathered neighbour values (kCoarseNmax doubles).

template <typename FT>
__device__ void group_fwd(bool act, const ApTask& T, int gl, int gs, const ApPull* __restrict__ pulls,
                          const FT* __restrict__ fac, double* __restrict__ stage, double* __restrict__ y,
                          double* ys, double* yn) {
    // the vectors in the factor's type (each FP64 value converted once);
    // with a float factor both fit in the space of ys
    FT* ysf = reinterpret_cast<FT*>(ys);
    FT* ynf = sizeof(FT) == sizeof(double) ? reinterpret_cast<FT*>(yn) : ysf + kCoarseSmax;
    const int s = act ? T.s : 0;
    for (int j = gl; j < s; j += gs) {
        double v = y[T.y + j];
        v = sub_pulls(v, pulls, T.pull0, T.pull1, stage, j);
        ysf[j] = (FT)v;
    }
    __syncwarp();
    if (act) {
        const FT* Wm = fac + T.w;
        for (int i = gl; i < s; i += gs) {
            const FT* wi = Wm + (int64_t)i * s;
            FT a0 = FT(0), a1 = FT(0), a2 = FT(0), a3 = FT(0);
            int j = 0;
            for (; j + 3 < s; j += 4) {
                a0 += wi[j] * ysf[j];
                a1 += wi[j + 1] * ysf[j + 1];
                a2 += wi[j + 2] * ysf[j + 2];
                a3 += wi[j + 3] * ysf[j + 3];
            }
            for (; j < s; j++) a0 += wi[j] * ysf[j];
            ynf[i] = (a0 + a1) + (a2 + a3);
        }
    }
    __syncwarp();
    if (act) {
        for (int j = gl; j < s; j += gs) y[T.y + j] = (double)ynf[j];
        const int f = s - T.r;
        const FT* C = fac + T.cm;
        const FT* yf = ynf + T.r;
        for (int j = gl; j < T.ncols; j += gs) {
            const FT* cj = C + j;
            FT a0 = FT(0), a1 = FT(0), a2 = FT(0), a3 = FT(0);
            int i = 0;
            for (; i + 3 < f; i += 4) {
                a0 += cj[(int64_t)i * T.ncap] * yf[i];
                a1 += cj[(int64_t)(i + 1) * T.ncap] * yf[i + 1];
                a2 += cj[(int64_t)(i + 2) * T.ncap] * yf[i + 2];
                a3 += cj[(int64_t)(i + 3) * T.ncap] * yf[i + 3];
            }
            for (; i < f; i++) a0 += cj[(int64_t)i * T.ncap] * yf[i];
            stage[T.stg + j] = (double)((a0 + a1) + (a2 + a3));
        }
    }
    __syncwarp();
}

template <typename FT>
__device__ void group_bwd(bool act, const ApTask& T, int gl, int gs, const ApNb* __restrict__ nbs,
                          const FT* __restrict__ fac, double* __restrict__ y, double* xs, double* xn) {
    // xs (FP64, updated in place) and copies in the factor's type of the
    // neighbour values and of xs: each FP64 value converted once.  With a
    // float factor the copies fit in the space of xn (kCoarseNmax doubles).
    FT* xnf = reinterpret_cast<FT*>(xn);
    FT* xsf = sizeof(FT) == sizeof(double) ? reinterpret_cast<FT*>(xs) : xnf + kCoarseNmax;
    const int s = act ? T.s : 0, r = T.r, f = s - r;
    for (int i = gl; i < s; i += gs) xs[i] = y[T.y + i];
    const int ncols = act ? T.ncols : 0;
    if (act) gather_nbs<FT>(nbs, T.nb0, T.nb1, y, xnf, gl, gs);
    __syncwarp();
    if (act) {
        const FT* C = fac + T.cm;
        for (int i = gl; i < f; i += gs) {
            const FT* ci = C + (int64_t)i * T.ncap;
            FT a0 = FT(0), a1 = FT(0), a2 = FT(0), a3 = FT(0);
            int j = 0;
            for (; j + 3 < ncols; j += 4) {
                a0 += ci[j] * xnf[j];
                a1 += ci[j + 1] * xnf[j + 1];
                a2 += ci[j + 2] * xnf[j + 2];
                a3 += ci[j + 3] * xnf[j + 3];
            }
            for (; j < ncols; j++) a0 += ci[j] * xnf[j];
            xs[r + i] -= (double)((a0 + a1) + (a2 + a3));
        }
    }
    __syncwarp();
    if (sizeof(FT) != sizeof(double))
        for (int i = gl; i < s; i += gs) xsf[i] = (FT)xs[i];
    __syncwarp();
    if (act) {
        const FT* Wm = fac + T.w;
        for (int j = gl; j < s; j += gs) {
            FT a0 = FT(0), a1 = FT(0), a2 = FT(0), a3 = FT(0);
            int i = 0;
            for (; i + 3 < s; i += 4) {
                a0 += Wm[(int64_t)i * s + j] * xsf[i];
                a1 += Wm[(int64_t)(i + 1) * s + j] * xsf[i + 1];
                a2 += Wm[(int64_t)(i + 2) * s + j] * xsf[i + 2];
                a3 += Wm[(int64_t)(i + 3) * s + j] * xsf[i + 3];
            }
            for (; i < s; i++) a0 += Wm[(int64_t)i * s + j] * xsf[i];
            y[T.y + j] = (double)((a0 + a1) + (a2 + a3));
        }
    }
    __syncwarp();
}

// Forward over the coarse levels, the dense top (L^-T L^-1), then backward,
// with __syncthreads between stages instead of kernel boundaries.  `off` is
// added to every level vector, stage and top-vector address (a private
// workspace per CTA when the chain is run on many right-hand sides at once).
template <typename FT>
__device__ void coarse_chain(const ApLevel* __restrict__ lvl, int nlev, int ntop, const double* __restrict__ Ltop,
                             double* __restrict__ ytop, int64_t off) {
    extern __shared__ double sh[];
    const int tid = threadIdx.x, NT = blockDim.x, lane = tid & 31, wid = tid >> 5, nwarp = NT >> 5;
    double* wsh = sh + (size_t)wid * (kCoarseSmax + kCoarseNmax);
    ytop += off;
    for (int l = 0; l < nlev; l++) {
        const ApLevel V = lvl[l];
        double* yv = V.y + off;
        double* ynx = V.ynext + off;
        double* stg = V.stage + off;
        double* ys = wsh;
        double* yn = ys + kCoarseSmax;
        for (int ph = 0; ph < V.nph; ph++) {
            const int b = V.ph[ph], e = V.ph[ph + 1];
            for (int t = b + wid; t < e; t += nwarp) group_fwd<FT>(true, V.tasks[t], lane, 32, V.pulls, static_cast<const FT*>(V.fac), stg, yv, ys, yn);
            __syncthreads();
        }
        for (int k = wid; k < V.nfin; k += nwarp) {
            const ApFin F = V.fins[k];
            for (int j = lane; j < F.len; j += 32) {
                double v = yv[F.y + j];
                v = sub_pulls(v, V.pulls, F.pull0, F.pull1, stg, j);
                yv[F.y + j] = v;
                ynx[F.dst + j] = v;
            }
        }
        __syncthreads();
    }
    for (int k = 0; k < ntop; k++) {
        const double yk = ytop[k] / Ltop[(int64_t)k * ntop + k];
        __syncthreads();
        if (tid == 0) ytop[k] = yk;
        for (int i = k + 1 + tid; i < ntop; i += NT) ytop[i] -= Ltop[(int64_t)i * ntop + k] * yk;
        __syncthreads();
    }
    for (int k = ntop - 1; k >= 0; k--) {
        const double yk = ytop[k] / Ltop[(int64_t)k * ntop + k];
        __syncthreads();
        if (tid == 0) ytop[k] = yk;
        for (int i = tid; i < k; i += NT) ytop[i] -= Ltop[(int64_t)k * ntop + i] * yk;
        __syncthreads();
    }
    for (int l = nlev - 1; l >= 0; l--) {
        const ApLevel V = lvl[l];
        double* yv = V.y + off;
        const double* ynx = V.ynext + off;
        double* xs = wsh;
        double* xn = xs + kCoarseSmax;
        for (int k = wid; k < V.nvcopy; k += nwarp) {
            const VCopyDev c = V.vcopy[k];
            for (int j = lane; j < c.len; j += 32) yv[c.src + j] = ynx[c.dst + j];
        }
        __syncthreads();
        for (int ph = V.nph - 1; ph >= 0; ph--) {
            const int b = V.ph[ph], e = V.ph[ph + 1];
            for (int t = b + wid; t < e; t += nwarp) group_bwd<FT>(true, V.tasks[t], lane, 32, V.nbs, static_cast<const FT*>(V.fac), yv, xs, xn);
            __syncthreads();
        }
    }
}

template <typename FT>
__global__ void __launch_bounds__(kCoarseThreads)
k_ap_coarse(const ApLevel* __restrict__ lvl, int nlev, int ntop, const double* __restrict__ Ltop,
            double* __restrict__ ytop) {
    griddep_wait();
    griddep_release();
    coarse_chain<FT>(lvl, nlev, ntop, Ltop, ytop, 0);
}

// Explicit coarse operator: CTA j runs the coarse chain on the unit vector e_j
// in its own workspace (stride doubles apart) and writes the result as row j
// of Mc (n x n; symmetric up to rounding).  yin0 is CTA 0's input vector.
template <typename FT>
__global__ void __launch_bounds__(kCoarseThreads)
k_ap_coarse_batch(const ApLevel* __restrict__ lvl, int nlev, int ntop, const double* __restrict__ Ltop,
                  double* __restrict__ ytop, double* __restrict__ yin0, int n, int64_t stride,
                  double* __restrict__ Mc) {
    const int64_t off = (int64_t)blockIdx.x * stride;
    double* yin = yin0 + off;
    for (int i = threadIdx.x; i < n; i += blockDim.x) yin[i] = (i == (int)blockIdx.x) ? 1.0 : 0.0;
    __syncthreads();
    coarse_chain<FT>(lvl, nlev, ntop, Ltop, ytop, off);
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) Mc[(int64_t)blockIdx.x * n + i] = yin[i];
}

// y = Mc x (n x n, row-major): one warp per row, lanes over columns.
__global__ void __launch_bounds__(256) k_dense_gemv(int n, const double* __restrict__ Mc,
                                                    const double* __restrict__ x, double* __restrict__ y) {
    griddep_wait();
    griddep_release();
    const int lane = threadIdx.x & 31;
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= n) return;
    const double* m = Mc + (int64_t)row * n;
    double a0 = 0.0, a1 = 0.0;
    int j = lane;
    for (; j + 32 < n; j += 64) {
        a0 += m[j] * x[j];
        a1 += m[j + 32] * x[j + 32];
    }
    if (j < n) a0 += m[j] * x[j];
    const double t = warp_sum(a0 + a1);
    if (lane == 0) y[row] = t;
}

// reverse: y_level[src] <- (to_top ? ytop : y_next)[dst]; forward the other way
__global__ void k_vcopy(const VCopyDev* __restrict__ cps, int ncps, const double* __restrict__ src,
                        double* __restrict__ dst, int reverse, const double* __restrict__ ytop) {
    griddep_wait();
    griddep_release();
    const int c = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (c >= ncps) return;
    const VCopyDev v = cps[c];
    const double* from = (reverse && v.to_top) ? ytop : src;
    for (int i = threadIdx.x & 31; i < v.len; i += 32) {
        if (reverse) dst[v.src + i] = from[v.dst + i];
        else dst[v.dst + i] = src[v.src + i];
    }
}

// Dense Cholesky of every top (one CTA per problem), status like the factor.
__global__ void __launch_bounds__(256) k_tops_cholesky(const TopDev* __restrict__ tops, int32_t* status) {
    __shared__ int flag;
    __shared__ double rd;
    const TopDev tp = tops[blockIdx.x];
    const int n = tp.n, tid = threadIdx.x, NT = blockDim.x;
    double* a = tp.L;
    if (tid == 0) flag = 0;
    for (int j = 0; j < n; j++) {
        __syncthreads();
        if (tid == 0) {
            const double d = a[(int64_t)j * n + j];
            if (!(d > 0.0)) flag = 1;
            else {
                a[(int64_t)j * n + j] = sqrt(d);
                rd = 1.0 / sqrt(d);
            }
        }
        __syncthreads();
        if (flag) {
            if (tid == 0 && atomicCAS(status, 0, ST_NOT_SPD) == 0) {
                status[1] = -1;
                status[2] = blockIdx.x;
            }
            return;
        }
        for (int i = j + 1 + tid; i < n; i += NT) a[(int64_t)i * n + j] *= rd;
        __syncthreads();
        const int m = n - j - 1;
        for (int idx = tid; idx < m * m; idx += NT) {
            const int i = j + 1 + idx / m, k = j + 1 + idx % m;
            if (k <= i) a[(int64_t)i * n + k] -= a[(int64_t)i * n + j] * a[(int64_t)k * n + j];
        }
    }
    __syncthreads();
    for (int idx = tid; idx < n * n; idx += NT)
        if (idx % n > idx / n) a[idx] = 0.0;
}

// y <- L^-T L^-1 y for every top (one CTA per problem).
__global__ void __launch_bounds__(256) k_tops_solve(const TopDev* __restrict__ tops, double* __restrict__ ytop) {
    griddep_wait();
    griddep_release();
    const TopDev tp = tops[blockIdx.x];
    const int n = tp.n, tid = threadIdx.x, NT = blockDim.x;
    const double* L = tp.L;
    double* y = ytop + tp.vec_off;
    for (int k = 0; k < n; k++) {
        __syncthreads();
        const double yk = y[k] / L[(int64_t)k * n + k];
        __syncthreads();
        if (tid == 0) y[k] = yk;
        for (int i = k + 1 + tid; i < n; i += NT) y[i] -= L[(int64_t)i * n + k] * yk;
    }
    for (int k = n - 1; k >= 0; k--) {
        __syncthreads();
        const double yk = y[k] / L[(int64_t)k * n + k];
        __syncthreads();
        if (tid == 0) y[k] = yk;
        for (int i = tid; i < k; i += NT) y[i] -= L[(int64_t)k * n + i] * yk;
    }
}

// y <- L^-T L^-1 y for the dense top (one CTA).
__global__ void __launch_bounds__(1024) k_top_solve(int n, const double* __restrict__ L, double* __restrict__ y) {
    const int tid = threadIdx.x, NT = blockDim.x;
    for (int k = 0; k < n; k++) {
        __syncthreads();
        const double yk = y[k] / L[(int64_t)k * n + k];
        __syncthreads();
        if (tid == 0) y[k] = yk;
        for (int i = k + 1 + tid; i < n; i += NT) y[i] -= L[(int64_t)i * n + k] * yk;
    }
    for (int k = n - 1; k >= 0; k--) {
        __syncthreads();
        const double yk = y[k] / L[(int64_t)k * n + k];
        __syncthreads();
        if (tid == 0) y[k] = yk;
        for (int i = tid; i < k; i += NT) y[i] -= L[(int64_t)k * n + i] * yk;
    }
}

__global__ void k_permute(int64_t n, const int32_t* __restrict__ perm, const double* __restrict__ src,
                          double* __restrict__ dst, int inverse) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (inverse) dst[perm[i]] = src[i];
    else dst[i] = src[perm[i]];
}

// ---------------------------------------------------------------------------
// Krylov pieces
// ---------------------------------------------------------------------------
__global__ void k_spmv(int64_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                       const double* __restrict__ val, const double* __restrict__ x, double* __restrict__ y) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double t = 0.0;
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; e++) t += val[e] * x[col[e]];
    y[i] = t;
}

__global__ void __launch_bounds__(256) k_dot_partial(int64_t n, const double* __restrict__ a,
                                                     const double* __restrict__ b, double* __restrict__ partial) {
    __shared__ double red[32];
    double t = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        t += a[i] * b[i];
    t = block_sum(t, red);
    if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

__global__ void __launch_bounds__(1024) k_sum_partials(const double* __restrict__ partial, int np,
                                                       double* __restrict__ out) {
    __shared__ double red[32];
    double t = 0.0;
    for (int i = threadIdx.x; i < np; i += blockDim.x) t += partial[i];
    t = block_sum(t, red);
    if (threadIdx.x == 0) *out = t;
}

__global__ void k_pcg_xr(int64_t n, const double* __restrict__ rz, const double* __restrict__ pq,
                         const double* __restrict__ p, const double* __restrict__ q, double* __restrict__ x,
                         double* __restrict__ r) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double alpha = *rz / *pq;
    x[i] += alpha * p[i];
    r[i] -= alpha * q[i];
}

__global__ void k_pcg_p(int64_t n, const double* __restrict__ rzn, const double* __restrict__ rzo,
                        const double* __restrict__ z, double* __restrict__ p) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double beta = *rzn / *rzo;
    p[i] = z[i] + beta * p[i];
}

// ---- fused PCG steps: each adds a dot product to its vector pass ----
// The blocks' partial sums go to partial[block]; the last block to arrive
// (counted in *count, which it resets to zero) adds them in index order into
// *out, so the value depends only on the grid, not on the arrival order.
__device__ __forceinline__ void dot_finish(double v, double* __restrict__ partial, unsigned* __restrict__ count,
                                           double* __restrict__ out) {
    __shared__ double red[32];
    __shared__ int last;
    v = block_sum(v, red);
    if (threadIdx.x == 0) {
        partial[blockIdx.x] = v;
        __threadfence();
        last = atomicAdd(count, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last) {
        __threadfence();
        double t = 0.0;
        for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) t += __ldcg(partial + i);
        t = block_sum(t, red);
        if (threadIdx.x == 0) {
            *out = t;
            *count = 0;
        }
    }
}

// y = A x and *out = x^T y (the SpMV and p^T A p of a PCG step)
__global__ void __launch_bounds__(256) k_spmv_dot(int64_t n, const int64_t* __restrict__ rowptr,
                                                  const int32_t* __restrict__ col, const double* __restrict__ val,
                                                  const double* __restrict__ x, double* __restrict__ y,
                                                  double* __restrict__ partial, unsigned* __restrict__ count,
                                                  double* __restrict__ out) {
    double d = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double t = 0.0;
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; e++) t += val[e] * x[col[e]];
        y[i] = t;
        d += x[i] * t;
    }
    dot_finish(d, partial, count, out);
}

// x += alpha p, r -= alpha q with alpha = rz / pq, and *out = r^T r
__global__ void __launch_bounds__(256) k_pcg_xr_dot(int64_t n, const double* __restrict__ rz,
                                                    const double* __restrict__ pq, const double* __restrict__ p,
                                                    const double* __restrict__ q, double* __restrict__ x,
                                                    double* __restrict__ r, double* __restrict__ partial,
                                                    unsigned* __restrict__ count, double* __restrict__ out) {
    const double alpha = *rz / *pq;
    double d = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        x[i] += alpha * p[i];
        const double ri = r[i] - alpha * q[i];
        r[i] = ri;
        d += ri * ri;
    }
    dot_finish(d, partial, count, out);
}

// *out = a^T b in one launch
__global__ void __launch_bounds__(256) k_dot_fused(int64_t n, const double* __restrict__ a,
                                                   const double* __restrict__ b, double* __restrict__ partial,
                                                   unsigned* __restrict__ count, double* __restrict__ out) {
    double d = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        d += a[i] * b[i];
    dot_finish(d, partial, count, out);
}

// ---- batched PCG: independent problems on one block-diagonal system ----
// Problem p owns entries pp[p] .. pp[p+1] of every vector; its scalars are
// sc[p * kBScal + slot] and its flags fl[p * kBFlag + slot] (BF_* slots).

// sc[p][slot] = a_p . b_p, one CTA per problem (fixed summation order).
__global__ void __launch_bounds__(256) k_seg_dot(const int64_t* __restrict__ pp, const double* __restrict__ a,
                                                 const double* __restrict__ b, double* __restrict__ sc, int slot) {
    __shared__ double red[32];
    const int p = blockIdx.x;
    const int64_t lo = pp[p], hi = pp[p + 1];
    double t = 0.0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) t += a[i] * b[i];
    t = block_sum(t, red);
    if (threadIdx.x == 0) sc[(int64_t)p * kBScal + slot] = t;
}

// x += alpha p, r -= alpha q on the active problems (alpha = rz / pq).
__global__ void k_bpcg_xr(const int64_t* __restrict__ pp, const double* __restrict__ sc,
                          const int32_t* __restrict__ fl, const double* __restrict__ p,
                          const double* __restrict__ q, double* __restrict__ x, double* __restrict__ r) {
    const int pr = blockIdx.y;
    if (!fl[pr * kBFlag + BF_ACTIVE]) return;
    const int64_t i = pp[pr] + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= pp[pr + 1]) return;
    const double alpha = sc[pr * kBScal + BS_RZ] / sc[pr * kBScal + BS_PQ];
    x[i] += alpha * p[i];
    r[i] -= alpha * q[i];
}

// p = z + beta p on the active problems (beta = rz_new / rz, 0 on a restart).
__global__ void k_bpcg_p(const int64_t* __restrict__ pp, const double* __restrict__ sc,
                         const int32_t* __restrict__ fl, const double* __restrict__ z, double* __restrict__ p) {
    const int pr = blockIdx.y;
    if (!fl[pr * kBFlag + BF_ACTIVE]) return;
    const int64_t i = pp[pr] + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= pp[pr + 1]) return;
    const double beta = fl[pr * kBFlag + BF_RESTART] ? 0.0 : sc[pr * kBScal + BS_RZN] / sc[pr * kBScal + BS_RZ];
    p[i] = z[i] + beta * p[i];
}

// r_p = q_p for the problems restarted from their true residual.
__global__ void k_bpcg_restart_copy(const int64_t* __restrict__ pp, const int32_t* __restrict__ fl,
                                    const double* __restrict__ q, double* __restrict__ r) {
    const int pr = blockIdx.y;
    if (!fl[pr * kBFlag + BF_ACTIVE] || !fl[pr * kBFlag + BF_RESTART]) return;
    const int64_t i = pp[pr] + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= pp[pr + 1]) return;
    r[i] = q[i];
}

// Per-problem bookkeeping, one CTA.  mode 0: start (active = b != 0,
// restart = 1); 1: after the p update (rz = rz_new, restart = 0); 2: after
// the x, r update (iteration count, candidates whose recursive residual is
// below rtol); 3: true-residual check of the candidates (done, or restart).
// cnt[0] = candidates, cnt[1] = active problems afterwards.
__global__ void __launch_bounds__(256) k_bpcg_book(int nprob, int mode, double rtol, double* __restrict__ sc,
                                                   int32_t* __restrict__ fl, int32_t* __restrict__ cnt) {
    __shared__ int s_cand, s_act;
    if (threadIdx.x == 0) { s_cand = 0; s_act = 0; }
    __syncthreads();
    for (int p = threadIdx.x; p < nprob; p += blockDim.x) {
        double* s = sc + (int64_t)p * kBScal;
        int32_t* f = fl + (int64_t)p * kBFlag;
        if (mode == 0) {
            f[BF_ACTIVE] = s[BS_BB] > 0.0;
            f[BF_RESTART] = 1;
            f[BF_CAND] = 0;
            f[BF_ITERS] = 0;
            s[BS_REL] = 0.0;
        } else if (mode == 1) {
            if (f[BF_ACTIVE]) { s[BS_RZ] = s[BS_RZN]; f[BF_RESTART] = 0; }
        } else if (mode == 2) {
            if (f[BF_ACTIVE]) {
                f[BF_ITERS] += 1;
                s[BS_REL] = sqrt(s[BS_RR] / s[BS_BB]);
                if (s[BS_REL] <= rtol) { f[BF_CAND] = 1; atomicAdd(&s_cand, 1); }
            }
        } else if (f[BF_ACTIVE] && f[BF_CAND]) {
            f[BF_CAND] = 0;
            s[BS_REL] = sqrt(s[BS_RRT] / s[BS_BB]);
            if (s[BS_REL] <= rtol) f[BF_ACTIVE] = 0;
            else f[BF_RESTART] = 1;
        }
        if (f[BF_ACTIVE]) atomicAdd(&s_act, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) { cnt[0] = s_cand; cnt[1] = s_act; }
}

__global__ void k_axpby(int64_t n, double a, const double* __restrict__ x, double b, double* __restrict__ y) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    y[i] = a * x[i] + b * y[i];
}

// y += sign * sum_k coef[k] * V[k*ldv + i]
__global__ void k_gmres_update(int64_t n, int k, const double* __restrict__ coef, const double* __restrict__ V,
                               int64_t ldv, double* __restrict__ y, double sign) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double t = 0.0;
    for (int j = 0; j < k; j++) t += coef[j] * V[(int64_t)j * ldv + i];
    y[i] += sign * t;
}

// partial[j * nb + blk] = sum over the block's rows of V[j] . w  (j < k)
__global__ void __launch_bounds__(256) k_gemv_t_partial(int64_t n, int k, const double* __restrict__ V,
                                                        int64_t ldv, const double* __restrict__ w,
                                                        double* __restrict__ partial) {
    __shared__ double red[32];
    for (int j = 0; j < k; j++) {
        double t = 0.0;
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
            t += V[(int64_t)j * ldv + i] * w[i];
        t = block_sum(t, red);
        if (threadIdx.x == 0) partial[(int64_t)j * gridDim.x + blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(256) k_gemv_t_final(int k, int np, const double* __restrict__ partial,
                                                      double* __restrict__ out) {
    __shared__ double red[32];
    const int j = blockIdx.x;
    if (j >= k) return;
    double t = 0.0;
    for (int i = threadIdx.x; i < np; i += blockDim.x) t += partial[(int64_t)j * np + i];
    t = block_sum(t, red);
    if (threadIdx.x == 0) out[j] = t;
}

// FP64 FMA throughput probe: 8 independent chains per thread.
// FMA throughput probe: 8 independent fma chains per thread (T = double for
// the FP64 pipe, float for the FP32 pipe)
template <typename T>
__global__ void __launch_bounds__(256) k_fma_peak(int iters, double* sink) {
    T a[8];
#pragma unroll
    for (int u = 0; u < 8; u++) a[u] = (T)(1.0 + 1e-6 * (threadIdx.x + u));
    const T b = (T)0.999999, c = (T)1e-7;
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int u = 0; u < 8; u++) a[u] = fma(a[u], b, c);
    }
    T t = 0;
#pragma unroll
    for (int u = 0; u < 8; u++) t += a[u];
    if (t == (T)12345.0) sink[0] = (double)t;  // keeps the chains alive
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

std::atomic<int64_t> g_launches{0};
inline void counted(int k = 1) { g_launches.fetch_add(k, std::memory_order_relaxed); }

}  // namespace

// Fixed device scratch of the allocation-free PCG (hs_krylov_noalloc): four
// work vectors of at most kNoAllocMaxN doubles, the dot-product partial sums
// and a few scalars.  Compiled into the library; every device that loads it
// holds the array until the process exits.
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

cudaError_t noalloc_scratch(double** ptr) {
    static std::mutex mu;
    static double* addr[kNoAllocMaxDevices] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kNoAllocMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        // the symbol names a host-side stand-in; only this call yields the
        // array's address on the current device
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        addr[dev] = static_cast<double*>(p);
    }
    *ptr = addr[dev];
    return cudaSuccess;
}

// Evaluates the Cholesky pivot helpers element by element (a self-check of
// the Newton-refined reciprocals against CUDA's own operations).
__global__ void k_eval_recip(int64_t n, const double* x, double* rs, double* rc) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double v = x[i];
    rs[i] = rsqrt_newton(v);
    rc[i] = rcp_newton(v);
}

cudaError_t launch_eval_recip(cudaStream_t st, int64_t n, const double* x, double* rs, double* rc) {
    if (n <= 0) return cudaSuccess;
    k_eval_recip<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, x, rs, rc);
    counted();
    return cudaGetLastError();
}

int64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }
void launch_count_add(int64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
cudaError_t launch_scatter_csr(cudaStream_t st, int64_t n, const int64_t* rowptr, const int32_t* col,
                               const double* val, const int32_t* dof_cluster, const int32_t* dof_local,
                               const int32_t* blk_ptr, const int32_t* blk_col, const int64_t* blk_off,
                               const int32_t* blk_ld, double* blocks) {
    if (n <= 0) return cudaSuccess;
    counted();
    k_scatter_csr<<<blocks_for(n, 256), 256, 0, st>>>(n, rowptr, col, val, dof_cluster, dof_local, blk_ptr,
                                                      blk_col, blk_off, blk_ld, blocks);
    return cudaGetLastError();
}

cudaError_t launch_check_csr(cudaStream_t st, int64_t n, int64_t nnz, const int64_t* rowptr, const int32_t* col,
                             int32_t* bad) {
    if (n < 0 || nnz < 0) return cudaErrorInvalidValue;
    const int64_t work = std::max(n, nnz);
    const unsigned nb = (unsigned)std::max<int64_t>(1, std::min<int64_t>(blocks_for(work, 256), 4 * 152));
    counted();
    k_check_csr<<<nb, 256, 0, st>>>(n, nnz, rowptr, col, bad);
    return cudaGetLastError();
}

size_t factor_smem_bytes(int smax, int wmax, int lmax, bool xsh) {
    const size_t base = sizeof(double) * ((size_t)smax * smax + 2 * (size_t)smax + (size_t)wmax + 64) +
                        sizeof(EntryMeta) * (size_t)lmax + 2 * sizeof(int64_t) * (size_t)wmax +
                        sizeof(int) * ((size_t)lmax + 2);
    // then G^-1 (doubles)
    return (base + 15) / 16 * 16 + (xsh ? sizeof(double) * (size_t)smax * smax : 0);
}

template <typename FT>
cudaError_t factor_phase_t(cudaStream_t st, const TaskDev* tasks, int t0, int ntasks, int smax, int wmax, int lmax,
                           const ListDev* lists, double* blocks, const int64_t* blk_off, const int32_t* blk_ld,
                           int32_t* cur, FT* fac, int32_t* meta, double* ws, double eps2, int32_t* status,
                           int32_t level, float* feat, const float* model) {
    // G^-1 in shared memory when it fits beside the rest
    const int use_x = factor_smem_bytes(smax, wmax, lmax, true) <= (size_t)kFactorMaxSmem;
    const size_t smem = factor_smem_bytes(smax, wmax, lmax, use_x);
    int dev = 0, sms = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    counted();
    if (ntasks <= sms) {
        e = cudaFuncSetAttribute(k_factor_phase<FT, 2 * kFactorThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        k_factor_phase<FT, 2 * kFactorThreads><<<ntasks, 2 * kFactorThreads, smem, st>>>(
            tasks, t0, lists, blocks, blk_off, blk_ld, cur, fac, meta, ws, eps2, status, level, smax, wmax, lmax, feat,
            model, use_x);
    } else {
        e = cudaFuncSetAttribute(k_factor_phase<FT, kFactorThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        k_factor_phase<FT, kFactorThreads><<<ntasks, kFactorThreads, smem, st>>>(
            tasks, t0, lists, blocks, blk_off, blk_ld, cur, fac, meta, ws, eps2, status, level, smax, wmax, lmax, feat,
            model, use_x);
    }
    return cudaGetLastError();
}

cudaError_t launch_factor_phase(cudaStream_t st, const TaskDev* tasks, int t0, int ntasks, int smax, int wmax,
                                int lmax, const ListDev* lists, double* blocks, const int64_t* blk_off,
                                const int32_t* blk_ld, int32_t* cur, void* fac, int fp32, int32_t* meta, double* ws,
                                double eps2, int32_t* status, int32_t level, float* feat, const float* model) {
    if (ntasks <= 0) return cudaSuccess;
    if (fp32)
        return factor_phase_t(st, tasks, t0, ntasks, smax, wmax, lmax, lists, blocks, blk_off, blk_ld, cur,
                              static_cast<float*>(fac), meta, ws, eps2, status, level, feat, model);
    return factor_phase_t(st, tasks, t0, ntasks, smax, wmax, lmax, lists, blocks, blk_off, blk_ld, cur,
                          static_cast<double*>(fac), meta, ws, eps2, status, level, feat, model);
}

size_t fused_smem_bytes(int smax, int wmax, int lmax, int64_t mcap) {
    return sizeof(double) * (size_t)kFusedWarps * fused_warp_doubles(smax, wmax, lmax, mcap) +
           sizeof(int) * (size_t)kFusedWarps * (lmax + 2);
}

cudaError_t launch_factor_level_fused(cudaStream_t st, const TaskDev* tasks, const int32_t* ph_task,
                                      const TargetDev* targets, const int32_t* ph_target, const ContribDev* contribs,
                                      int nph, const ListDev* lists, double* blocks, const int64_t* blk_off,
                                      const int32_t* blk_ld, int32_t* cur, void* fac, int fp32, int32_t* meta,
                                      double* ws, double eps2, int32_t* status, int32_t level, int smax, int wmax,
                                      int lmax, int64_t mcap, int max_items, unsigned* bar, float* feat,
                                      const float* model, int wait_polls, int cluster_ok) {
    if (nph <= 0) return cudaSuccess;
    const size_t smem = fused_smem_bytes(smax, wmax, lmax, mcap);
    long long wait_limit = wait_polls == 0 ? kBarrierSpins : (wait_polls < 0 ? 0LL : (long long)wait_polls);
    cudaError_t e;
    void* args[] = {&tasks,  &ph_task, &targets, &ph_target, &contribs, &nph,  &lists, &blocks,
                    &blk_off, &blk_ld, &cur,     &fac,       &meta,     &ws,   &eps2,  &status,
                    &level,  &smax,    &wmax,    &lmax,      &mcap,     &bar,  &feat,  &model, &wait_limit};
    if (wait_polls == 0 && cluster_ok) {
        // a level whose phases have few items (the caller's choice) runs in
        // one thread-block cluster of up to kClusterCtas CTAs (hardware
        // barrier between steps); a test limit on the waits (wait_polls != 0)
        // keeps the bounded grid barrier
        const void* fc = fp32 ? reinterpret_cast<const void*>(&k_factor_level_fused<float, true>)
                              : reinterpret_cast<const void*>(&k_factor_level_fused<double, true>);
        if ((e = cudaFuncSetAttribute(fc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
            return e;
        if ((e = cudaFuncSetAttribute(fc, cudaFuncAttributeNonPortableClusterSizeAllowed, 1)) != cudaSuccess)
            return e;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = kClusterCtas;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(kClusterCtas);
        cfg.blockDim = dim3(kFusedWarps * 32);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int maxc = 0;
        if ((e = cudaOccupancyMaxPotentialClusterSize(&maxc, fc, &cfg)) != cudaSuccess) return e;
        if (maxc >= kClusterCtas / 2) {
            const int csize = std::min(kClusterCtas, maxc);
            at[0].val.clusterDim.x = csize;
            cfg.gridDim = dim3(csize);
            counted();
            return cudaLaunchKernelExC(&cfg, fc, args);
        }
    }
    const void* fn = fp32 ? reinterpret_cast<const void*>(&k_factor_level_fused<float, false>)
                          : reinterpret_cast<const void*>(&k_factor_level_fused<double, false>);
    if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
        return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kFusedWarps * 32, smem)) != cudaSuccess)
        return e;
    if (per_sm <= 0) return cudaErrorInvalidConfiguration;
    // every CTA must be resident (grid barrier): at most per_sm * sms CTAs, and
    // no more than the largest phase needs
    // at least one CTA per SM (up to the largest phase's items), at most all
    // that can be resident together
    const int want = std::max(std::min(max_items, sms), (max_items + kFusedWarps - 1) / kFusedWarps);
    const int grid = std::max(1, std::min(per_sm * sms, want));
    if ((e = cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), st)) != cudaSuccess) return e;
    counted();
    return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kFusedWarps * 32), args, smem, st);
}

cudaError_t launch_schur_phase(cudaStream_t st, const TargetDev* targets, int g0, int ntargets,
                               const ContribDev* contribs, const TaskDev* tasks, const void* fac,
                               const int32_t* meta, double* blocks, const int64_t* blk_off, const int32_t* blk_ld,
                               const int32_t* cur, int fp32, int products) {
    if (ntargets <= 0) return cudaSuccess;
    counted();
    if (fp32 && products == kProductsTf32x3)
        k_schur_phase_tc<3><<<ntargets, 256, 0, st>>>(targets, g0, contribs, tasks, static_cast<const float*>(fac),
                                                      meta, blocks, blk_off, blk_ld, cur);
    else if (fp32 && products == kProductsBf16)
        k_schur_phase_bf16<<<ntargets, 256, 0, st>>>(targets, g0, contribs, tasks, static_cast<const float*>(fac),
                                                     meta, blocks, blk_off, blk_ld, cur);
    else if (fp32 && products == kProductsTf32)
        k_schur_phase_tc<1><<<ntargets, 256, 0, st>>>(targets, g0, contribs, tasks, static_cast<const float*>(fac),
                                                      meta, blocks, blk_off, blk_ld, cur);
    else if (fp32)
        k_schur_phase<float><<<ntargets, 256, 0, st>>>(targets, g0, contribs, tasks, static_cast<const float*>(fac),
                                                       meta, blocks, blk_off, blk_ld, cur);
    else
        k_schur_phase<double><<<ntargets, 256, 0, st>>>(targets, g0, contribs, tasks, static_cast<const double*>(fac),
                                                        meta, blocks, blk_off, blk_ld, cur);
    return cudaGetLastError();
}

cudaError_t launch_copy_blocks(cudaStream_t st, const CopyDev* cps, int ncps, const double* src, double* dst) {
    if (ncps <= 0) return cudaSuccess;
    counted();
    k_copy_blocks<<<ncps, 128, 0, st>>>(cps, src, dst);
    return cudaGetLastError();
}

cudaError_t launch_dense_cholesky(cudaStream_t st, int n, double* a, int32_t* status) {
    if (n <= 0) return cudaSuccess;
    counted();
    k_dense_cholesky<<<1, 1024, 0, st>>>(n, a, status);
    return cudaGetLastError();
}

// Launch on st with programmatic stream serialisation (the kernel must call
// griddep_wait() before its first global access).
template <typename... KArgs, typename... Args>
cudaError_t launch_chained(void (*k)(KArgs...), unsigned grid, unsigned block, size_t smem, cudaStream_t st,
                           Args... args) {
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, k, args...);
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_ap_fwd(cudaStream_t st, const ApTask* tasks, int t0, int ntasks, int smax,
                          const ApPull* pulls, const void* fac, int fp32, double* stage, double* y) {
    if (ntasks <= 0) return cudaSuccess;
    counted();
    // the two vectors, then (FP32 factor) one float4 per thread for the
    // row-chunk partial sums
    const size_t smem = sizeof(double) * 2 * smax + (fp32 ? sizeof(float) * 4 * kApplyThreads : 0);
    if (fp32)
        return launch_chained(k_ap_fwd<float>, ntasks, kApplyThreads, smem, st, tasks, t0, pulls,
                              static_cast<const float*>(fac), stage, y, smax);
    return launch_chained(k_ap_fwd<double>, ntasks, kApplyThreads, smem, st, tasks, t0, pulls,
                          static_cast<const double*>(fac), stage, y, smax);
}

cudaError_t launch_ap_fin(cudaStream_t st, const ApFin* fins, int nfin, const ApPull* pulls, const double* stage,
                          double* y, double* ynext, double* ytop) {
    if (nfin <= 0) return cudaSuccess;
    counted();
    return launch_chained(k_ap_fin, nfin, kApplyThreads, 0, st, fins, pulls, stage, y, ynext, ytop);
}

cudaError_t launch_ap_bwd(cudaStream_t st, const ApTask* tasks, int t0, int ntasks, int smax, int nmax,
                          const ApNb* nbs, const void* fac, int fp32, double* y) {
    if (ntasks <= 0) return cudaSuccess;
    counted();
    const size_t smem = sizeof(double) * (2 * (size_t)smax + kApplyThreads + nmax);
    if (fp32)
        return launch_chained(k_ap_bwd<float>, ntasks, kApplyThreads, smem, st, tasks, t0, nbs,
                              static_cast<const float*>(fac), y, smax, nmax);
    return launch_chained(k_ap_bwd<double>, ntasks, kApplyThreads, smem, st, tasks, t0, nbs,
                          static_cast<const double*>(fac), y, smax, nmax);
}

cudaError_t launch_ap_coarse_batch(cudaStream_t st, const ApLevel* lvl, int nlev, int ntop, const double* L,
                                   double* ytop0, double* yin0, int n, int64_t stride, double* Mc, int fp32) {
    if (n <= 0) return cudaSuccess;
    counted();
    const int threads = 256;  // 4 CTAs per SM fit in registers: one wave for ~600 columns
    const size_t smem = sizeof(double) * (kCoarseSmax + kCoarseNmax) * (threads / 32);
    cudaError_t e = fp32 ? cudaFuncSetAttribute(k_ap_coarse_batch<float>,
                                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                         : cudaFuncSetAttribute(k_ap_coarse_batch<double>,
                                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (fp32)
        k_ap_coarse_batch<float><<<n, threads, smem, st>>>(lvl, nlev, ntop, L, ytop0, yin0, n, stride, Mc);
    else
        k_ap_coarse_batch<double><<<n, threads, smem, st>>>(lvl, nlev, ntop, L, ytop0, yin0, n, stride, Mc);
    return cudaGetLastError();
}

cudaError_t launch_dense_gemv(cudaStream_t st, int n, const double* Mc, const double* x, double* y) {
    if (n <= 0) return cudaSuccess;
    counted();
    return launch_chained(k_dense_gemv, (n + 7) / 8, 256, 0, st, n, Mc, x, y);
}

cudaError_t launch_ap_coarse(cudaStream_t st, const ApLevel* lvl, int nlev, int ntop, const double* L, double* ytop,
                             int fp32) {
    if (nlev <= 0 && ntop <= 0) return cudaSuccess;
    counted();
    const size_t smem = sizeof(double) * (kCoarseSmax + kCoarseNmax) * (kCoarseThreads / 32);
    cudaError_t e = fp32 ? cudaFuncSetAttribute(k_ap_coarse<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                (int)smem)
                         : cudaFuncSetAttribute(k_ap_coarse<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                (int)smem);
    if (e != cudaSuccess) return e;
    if (fp32) return launch_chained(k_ap_coarse<float>, 1, kCoarseThreads, smem, st, lvl, nlev, ntop, L, ytop);
    return launch_chained(k_ap_coarse<double>, 1, kCoarseThreads, smem, st, lvl, nlev, ntop, L, ytop);
}

cudaError_t launch_vcopy(cudaStream_t st, const VCopyDev* cps, int ncps, const double* src, double* dst,
                         int reverse, const double* ytop) {
    if (ncps <= 0) return cudaSuccess;
    counted();
    return launch_chained(k_vcopy, blocks_for(ncps, 8), 256, 0, st, cps, ncps, src, dst, reverse, ytop);
}

cudaError_t launch_tops_cholesky(cudaStream_t st, const TopDev* tops, int ntops, int32_t* status) {
    if (ntops <= 0) return cudaSuccess;
    counted();
    k_tops_cholesky<<<ntops, 256, 0, st>>>(tops, status);
    return cudaGetLastError();
}

cudaError_t launch_tops_solve(cudaStream_t st, const TopDev* tops, int ntops, double* ytop) {
    if (ntops <= 0) return cudaSuccess;
    counted();
    return launch_chained(k_tops_solve, ntops, 256, 0, st, tops, ytop);
}

cudaError_t launch_top_solve(cudaStream_t st, int n, const double* L, double* y) {
    if (n <= 0) return cudaSuccess;
    counted();
    k_top_solve<<<1, 1024, 0, st>>>(n, L, y);
    return cudaGetLastError();
}

cudaError_t launch_permute(cudaStream_t st, int64_t n, const int32_t* perm, const double* src, double* dst,
                           int inverse) {
    if (n <= 0) return cudaSuccess;
    counted();
    k_permute<<<blocks_for(n, 256), 256, 0, st>>>(n, perm, src, dst, inverse);
    return cudaGetLastError();
}

cudaError_t launch_spmv(cudaStream_t st, int64_t n, const int64_t* rowptr, const int32_t* col, const double* val,
                        const double* x, double* y) {
    if (n <= 0) return cudaSuccess;
    counted();
    k_spmv<<<blocks_for(n, 256), 256, 0, st>>>(n, rowptr, col, val, x, y);
    return cudaGetLastError();
}

cudaError_t launch_dot(cudaStream_t st, int64_t n, const double* a, const double* b, double* partial, double* out) {
    counted();
    k_dot_partial<<<kDotParts, 256, 0, st>>>(n, a, b, partial);
    counted();
    k_sum_partials<<<1, 1024, 0, st>>>(partial, kDotParts, out);
    return cudaGetLastError();
}

// grid of the fused PCG kernels: one thread per entry up to kDotParts blocks
inline unsigned fused_grid(int64_t n) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(blocks_for(n, 256), kDotParts));
}

cudaError_t launch_spmv_dot(cudaStream_t st, int64_t n, const int64_t* rowptr, const int32_t* col, const double* val,
                            const double* x, double* y, double* partial, unsigned* count, double* out) {
    counted();
    k_spmv_dot<<<fused_grid(n), 256, 0, st>>>(n, rowptr, col, val, x, y, partial, count, out);
    return cudaGetLastError();
}

cudaError_t launch_pcg_xr_dot(cudaStream_t st, int64_t n, const double* rz, const double* pq, const double* p,
                              const double* q, double* x, double* r, double* partial, unsigned* count, double* out) {
    counted();
    k_pcg_xr_dot<<<fused_grid(n), 256, 0, st>>>(n, rz, pq, p, q, x, r, partial, count, out);
    return cudaGetLastError();
}

cudaError_t launch_dot_fused(cudaStream_t st, int64_t n, const double* a, const double* b, double* partial,
                             unsigned* count, double* out) {
    counted();
    k_dot_fused<<<fused_grid(n), 256, 0, st>>>(n, a, b, partial, count, out);
    return cudaGetLastError();
}

cudaError_t launch_pcg_update_xr(cudaStream_t st, int64_t n, const double* rz, const double* pq, const double* p,
                                 const double* q, double* x, double* r) {
    counted();
    k_pcg_xr<<<blocks_for(n, 256), 256, 0, st>>>(n, rz, pq, p, q, x, r);
    return cudaGetLastError();
}

cudaError_t launch_pcg_update_p(cudaStream_t st, int64_t n, const double* rz_new, const double* rz_old,
                                const double* z, double* p) {
    counted();
    k_pcg_p<<<blocks_for(n, 256), 256, 0, st>>>(n, rz_new, rz_old, z, p);
    return cudaGetLastError();
}

cudaError_t launch_seg_dot(cudaStream_t st, int nprob, const int64_t* pp, const double* a, const double* b,
                           double* sc, int slot) {
    if (nprob <= 0) return cudaSuccess;
    counted();
    k_seg_dot<<<nprob, 256, 0, st>>>(pp, a, b, sc, slot);
    return cudaGetLastError();
}

cudaError_t launch_bpcg_vec(cudaStream_t st, int op, int nprob, int64_t maxlen, const int64_t* pp, const double* sc,
                            const int32_t* fl, const double* a, const double* b, double* c, double* d) {
    if (nprob <= 0 || maxlen <= 0) return cudaSuccess;
    if (nprob > 65535) return cudaErrorInvalidValue;
    counted();
    const dim3 grid((unsigned)blocks_for(maxlen, 256), (unsigned)nprob);
    if (op == 0) k_bpcg_xr<<<grid, 256, 0, st>>>(pp, sc, fl, a, b, c, d);
    else if (op == 1) k_bpcg_p<<<grid, 256, 0, st>>>(pp, sc, fl, a, c);
    else k_bpcg_restart_copy<<<grid, 256, 0, st>>>(pp, fl, a, c);
    return cudaGetLastError();
}

cudaError_t launch_bpcg_book(cudaStream_t st, int nprob, int mode, double rtol, double* sc, int32_t* fl,
                             int32_t* cnt) {
    counted();
    k_bpcg_book<<<1, 256, 0, st>>>(nprob, mode, rtol, sc, fl, cnt);
    return cudaGetLastError();
}

cudaError_t launch_axpby(cudaStream_t st, int64_t n, double a, const double* x, double b, double* y) {
    counted();
    k_axpby<<<blocks_for(n, 256), 256, 0, st>>>(n, a, x, b, y);
    return cudaGetLastError();
}

cudaError_t launch_gmres_update(cudaStream_t st, int64_t n, int k, const double* coef, const double* V,
                                int64_t ldv, double* y, double sign) {
    if (k <= 0) return cudaSuccess;
    counted();
    k_gmres_update<<<blocks_for(n, 256), 256, 0, st>>>(n, k, coef, V, ldv, y, sign);
    return cudaGetLastError();
}

cudaError_t launch_fp64_peak(cudaStream_t st, int nblocks, int iters, double* sink) {
    counted();
    k_fma_peak<double><<<nblocks, 256, 0, st>>>(iters, sink);
    return cudaGetLastError();
}

cudaError_t launch_fp32_peak(cudaStream_t st, int nblocks, int iters, double* sink) {
    counted();
    k_fma_peak<float><<<nblocks, 256, 0, st>>>(iters, sink);
    return cudaGetLastError();
}

cudaError_t launch_gemv_t(cudaStream_t st, int64_t n, int k, const double* V, int64_t ldv, const double* w,
                          double* partial, double* out) {
    if (k <= 0) return cudaSuccess;
    const int nb = 256;
    counted();
    k_gemv_t_partial<<<nb, 256, 0, st>>>(n, k, V, ldv, w, partial);
    counted();
    k_gemv_t_final<<<k, 256, 0, st>>>(k, nb, partial, out);
    return cudaGetLastError();
}

}  // namespace hs
