// hs_kernels.cu -- sm_103a kernels of the hierarchical solver.
//
// Factorization (Algorithm 1), per phase of independent clusters:
//   k_factor_phase : one CTA per cluster: Cholesky of A_ss (Sec. 2), scaling
//                    G^-1 [A_sn A_sw] (Eq. scaling), column-pivoted QR of the
//                    scaled fill block with every reflector applied to the
//                    whole row (Eq. offdiag_new, Eq. sparse), write-back of the
//                    coarse row (Eq. perm) and of the factor {G, U, C, r}.
//   k_schur_phase  : one CTA per target block: X_nn = A_nn - C^T C (Eq. elim),
//                    contributions summed in ascending cluster order.
// Solve (Algorithm 2): k_apply_fwd / k_apply_bwd per phase with the explicit
// per-cluster operator W = U^T G^-1, k_apply_fin / k_vcopy between levels,
// k_top_solve for the dense top.
// Krylov: CSR SpMV, deterministic two-stage dot products, vector updates.
//
// Decisions that must agree with any other implementation of the method:
// rank = smallest k with sum of squared trailing column norms <= eps^2;
// pivot = lowest unpivoted column index with squared norm >= (1 - 1e-10) *
// the largest; Householder beta = -sign(alpha) * norm, v_k = 1,
// tau = (beta - alpha) / beta.
#include <atomic>
#include <cfloat>
#include <climits>
#include <cstdint>
#include <mutex>

#include "hs_internal.h"

namespace hs {

namespace {

constexpr double kPivotTie = 1e-10;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
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

// ---------------------------------------------------------------------------
// Factor one phase: one CTA per cluster.
// Shared memory: G (s*s) | rdiag (s) | v (s) | cn (wmax) | red (64) | ioff (lmax+1 ints) | flags
// ---------------------------------------------------------------------------
constexpr int kFactorThreads = 256;

__global__ void __launch_bounds__(kFactorThreads)
k_factor_phase(const TaskDev* __restrict__ tasks, int t0, const ListDev* __restrict__ lists,
               double* __restrict__ blocks, const int64_t* __restrict__ blk_off,
               const int32_t* __restrict__ blk_ld, int32_t* __restrict__ cur, double* __restrict__ fac,
               int32_t* __restrict__ meta, double* __restrict__ ws, double eps2, int32_t* status,
               int32_t level, int smax, int wmax) {
    extern __shared__ double sm[];
    const TaskDev T = tasks[t0 + blockIdx.x];
    const int s = T.s, tid = threadIdx.x, NT = blockDim.x;
    const int L = T.nn + T.nw;
    double* G = sm;
    double* rdiag = G + (size_t)smax * smax;
    double* v = rdiag + smax;
    double* cn = v + smax;
    double* red = cn + wmax;
    int* ioff = reinterpret_cast<int*>(red + 64);
    __shared__ int s_flag;
    __shared__ double s_hh[3];

    // column offsets of the row blocks (compact, current widths)
    if (tid == 0) {
        int o = 0;
        for (int e = 0; e < L; e++) {
            ioff[e] = o;
            o += cur[lists[T.list + e].q];
        }
        ioff[L] = o;
        s_flag = 0;
    }
    // A_ss -> shared memory
    {
        const double* A = blocks + blk_off[T.diag_blk];
        const int ld = blk_ld[T.diag_blk];
        for (int idx = tid; idx < s * s; idx += NT) G[idx] = A[(int64_t)(idx / s) * ld + idx % s];
    }
    __syncthreads();
    const int W = ioff[L], ncols = ioff[T.nn], Wn = W - ncols;

    // Cholesky A_ss = G G^T (right-looking, in shared memory)
    for (int j = 0; j < s; j++) {
        if (tid == 0) {
            const double d = G[j * s + j];
            if (!(d > 0.0)) {
                s_flag = 1;
            } else {
                const double g = sqrt(d);
                G[j * s + j] = g;
                rdiag[j] = 1.0 / g;
            }
        }
        __syncthreads();
        if (s_flag) {
            if (tid == 0 && atomicCAS(status, 0, ST_NOT_SPD) == 0) {
                status[1] = level;
                status[2] = T.c;
            }
            return;
        }
        const double rj = rdiag[j];
        for (int i = j + 1 + tid; i < s; i += NT) G[i * s + j] *= rj;
        __syncthreads();
        const int m = s - j - 1;
        for (int idx = tid; idx < m * m; idx += NT) {
            const int i = j + 1 + idx / m, k = j + 1 + idx % m;
            if (k <= i) G[i * s + k] -= G[i * s + j] * G[k * s + j];
        }
        __syncthreads();
    }
    for (int idx = tid; idx < s * s; idx += NT)
        if (idx % s > idx / s) G[idx] = 0.0;
    __syncthreads();

    // gather the block row [A_sn | A_sw | I] into the workspace (row-major, ld Wt);
    // the identity columns come out as W = U^T G^-1, the solve-phase operator
    const int Wt = W + s;
    double* M = ws + T.m_off;
    for (int e = 0; e < L; e++) {
        const ListDev le = lists[T.list + e];
        const int wq = ioff[e + 1] - ioff[e];
        const double* src = blocks + blk_off[le.blk_cq];
        const int ld = blk_ld[le.blk_cq];
        const int o = ioff[e];
        for (int idx = tid; idx < s * wq; idx += NT) {
            const int i = idx / wq, j = idx % wq;
            M[(int64_t)i * Wt + o + j] = src[(int64_t)i * ld + j];
        }
    }
    for (int idx = tid; idx < s * s; idx += NT) {
        const int i = idx / s, j = idx % s;
        M[(int64_t)i * Wt + W + j] = (i == j) ? 1.0 : 0.0;
    }
    __syncthreads();

    // scaling: M <- G^-1 M (forward substitution, one thread per column;
    // identity column j is zero above row j)
    for (int j = tid; j < Wt; j += NT) {
        const int i0 = (j >= W) ? j - W : 0;
        for (int i = i0; i < s; i++) {
            double acc = M[(int64_t)i * Wt + j];
            for (int k = i0; k < i; k++) acc -= G[i * s + k] * M[(int64_t)k * Wt + j];
            M[(int64_t)i * Wt + j] = acc * rdiag[i];
        }
    }
    __syncthreads();

    // column-pivoted QR of the fill columns, reflectors applied to the whole row
    for (int j = tid; j < Wn; j += NT) {
        double c = 0.0;
        for (int i = 0; i < s; i++) {
            const double x = M[(int64_t)i * Wt + ncols + j];
            c += x * x;
        }
        cn[j] = c;
    }
    __syncthreads();
    int k = 0;
    while (k < s) {
        double lt = 0.0, lm = 0.0;
        for (int j = tid; j < Wn; j += NT) {
            const double c = cn[j];
            if (c >= 0.0) {
                lt += c;
                lm = fmax(lm, c);
            }
        }
        const double total = block_sum(lt, red);
        const double cmax = block_max(lm, red);
        if (total <= eps2) break;
        const double thr = (1.0 - kPivotTie) * cmax;
        int lp = INT_MAX;
        for (int j = tid; j < Wn; j += NT)
            if (cn[j] >= 0.0 && cn[j] >= thr) {
                lp = j;
                break;  // lowest of this thread's columns
            }
        const int p = block_min_int(lp, reinterpret_cast<int*>(red));
        const int pc = ncols + p;
        double ls = 0.0;
        for (int i = k + 1 + tid; i < s; i += NT) {
            const double x = M[(int64_t)i * Wt + pc];
            ls += x * x;
        }
        const double sig = block_sum(ls, red);
        if (tid == 0) {
            const double alpha = M[(int64_t)k * Wt + pc];
            const double nrm = sqrt(alpha * alpha + sig);
            const double beta = alpha >= 0.0 ? -nrm : nrm;
            s_hh[0] = beta;
            s_hh[1] = (beta - alpha) / beta;
            s_hh[2] = 1.0 / (alpha - beta);
            cn[p] = -1.0;
        }
        __syncthreads();
        const double beta = s_hh[0], tau = s_hh[1], scal = s_hh[2];
        for (int i = tid; i < s; i += NT) {
            double vi = 0.0;
            if (i == k) vi = 1.0;
            else if (i > k) vi = M[(int64_t)i * Wt + pc] * scal;
            v[i] = vi;
        }
        __syncthreads();
        for (int i = k + tid; i < s; i += NT) M[(int64_t)i * Wt + pc] = (i == k) ? beta : 0.0;
        for (int j = tid; j < Wt; j += NT) {
            if (j == pc) continue;
            const bool cand = (j >= ncols && j < W);
            if (cand && cn[j - ncols] < 0.0) continue;  // pivoted: zero below its row
            double t = M[(int64_t)k * Wt + j];
            for (int i = k + 1; i < s; i++) t += v[i] * M[(int64_t)i * Wt + j];
            t *= tau;
            M[(int64_t)k * Wt + j] -= t;
            double c = 0.0;
            for (int i = k + 1; i < s; i++) {
                const double x = M[(int64_t)i * Wt + j] - t * v[i];
                M[(int64_t)i * Wt + j] = x;
                if (cand) c += x * x;
            }
            if (cand) cn[j - ncols] = c;
        }
        __syncthreads();
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
        double* Wf = fac + T.w_off;
        for (int idx = tid; idx < s * s; idx += NT) Wf[idx] = M[(int64_t)(idx / s) * Wt + W + idx % s];
        double* Cf = fac + T.c_off;
        const int f = s - r;
        for (int idx = tid; idx < f * ncols; idx += NT) {
            const int i = idx / ncols, j = idx % ncols;
            Cf[(int64_t)i * T.ncap + j] = M[(int64_t)(r + i) * Wt + j];
        }
    }
    // write back the coarse row (identity diagonal, U^T G^-1 A_sn, V1^T)
    if (T.nw > 0 && r > 0) {
        for (int e = 0; e < L; e++) {
            const ListDev le = lists[T.list + e];
            const int wq = ioff[e + 1] - ioff[e], o = ioff[e];
            double* dcq = blocks + blk_off[le.blk_cq];
            const int ldcq = blk_ld[le.blk_cq];
            double* dqc = blocks + blk_off[le.blk_qc];
            const int ldqc = blk_ld[le.blk_qc];
            for (int idx = tid; idx < r * wq; idx += NT) {
                const int i = idx / wq, j = idx % wq;
                const double x = M[(int64_t)i * Wt + o + j];
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

// ---------------------------------------------------------------------------
// Schur update of one phase: one CTA per target block (p, q), p <= q.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
k_schur_phase(const TargetDev* __restrict__ targets, int g0, const ContribDev* __restrict__ contribs,
              const TaskDev* __restrict__ tasks, const double* __restrict__ fac,
              const int32_t* __restrict__ meta, double* __restrict__ blocks,
              const int64_t* __restrict__ blk_off, const int32_t* __restrict__ blk_ld,
              const int32_t* __restrict__ cur) {
    const TargetDev g = targets[g0 + blockIdx.x];
    const int mp = cur[g.p], mq = cur[g.q];
    double* A = blocks + blk_off[g.blk_pq];
    const int lda = blk_ld[g.blk_pq];
    double* At = blocks + blk_off[g.blk_qp];
    const int ldt = blk_ld[g.blk_qp];
    for (int idx = threadIdx.x; idx < mp * mq; idx += blockDim.x) {
        const int i = idx / mq, j = idx % mq;
        double acc = A[(int64_t)i * lda + j];
        for (int c = g.c_begin; c < g.c_end; c++) {
            const ContribDev cb = contribs[c];
            const TaskDev T = tasks[cb.task];
            const int32_t* mt = meta + T.meta;
            const int r = mt[0], f = T.s - r;
            const int op = mt[1 + 2 * cb.kp], oq = mt[1 + 2 * cb.kq];
            const double* C = fac + T.c_off;
            double sub = 0.0;
            for (int k = 0; k < f; k++) sub += C[(int64_t)k * T.ncap + op + i] * C[(int64_t)k * T.ncap + oq + j];
            acc -= sub;
        }
        A[(int64_t)i * lda + j] = acc;
        if (g.p != g.q) At[(int64_t)j * ldt + i] = acc;
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

// ----- solve phase, fine levels: one CTA per task, one launch per phase -----

// Forward step of one phase:
//   y_c -= staged updates of the tasks of earlier phases that have c as a
//          neighbour (ascending task order);
//   y_c <- W_c y_c with W_c = U^T G^-1;
//   stage d_c = C_c^T y_c(r:), the update of every neighbour of c (Eq. elim
//          applied to the vector), consumed by later tasks or at level end.
__global__ void __launch_bounds__(kApplyThreads)
k_ap_fwd(const ApTask* __restrict__ tasks, int t0, const ApPull* __restrict__ pulls,
         const double* __restrict__ fac, double* __restrict__ stage, double* __restrict__ y, int smax) {
    extern __shared__ double sh[];
    double* ys = sh;
    double* yn = sh + smax;
    const ApTask T = tasks[t0 + blockIdx.x];
    const int s = T.s, tid = threadIdx.x, NT = blockDim.x;
    double* yg = y + T.y;
    for (int j = tid; j < s; j += NT) {
        double v = yg[j];
        for (int pi = T.pull0; pi < T.pull1; pi++) v -= stage[pulls[pi].off + j];
        ys[j] = v;
    }
    __syncthreads();
    const double* Wm = fac + T.w;
    const int lane = tid & 31, wid = tid >> 5, nwarp = NT >> 5;
    for (int i0 = 4 * wid; i0 < s; i0 += 4 * nwarp) {
        double a[4] = {0.0, 0.0, 0.0, 0.0};
        for (int j = lane; j < s; j += 32) {
            const double yj = ys[j];
#pragma unroll
            for (int u = 0; u < 4; u++)
                if (i0 + u < s) a[u] += Wm[(int64_t)(i0 + u) * s + j] * yj;
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const double t = warp_sum(a[u]);
            if (lane == 0 && i0 + u < s) yn[i0 + u] = t;
        }
    }
    __syncthreads();
    for (int j = tid; j < s; j += NT) yg[j] = yn[j];
    const int f = s - T.r;
    const double* C = fac + T.cm;
    const double* yf = yn + T.r;
    for (int j = tid; j < T.ncols; j += NT) {
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
        const double* cj = C + j;
        int i = 0;
        for (; i + 3 < f; i += 4) {
            a0 += cj[(int64_t)i * T.ncap] * yf[i];
            a1 += cj[(int64_t)(i + 1) * T.ncap] * yf[i + 1];
            a2 += cj[(int64_t)(i + 2) * T.ncap] * yf[i + 2];
            a3 += cj[(int64_t)(i + 3) * T.ncap] * yf[i + 3];
        }
        for (; i < f; i++) a0 += cj[(int64_t)i * T.ncap] * yf[i];
        stage[T.stg + j] = (a0 + a1) + (a2 + a3);
    }
}

// End of a level's forward solve, one CTA per cluster with a coarse part.
__global__ void __launch_bounds__(kApplyThreads)
k_ap_fin(const ApFin* __restrict__ fins, const ApPull* __restrict__ pulls, const double* __restrict__ stage,
         double* __restrict__ y, double* __restrict__ ynext) {
    const ApFin F = fins[blockIdx.x];
    for (int j = threadIdx.x; j < F.len; j += blockDim.x) {
        double v = y[F.y + j];
        for (int pi = F.pull0; pi < F.pull1; pi++) v -= stage[pulls[pi].off + j];
        y[F.y + j] = v;
        ynext[F.dst + j] = v;
    }
}

// Backward step of one phase: x_c(r:) -= C x_n, then x_c <- W_c^T x_c.
__global__ void __launch_bounds__(kApplyThreads)
k_ap_bwd(const ApTask* __restrict__ tasks, int t0, const ApNb* __restrict__ nbs, const double* __restrict__ fac,
         double* __restrict__ y, int smax) {
    extern __shared__ double sh[];
    double* xs = sh;
    double* part = sh + smax;
    double* xn = part + blockDim.x;
    const ApTask T = tasks[t0 + blockIdx.x];
    const int s = T.s, r = T.r, f = s - r, tid = threadIdx.x, NT = blockDim.x;
    double* yg = y + T.y;
    for (int i = tid; i < s; i += NT) xs[i] = yg[i];
    for (int e = T.nb0; e < T.nb1; e++) {
        const ApNb nb = nbs[e];
        for (int j = tid; j < nb.m; j += NT) xn[nb.col + j] = y[nb.y + j];
    }
    __syncthreads();
    const double* C = fac + T.cm;
    const int lane = tid & 31, wid = tid >> 5, nwarp = NT >> 5;
    for (int i0 = 2 * wid; i0 < f; i0 += 2 * nwarp) {
        double a0 = 0.0, a1 = 0.0;
        const bool two = i0 + 1 < f;
        for (int j = lane; j < T.ncols; j += 32) {
            const double xj = xn[j];
            a0 += C[(int64_t)i0 * T.ncap + j] * xj;
            if (two) a1 += C[(int64_t)(i0 + 1) * T.ncap + j] * xj;
        }
        a0 = warp_sum(a0);
        a1 = warp_sum(a1);
        if (lane == 0) {
            xs[r + i0] -= a0;
            if (two) xs[r + i0 + 1] -= a1;
        }
    }
    __syncthreads();
    const double* Wm = fac + T.w;
    if (s >= NT) {
        for (int jj = tid; jj < s; jj += NT) {
            double a0 = 0.0, a1 = 0.0;
            int i = 0;
            for (; i + 1 < s; i += 2) {
                a0 += Wm[(int64_t)i * s + jj] * xs[i];
                a1 += Wm[(int64_t)(i + 1) * s + jj] * xs[i + 1];
            }
            if (i < s) a0 += Wm[(int64_t)i * s + jj] * xs[i];
            yg[jj] = a0 + a1;
        }
        return;
    }
    const int G = NT / s, g = tid / s, j = tid % s;
    double a0 = 0.0, a1 = 0.0;
    if (g < G) {
        int i = g;
        for (; i + G < s; i += 2 * G) {
            a0 += Wm[(int64_t)i * s + j] * xs[i];
            a1 += Wm[(int64_t)(i + G) * s + j] * xs[i + G];
        }
        if (i < s) a0 += Wm[(int64_t)i * s + j] * xs[i];
    }
    part[tid] = a0 + a1;
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

__device__ void group_fwd(bool act, const ApTask& T, int gl, int gs, const ApPull* __restrict__ pulls,
                          const double* __restrict__ fac, double* __restrict__ stage, double* __restrict__ y,
                          double* ys, double* yn) {
    const int s = act ? T.s : 0;
    for (int j = gl; j < s; j += gs) {
        double v = y[T.y + j];
        for (int pi = T.pull0; pi < T.pull1; pi++) v -= stage[pulls[pi].off + j];
        ys[j] = v;
    }
    __syncwarp();
    if (act) {
        const double* Wm = fac + T.w;
        for (int i = gl; i < s; i += gs) {
            const double* wi = Wm + (int64_t)i * s;
            double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
            int j = 0;
            for (; j + 3 < s; j += 4) {
                a0 += wi[j] * ys[j];
                a1 += wi[j + 1] * ys[j + 1];
                a2 += wi[j + 2] * ys[j + 2];
                a3 += wi[j + 3] * ys[j + 3];
            }
            for (; j < s; j++) a0 += wi[j] * ys[j];
            yn[i] = (a0 + a1) + (a2 + a3);
        }
    }
    __syncwarp();
    if (act) {
        for (int j = gl; j < s; j += gs) y[T.y + j] = yn[j];
        const int f = s - T.r;
        const double* C = fac + T.cm;
        const double* yf = yn + T.r;
        for (int j = gl; j < T.ncols; j += gs) {
            const double* cj = C + j;
            double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
            int i = 0;
            for (; i + 3 < f; i += 4) {
                a0 += cj[(int64_t)i * T.ncap] * yf[i];
                a1 += cj[(int64_t)(i + 1) * T.ncap] * yf[i + 1];
                a2 += cj[(int64_t)(i + 2) * T.ncap] * yf[i + 2];
                a3 += cj[(int64_t)(i + 3) * T.ncap] * yf[i + 3];
            }
            for (; i < f; i++) a0 += cj[(int64_t)i * T.ncap] * yf[i];
            stage[T.stg + j] = (a0 + a1) + (a2 + a3);
        }
    }
    __syncwarp();
}

__device__ void group_bwd(bool act, const ApTask& T, int gl, int gs, const ApNb* __restrict__ nbs,
                          const double* __restrict__ fac, double* __restrict__ y, double* xs, double* xn) {
    const int s = act ? T.s : 0, r = T.r, f = s - r;
    for (int i = gl; i < s; i += gs) xs[i] = y[T.y + i];
    const int ncols = act ? T.ncols : 0;
    for (int e = act ? T.nb0 : 0; e < (act ? T.nb1 : 0); e++) {
        const ApNb nb = nbs[e];
        for (int j = gl; j < nb.m; j += gs) xn[nb.col + j] = y[nb.y + j];
    }
    __syncwarp();
    if (act) {
        const double* C = fac + T.cm;
        for (int i = gl; i < f; i += gs) {
            const double* ci = C + (int64_t)i * T.ncap;
            double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
            int j = 0;
            for (; j + 3 < ncols; j += 4) {
                a0 += ci[j] * xn[j];
                a1 += ci[j + 1] * xn[j + 1];
                a2 += ci[j + 2] * xn[j + 2];
                a3 += ci[j + 3] * xn[j + 3];
            }
            for (; j < ncols; j++) a0 += ci[j] * xn[j];
            xs[r + i] -= (a0 + a1) + (a2 + a3);
        }
    }
    __syncwarp();
    if (act) {
        const double* Wm = fac + T.w;
        for (int j = gl; j < s; j += gs) {
            double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
            int i = 0;
            for (; i + 3 < s; i += 4) {
                a0 += Wm[(int64_t)i * s + j] * xs[i];
                a1 += Wm[(int64_t)(i + 1) * s + j] * xs[i + 1];
                a2 += Wm[(int64_t)(i + 2) * s + j] * xs[i + 2];
                a3 += Wm[(int64_t)(i + 3) * s + j] * xs[i + 3];
            }
            for (; i < s; i++) a0 += Wm[(int64_t)i * s + j] * xs[i];
            y[T.y + j] = (a0 + a1) + (a2 + a3);
        }
    }
    __syncwarp();
}

// Forward over the coarse levels, the dense top (L^-T L^-1), then backward,
// with __syncthreads between stages instead of kernel boundaries.  `off` is
// added to every level vector, stage and top-vector address (a private
// workspace per CTA when the chain is run on many right-hand sides at once).
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
            for (int t = b + wid; t < e; t += nwarp) group_fwd(true, V.tasks[t], lane, 32, V.pulls, V.fac, stg, yv, ys, yn);
            __syncthreads();
        }
        for (int k = wid; k < V.nfin; k += nwarp) {
            const ApFin F = V.fins[k];
            for (int j = lane; j < F.len; j += 32) {
                double v = yv[F.y + j];
                for (int pi = F.pull0; pi < F.pull1; pi++) v -= stg[V.pulls[pi].off + j];
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
            for (int t = b + wid; t < e; t += nwarp) group_bwd(true, V.tasks[t], lane, 32, V.nbs, V.fac, yv, xs, xn);
            __syncthreads();
        }
    }
}

__global__ void __launch_bounds__(kCoarseThreads)
k_ap_coarse(const ApLevel* __restrict__ lvl, int nlev, int ntop, const double* __restrict__ Ltop,
            double* __restrict__ ytop) {
    coarse_chain(lvl, nlev, ntop, Ltop, ytop, 0);
}

// Explicit coarse operator: CTA j runs the coarse chain on the unit vector e_j
// in its own workspace (stride doubles apart) and writes the result as row j
// of Mc (n x n; symmetric up to rounding).  yin0 is CTA 0's input vector.
__global__ void __launch_bounds__(kCoarseThreads)
k_ap_coarse_batch(const ApLevel* __restrict__ lvl, int nlev, int ntop, const double* __restrict__ Ltop,
                  double* __restrict__ ytop, double* __restrict__ yin0, int n, int64_t stride,
                  double* __restrict__ Mc) {
    const int64_t off = (int64_t)blockIdx.x * stride;
    double* yin = yin0 + off;
    for (int i = threadIdx.x; i < n; i += blockDim.x) yin[i] = (i == (int)blockIdx.x) ? 1.0 : 0.0;
    __syncthreads();
    coarse_chain(lvl, nlev, ntop, Ltop, ytop, off);
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) Mc[(int64_t)blockIdx.x * n + i] = yin[i];
}

// y = Mc x (n x n, row-major): one warp per row, lanes over columns.
__global__ void __launch_bounds__(256) k_dense_gemv(int n, const double* __restrict__ Mc,
                                                    const double* __restrict__ x, double* __restrict__ y) {
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

__global__ void k_vcopy(const VCopyDev* __restrict__ cps, int ncps, const double* __restrict__ src,
                        double* __restrict__ dst, int reverse) {
    const int c = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (c >= ncps) return;
    const VCopyDev v = cps[c];
    for (int i = threadIdx.x & 31; i < v.len; i += 32) {
        if (reverse) dst[v.src + i] = src[v.dst + i];
        else dst[v.dst + i] = src[v.src + i];
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
__global__ void __launch_bounds__(256) k_fp64_peak(int iters, double* sink) {
    double a[8];
#pragma unroll
    for (int u = 0; u < 8; u++) a[u] = 1.0 + 1e-9 * (threadIdx.x + u);
    const double b = 0.999999999, c = 1e-12;
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int u = 0; u < 8; u++) a[u] = fma(a[u], b, c);
    }
    double t = 0.0;
#pragma unroll
    for (int u = 0; u < 8; u++) t += a[u];
    if (t == 12345.0) sink[0] = t;  // keeps the chains alive
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

size_t factor_smem_bytes(int smax, int wmax, int lmax) {
    return sizeof(double) * ((size_t)smax * smax + 2 * (size_t)smax + (size_t)wmax + 64) +
           sizeof(int) * ((size_t)lmax + 1);
}

cudaError_t launch_factor_phase(cudaStream_t st, const TaskDev* tasks, int t0, int ntasks, int smax, int wmax,
                                int lmax, const ListDev* lists, double* blocks, const int64_t* blk_off,
                                const int32_t* blk_ld, int32_t* cur, double* fac, int32_t* meta, double* ws,
                                double eps2, int32_t* status, int32_t level) {
    if (ntasks <= 0) return cudaSuccess;
    const size_t smem = factor_smem_bytes(smax, wmax, lmax);
    cudaError_t e = cudaFuncSetAttribute(k_factor_phase, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    counted();
    k_factor_phase<<<ntasks, kFactorThreads, smem, st>>>(tasks, t0, lists, blocks, blk_off, blk_ld, cur, fac, meta,
                                                         ws, eps2, status, level, smax, wmax);
    return cudaGetLastError();
}

cudaError_t launch_schur_phase(cudaStream_t st, const TargetDev* targets, int g0, int ntargets,
                               const ContribDev* contribs, const TaskDev* tasks, const double* fac,
                               const int32_t* meta, double* blocks, const int64_t* blk_off, const int32_t* blk_ld,
                               const int32_t* cur, int precision) {
    (void)precision;
    if (ntargets <= 0) return cudaSuccess;
    counted();
    k_schur_phase<<<ntargets, 256, 0, st>>>(targets, g0, contribs, tasks, fac, meta, blocks, blk_off, blk_ld, cur);
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

cudaError_t launch_ap_fwd(cudaStream_t st, const ApTask* tasks, int t0, int ntasks, int smax,
                          const ApPull* pulls, const double* fac, double* stage, double* y) {
    if (ntasks <= 0) return cudaSuccess;
    counted();
    k_ap_fwd<<<ntasks, kApplyThreads, sizeof(double) * 2 * smax, st>>>(tasks, t0, pulls, fac, stage, y, smax);
    return cudaGetLastError();
}

cudaError_t launch_ap_fin(cudaStream_t st, const ApFin* fins, int nfin, const ApPull* pulls, const double* stage,
                          double* y, double* ynext) {
    if (nfin <= 0) return cudaSuccess;
    counted();
    k_ap_fin<<<nfin, kApplyThreads, 0, st>>>(fins, pulls, stage, y, ynext);
    return cudaGetLastError();
}

cudaError_t launch_ap_bwd(cudaStream_t st, const ApTask* tasks, int t0, int ntasks, int smax, int nmax,
                          const ApNb* nbs, const double* fac, double* y) {
    if (ntasks <= 0) return cudaSuccess;
    counted();
    k_ap_bwd<<<ntasks, kApplyThreads, sizeof(double) * (smax + kApplyThreads + nmax), st>>>(tasks, t0, nbs, fac, y,
                                                                                            smax);
    return cudaGetLastError();
}

cudaError_t launch_ap_coarse_batch(cudaStream_t st, const ApLevel* lvl, int nlev, int ntop, const double* L,
                                   double* ytop0, double* yin0, int n, int64_t stride, double* Mc) {
    if (n <= 0) return cudaSuccess;
    counted();
    const int threads = 256;
    const size_t smem = sizeof(double) * (kCoarseSmax + kCoarseNmax) * (threads / 32);
    k_ap_coarse_batch<<<n, threads, smem, st>>>(lvl, nlev, ntop, L, ytop0, yin0, n, stride, Mc);
    return cudaGetLastError();
}

cudaError_t launch_dense_gemv(cudaStream_t st, int n, const double* Mc, const double* x, double* y) {
    if (n <= 0) return cudaSuccess;
    counted();
    k_dense_gemv<<<(n + 7) / 8, 256, 0, st>>>(n, Mc, x, y);
    return cudaGetLastError();
}

cudaError_t launch_ap_coarse(cudaStream_t st, const ApLevel* lvl, int nlev, int ntop, const double* L, double* ytop) {
    if (nlev <= 0 && ntop <= 0) return cudaSuccess;
    counted();
    const size_t smem = sizeof(double) * (kCoarseSmax + kCoarseNmax) * (kCoarseThreads / 32);
    cudaError_t e = cudaFuncSetAttribute(k_ap_coarse, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_ap_coarse<<<1, kCoarseThreads, smem, st>>>(lvl, nlev, ntop, L, ytop);
    return cudaGetLastError();
}

cudaError_t launch_vcopy(cudaStream_t st, const VCopyDev* cps, int ncps, const double* src, double* dst,
                         int reverse) {
    if (ncps <= 0) return cudaSuccess;
    counted();
    k_vcopy<<<blocks_for(ncps, 8), 256, 0, st>>>(cps, ncps, src, dst, reverse);
    return cudaGetLastError();
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
    k_fp64_peak<<<nblocks, 256, 0, st>>>(iters, sink);
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
