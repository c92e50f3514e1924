// hs_nodc.cu -- the elimination step without deferred compression (the
// original LoRaSp step that Sec. 2 of the paper analyses), for comparing the
// two schemes on the whole solver.  One CTA per cluster of a phase, FP64
// arithmetic, the same task / list records and the same outputs as the
// deferred-compression kernel, so that the Schur-update kernel, the level
// assembly and the whole solve phase (Algorithm 2) run unchanged.
//
// Per cluster s with n-neighbour columns A_sn and fill columns A_sw:
//   1. column-pivoted Householder QR of the unscaled A_sw (Eq. offdiag), every
//      reflector applied to the whole row [A_sn | A_sw | I]: the identity
//      columns become U^T; rank r = smallest k with the squared trailing
//      Frobenius norm <= eps^2 * max_i (A_ss)_ii (the threshold deferred
//      compression applies when A_ss is a multiple of the identity);
//   2. A_ss <- U^T A_ss U (the reflectors from both sides, Eq. sparse);
//   3. Cholesky of the fine block, (U^T A_ss U)_ff = G_f G_f^T;
//   4. K = G_f^-1 [(U^T A_ss U)_fc | (U^T A_sn)_f | (U^T)_f];
//   5. the coarse DOFs after eliminating f: A_cc - K_c^T K_c, coupling to n
//      (U^T A_sn)_c - K_c^T K_n, coupling to w V_1^T; the rows c of the
//      solve-phase operator (U^T)_c - K_c^T G_f^-1 (U^T)_f;
//   6. stored: W = [[I, -K_c^T G_f^-1], [0, G_f^-1]] U^T (s x s) and C = K_n,
//      the same roles as W = U^T G^-1 and C with deferred compression: the
//      forward solve step is y_s <- W y_s, y_n -= C^T y_f.
// The pivot and Householder conventions are those of the other kernels:
// lowest-index column with squared norm >= (1 - 1e-6) times the largest;
// beta = -sign(alpha) * norm, v_k = 1, tau = (beta - alpha) / beta.
#include <cfloat>
#include <climits>
#include <cstdint>

#include "hs_internal.h"

namespace hs {

namespace {

constexpr int kNodcThreads = 256;
constexpr double kNodcPivotTie = 1e-6;

__device__ double nd_block_sum(double v, double* red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double t = lane < nw ? red[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    return t;
}

__device__ double nd_block_max(double v, double* red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double t = lane < nw ? red[lane] : -DBL_MAX;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t = fmax(t, __shfl_xor_sync(0xffffffffu, t, o));
    return t;
}

__device__ int nd_block_min_int(int v, double* red) {
    int* ri = reinterpret_cast<int*>(red);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if (lane == 0) ri[wid] = v;
    __syncthreads();
    int t = lane < nw ? ri[lane] : INT_MAX;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t = min(t, __shfl_xor_sync(0xffffffffu, t, o));
    return t;
}

struct NdEntry {
    int64_t cq, qc;
    int32_t ldcq, ldqc, w, pad;
};

// Shared memory (doubles): V (smax^2) | tau (smax) | A (smax^2) | cn (wmax) |
// red (64) | entries (lmax) | ioff (lmax + 1 ints) | flag
size_t nodc_smem(int smax, int wmax, int lmax) {
    return sizeof(double) * ((size_t)2 * smax * smax + smax + wmax + 64) + sizeof(NdEntry) * (size_t)lmax +
           sizeof(int) * (size_t)(lmax + 4);
}

template <typename FT>
__global__ void __launch_bounds__(kNodcThreads)
k_factor_nodc(const TaskDev* __restrict__ tasks, int t0, const ListDev* __restrict__ lists,
              double* __restrict__ blocks, const int64_t* __restrict__ blk_off, const int32_t* __restrict__ blk_ld,
              int32_t* __restrict__ cur, FT* __restrict__ fac, int32_t* __restrict__ meta,
              double* __restrict__ ws, double eps2, int32_t* status, int32_t level, int smax, int wmax, int lmax) {
    extern __shared__ double sm[];
    const TaskDev T = tasks[t0 + blockIdx.x];
    const int s = T.s, tid = threadIdx.x, NT = blockDim.x, L = T.nn + T.nw;
    double* V = sm;                               // reflector k in column k (v_k = 1)
    double* tau = V + (size_t)smax * smax;
    double* A = tau + smax;                       // A_ss, then U^T A_ss U, then its fine Cholesky
    double* cn = A + (size_t)smax * smax;         // squared column norms of the fill block
    double* red = cn + wmax;
    NdEntry* em = reinterpret_cast<NdEntry*>(red + 64);
    int* ioff = reinterpret_cast<int*>(em + lmax);
    int* flag = ioff + lmax + 1;

    for (int e = tid; e < L; e += NT) {
        const ListDev le = lists[T.list + e];
        NdEntry m;
        m.cq = blk_off[le.blk_cq];
        m.qc = blk_off[le.blk_qc];
        m.ldcq = blk_ld[le.blk_cq];
        m.ldqc = blk_ld[le.blk_qc];
        m.w = cur[le.q];
        m.pad = 0;
        em[e] = m;
    }
    __syncthreads();
    if (tid == 0) {
        int o = 0;
        for (int e = 0; e < L; e++) {
            ioff[e] = o;
            o += em[e].w;
        }
        ioff[L] = o;
        *flag = 0;
    }
    __syncthreads();
    const int W = ioff[L], ncols = ioff[T.nn], Wn = W - ncols, Wt = W + s;
    double* M = ws + T.m_off;  // [A_sn | A_sw | I], s x Wt, row-major
    {
        const double* Ad = blocks + blk_off[T.diag_blk];
        const int ld = blk_ld[T.diag_blk];
        for (int idx = tid; idx < s * s; idx += NT) A[idx] = Ad[(int64_t)(idx / s) * ld + idx % s];
    }
    for (int e = 0; e < L; e++) {
        const int wq = ioff[e + 1] - ioff[e], o = ioff[e];
        const double* src = blocks + em[e].cq;
        const int ld = em[e].ldcq;
        for (int idx = tid; idx < s * wq; idx += NT) {
            const int i = idx / wq, j = idx % wq;
            M[(int64_t)i * Wt + o + j] = src[(int64_t)i * ld + j];
        }
    }
    for (int idx = tid; idx < s * s; idx += NT) M[(int64_t)(idx / s) * Wt + W + idx % s] = (idx / s == idx % s);
    __syncthreads();
    double ldm = 0.0;
    for (int i = tid; i < s; i += NT) ldm = fmax(ldm, A[i * s + i]);
    const double thr2 = eps2 * nd_block_max(ldm, red);

    // 1. column-pivoted QR of the unscaled fill columns, reflectors on the whole row
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
    while (k < s && Wn > 0) {
        double lt = 0.0, lm = 0.0;
        for (int j = tid; j < Wn; j += NT)
            if (cn[j] >= 0.0) {
                lt += cn[j];
                lm = fmax(lm, cn[j]);
            }
        const double total = nd_block_sum(lt, red);
        const double cmax = nd_block_max(lm, red);
        if (total <= thr2) break;
        const double th = (1.0 - kNodcPivotTie) * cmax;
        int lp = INT_MAX;
        for (int j = tid; j < Wn; j += NT)
            if (cn[j] >= 0.0 && cn[j] >= th) {
                lp = j;
                break;
            }
        const int p = nd_block_min_int(lp, red);
        const int pc = ncols + p;
        double ls = 0.0;
        for (int i = k + 1 + tid; i < s; i += NT) {
            const double x = M[(int64_t)i * Wt + pc];
            ls += x * x;
        }
        const double sig = nd_block_sum(ls, red);
        const double alpha = M[(int64_t)k * Wt + pc];
        const double nrm = sqrt(alpha * alpha + sig);
        const double beta = alpha >= 0.0 ? -nrm : nrm;
        const double tk = (beta - alpha) / beta, scal = 1.0 / (alpha - beta);
        for (int i = tid; i < s; i += NT)
            V[i * smax + k] = i < k ? 0.0 : (i == k ? 1.0 : M[(int64_t)i * Wt + pc] * scal);
        if (tid == 0) {
            tau[k] = tk;
            cn[p] = -1.0;
        }
        __syncthreads();
        for (int i = k + tid; i < s; i += NT) M[(int64_t)i * Wt + pc] = (i == k) ? beta : 0.0;
        for (int j = tid; j < Wt; j += NT) {
            if (j == pc) continue;
            const bool cand = j >= ncols && j < W;
            if (cand && cn[j - ncols] < 0.0) continue;  // pivoted: zero below its row
            double t = M[(int64_t)k * Wt + j];
            for (int i = k + 1; i < s; i++) t += V[i * smax + k] * M[(int64_t)i * Wt + j];
            t *= tk;
            M[(int64_t)k * Wt + j] -= t;
            double c = 0.0;
            for (int i = k + 1; i < s; i++) {
                const double x = M[(int64_t)i * Wt + j] - t * V[i * smax + k];
                M[(int64_t)i * Wt + j] = x;
                if (cand) c += x * x;
            }
            if (cand) cn[j - ncols] = c;
        }
        __syncthreads();
        k++;
    }
    const int r = k, f = s - r;

    // 2. A <- U^T A U: reflector kk on the columns of A (from the left), then
    // on its rows (from the right)
    for (int kk = 0; kk < r; kk++) {
        for (int j = tid; j < s; j += NT) {
            double t = 0.0;
            for (int i = kk; i < s; i++) t += V[i * smax + kk] * A[i * s + j];
            t *= tau[kk];
            for (int i = kk; i < s; i++) A[i * s + j] -= t * V[i * smax + kk];
        }
        __syncthreads();
    }
    for (int kk = 0; kk < r; kk++) {
        for (int i = tid; i < s; i += NT) {
            double t = 0.0;
            for (int j = kk; j < s; j++) t += A[i * s + j] * V[j * smax + kk];
            t *= tau[kk];
            for (int j = kk; j < s; j++) A[i * s + j] -= t * V[j * smax + kk];
        }
        __syncthreads();
    }

    // 3. Cholesky of the fine block A[r:, r:] in place (lower triangle)
    for (int j = r; j < s; j++) {
        if (tid == 0) {
            const double d = A[j * s + j];
            if (!(d > 0.0)) {
                *flag = 1;
            } else {
                A[j * s + j] = sqrt(d);
            }
        }
        __syncthreads();
        if (*flag) {
            if (tid == 0 && atomicCAS(status, 0, ST_NOT_SPD) == 0) {
                status[1] = level;
                status[2] = T.c;
            }
            return;
        }
        const double g = A[j * s + j];
        for (int i = j + 1 + tid; i < s; i += NT) A[i * s + j] /= g;
        __syncthreads();
        const int m = s - j - 1;
        for (int idx = tid; idx < m * m; idx += NT) {
            const int i = j + 1 + idx / m, c = j + 1 + idx % m;
            if (c <= i) A[i * s + c] -= A[i * s + j] * A[c * s + j];
        }
        __syncthreads();
    }

    // 4. K = G_f^-1 [A_fc | (U^T A_sn)_f | (U^T)_f], column by column: the
    // first r columns live in A[r:, :r], the others in the rows r.. of M
    const int nk = r + ncols + s;
    for (int c = tid; c < nk; c += NT) {
        for (int i = 0; i < f; i++) {
            double* xi = c < r ? &A[(r + i) * s + c]
                               : &M[(int64_t)(r + i) * Wt + (c - r < ncols ? c - r : W + (c - r - ncols))];
            double acc = *xi;
            for (int q = 0; q < i; q++) {
                const double xq = c < r ? A[(r + q) * s + c]
                                        : M[(int64_t)(r + q) * Wt + (c - r < ncols ? c - r : W + (c - r - ncols))];
                acc -= A[(r + i) * s + r + q] * xq;
            }
            *xi = acc / A[(r + i) * s + r + i];
        }
    }
    __syncthreads();

    // 5. the coarse DOFs after eliminating f: A_cc -= K_c^T K_c (into V's
    // space, free now), rows c of [n columns | W] -= K_c^T K_(n | W)
    double* Acc = V;
    for (int idx = tid; idx < r * r; idx += NT) {
        const int i = idx / r, j = idx % r;
        double acc = A[i * s + j];
        for (int q = 0; q < f; q++) acc -= A[(r + q) * s + i] * A[(r + q) * s + j];
        Acc[idx] = acc;
    }
    for (int idx = tid; idx < r * (ncols + s); idx += NT) {
        const int i = idx / (ncols + s), c = idx % (ncols + s);
        const int col = c < ncols ? c : W + (c - ncols);
        double acc = M[(int64_t)i * Wt + col];
        for (int q = 0; q < f; q++) acc -= A[(r + q) * s + i] * M[(int64_t)(r + q) * Wt + col];
        M[(int64_t)i * Wt + col] = acc;
    }
    __syncthreads();

    // 6. factor records, stored operators, coarse write-back
    int32_t* mt = meta + T.meta;
    if (tid == 0) mt[0] = r;
    for (int e = tid; e < T.nn; e += NT) {
        mt[1 + 2 * e] = ioff[e];
        mt[2 + 2 * e] = ioff[e + 1] - ioff[e];
    }
    FT* Wf = fac + T.w_off;
    for (int idx = tid; idx < s * s; idx += NT) Wf[idx] = (FT)M[(int64_t)(idx / s) * Wt + W + idx % s];
    FT* Cf = fac + T.c_off;
    for (int idx = tid; idx < f * ncols; idx += NT) {
        const int i = idx / ncols, j = idx % ncols;
        Cf[(int64_t)i * T.ncap + j] = (FT)M[(int64_t)(r + i) * Wt + j];
    }
    if (T.nw > 0 && r > 0) {
        for (int e = 0; e < L; e++) {
            const int wq = ioff[e + 1] - ioff[e], o = ioff[e];
            double* dcq = blocks + em[e].cq;
            double* dqc = blocks + em[e].qc;
            for (int idx = tid; idx < r * wq; idx += NT) {
                const int i = idx / wq, j = idx % wq;
                const double x = M[(int64_t)i * Wt + o + j];
                dcq[(int64_t)i * em[e].ldcq + j] = x;
                dqc[(int64_t)j * em[e].ldqc + i] = x;
            }
        }
        double* dcc = blocks + blk_off[T.diag_blk];
        const int ld = blk_ld[T.diag_blk];
        for (int idx = tid; idx < r * r; idx += NT) {
            const int i = idx / r, j = idx % r;
            // the symmetric coarse block, from its lower triangle
            dcc[(int64_t)i * ld + j] = i >= j ? Acc[i * r + j] : Acc[j * r + i];
        }
    }
    if (tid == 0) cur[T.c] = (T.nw > 0) ? r : 0;
}

}  // namespace

size_t factor_nodc_smem_bytes(int smax, int wmax, int lmax) { return nodc_smem(smax, wmax, lmax); }

cudaError_t launch_factor_nodc(cudaStream_t st, const TaskDev* tasks, int t0, int ntasks, int smax, int wmax,
                               int lmax, const ListDev* lists, double* blocks, const int64_t* blk_off,
                               const int32_t* blk_ld, int32_t* cur, void* fac, int fp32, int32_t* meta, double* ws,
                               double eps2, int32_t* status, int32_t level) {
    if (ntasks <= 0) return cudaSuccess;
    const size_t smem = nodc_smem(smax, wmax, lmax);
    const void* fn = fp32 ? reinterpret_cast<const void*>(&k_factor_nodc<float>)
                          : reinterpret_cast<const void*>(&k_factor_nodc<double>);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (fp32)
        k_factor_nodc<float><<<ntasks, kNodcThreads, smem, st>>>(tasks, t0, lists, blocks, blk_off, blk_ld, cur,
                                                                 static_cast<float*>(fac), meta, ws, eps2, status,
                                                                 level, smax, wmax, lmax);
    else
        k_factor_nodc<double><<<ntasks, kNodcThreads, smem, st>>>(tasks, t0, lists, blocks, blk_off, blk_ld, cur,
                                                                  static_cast<double*>(fac), meta, ws, eps2, status,
                                                                  level, smax, wmax, lmax);
    launch_count_add(1);
    return cudaGetLastError();
}

}  // namespace hs
