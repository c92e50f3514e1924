/*
 * hs_oracle.c -- plain, slow FP64 CPU oracle of the hierarchical solver with
 * deferred compression (Chen, Cambier, Boman, Rajamanickam, Tuminaro, Darve,
 * "A Robust Hierarchical Solver for Ill-conditioned Systems with Applications
 * to Ice Sheet Modeling").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this file's library.  It shares no
 * code with the CUDA path.  No BLAS: every dense step is a plain loop.
 *
 * What each part follows:
 *   or_partition_extruded  Sec. 4.2 (extruded partitioning), Sec. 5
 *                          (geometric partition, cluster size), Sec. 5.2
 *                          (coarse partitions halve the fine ones).
 *   phase rule             Algorithm 1 processes the clusters of a level one
 *                          at a time; the order is not specified.  Reading
 *                          used here: repeatedly take the greedy maximal
 *                          independent set (ascending index) of the unprocessed
 *                          clusters in the current block graph; that set is
 *                          one phase; clusters of a phase go in ascending order.
 *   step_core              Sec. 3.1: scaling S_s (Eq. scaling), compression of
 *                          G^-1 A_sw (Eq. offdiag_new) by column-pivoted QR,
 *                          sparsification E_s (Eq. sparse).
 *   Schur update           Eq. elim: X_nn = A_nn - A_ns G^-T U2 U2^T G^-1 A_sn.
 *   write-back             Sec. 3.1: coarse DOFs keep identity diagonal,
 *                          coupling U1^T G^-1 A_sn to n and V1^T to w;
 *                          P_s moves them to the end (Eq. perm).
 *   next level             Algorithm 1: A_c of the coarse DOFs, parents merge
 *                          sibling clusters 2p, 2p+1.
 *   top                    Algorithm 1: conventional Cholesky when small.
 *   or_apply               Algorithm 2: forward W_i y, recursion, backward W_i^T x.
 *   or_pcg / or_gmres      Sec. 5 (preconditioned Krylov solve).
 *   step_nodc              the same elimination without deferred compression
 *                          (the original LoRaSp step that Sec. 2 analyses:
 *                          Eq. offdiag on the unscaled A_sw, then the
 *                          rotation of Eq. sparse and the elimination of the
 *                          fine DOFs, which here also updates the coarse ones).
 *
 * or_factor_create_ex runs the clusters of a phase on several threads
 * (OpenMP) when asked: their own computations in parallel, the Schur updates
 * in parallel over target rows with every block's contributions in ascending
 * cluster order, the write-backs in cluster order, so the result is the same
 * bit for bit as with one thread.
 *
 * Readings where the paper is silent (all shared with the CUDA path by
 * statement only, never by code):
 *   - tolerance is absolute on the scaled block; rank r = smallest k with
 *     ||R[k:,k:]||_F <= eps, checked as sum of squared trailing column
 *     norms <= eps^2 (Frobenius norm bounds the 2-norm of V2 in Eq. offdiag_new);
 *   - pivot = lowest-index unpivoted column whose squared trailing norm is at
 *     least (1 - 1e-6) times the largest (norms recomputed every step; the
 *     band lies well above the rounding of small trailing norms, so that
 *     implementations summing in different orders pivot alike);
 *   - Householder: beta = -sign(alpha) * norm, v_k = 1, tau = (beta-alpha)/beta;
 *   - neighbours of a cluster are the blocks present in the level's input
 *     matrix; every other present block is fill ("w");
 *   - a cluster with no fill block has rank 0 and leaves the matrix; every
 *     other cluster keeps a (possibly empty) coarse part and its blocks;
 *   - eliminating the fine part creates a block between every pair of the
 *     cluster's neighbours (structural, even when the update is zero);
 *   - without DC the same rank rule applies to the unscaled A_sw, at the
 *     threshold eps * sqrt(max_i (A_ss)_ii): the threshold DC applies when
 *     A_ss is a multiple of the identity, expressed in the units of A.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_ERR_ARG 1
#define OR_ERR_NOT_SPD 2
#define OR_ERR_NOCONV 3
#define OR_ERR_OOM 4

#define PIVOT_TIE 1e-6

/* ------------------------------------------------------------------------ */
/* Small helpers                                                            */
/* ------------------------------------------------------------------------ */

static void *xcalloc(size_t n, size_t sz) {
    if (n == 0) n = 1;
    return calloc(n, sz);
}

/* ------------------------------------------------------------------------ */
/* Partition (Sec. 4.2)                                                     */
/* ------------------------------------------------------------------------ */

static int uf_find(int *p, int x) {
    while (p[x] != x) {
        p[x] = p[p[x]];
        x = p[x];
    }
    return x;
}

typedef struct {
    double key;
    int id;
} keyed;

static int cmp_keyed(const void *a, const void *b) {
    const keyed *x = (const keyed *)a, *y = (const keyed *)b;
    if (x->key < y->key) return -1;
    if (x->key > y->key) return 1;
    return (x->id > y->id) - (x->id < y->id);
}

static int cmp_int(const void *a, const void *b) {
    int x = *(const int *)a, y = *(const int *)b;
    return (x > y) - (x < y);
}

typedef struct {
    int nl;                 /* number of lines */
    const double *lx, *ly;  /* line coordinates (or NULL) */
    const int *gptr, *gadj; /* line graph (CSR, sorted) */
    int L;                  /* bisection depth */
    int *leaf_of;           /* output: leaf of each line */
    int next_leaf;
    int *mark, *queue;      /* BFS scratch */
} bisect_ctx;

/* BFS order of the lines in set (size k), restricted to the set; neighbours in
 * ascending index; a new component starts at its lowest-index line. */
static void bfs_order(bisect_ctx *cx, const int *set, int k, int start, int *out) {
    int i, head = 0, tail = 0, done = 0;
    for (i = 0; i < k; i++) cx->mark[set[i]] = 1; /* 1 = in set, unvisited */
    while (done < k) {
        int s = start;
        if (cx->mark[s] != 1) {
            /* lowest-index unvisited line of the set */
            s = -1;
            for (i = 0; i < k; i++)
                if (cx->mark[set[i]] == 1 && (s < 0 || set[i] < s)) s = set[i];
        }
        cx->mark[s] = 2;
        cx->queue[tail++] = s;
        while (head < tail) {
            int u = cx->queue[head++], e;
            out[done++] = u;
            for (e = cx->gptr[u]; e < cx->gptr[u + 1]; e++) {
                int v = cx->gadj[e];
                if (cx->mark[v] == 1) {
                    cx->mark[v] = 2;
                    cx->queue[tail++] = v;
                }
            }
        }
        head = tail = 0;
    }
    for (i = 0; i < k; i++) cx->mark[set[i]] = 0;
}

static void bisect(bisect_ctx *cx, int *set, int k, int depth) {
    int i, left;
    if (depth == cx->L) {
        int leaf = cx->next_leaf++;
        for (i = 0; i < k; i++) cx->leaf_of[set[i]] = leaf;
        return;
    }
    left = (k + 1) / 2;
    if (cx->lx) {
        double mnx = cx->lx[set[0]], mxx = mnx, mny = cx->ly[set[0]], mxy = mny;
        int axis;
        keyed *kv = (keyed *)xcalloc((size_t)k, sizeof(keyed));
        for (i = 1; i < k; i++) {
            double x = cx->lx[set[i]], y = cx->ly[set[i]];
            if (x < mnx) mnx = x;
            if (x > mxx) mxx = x;
            if (y < mny) mny = y;
            if (y > mxy) mxy = y;
        }
        axis = (mxx - mnx >= mxy - mny) ? 0 : 1;
        for (i = 0; i < k; i++) {
            kv[i].key = axis == 0 ? cx->lx[set[i]] : cx->ly[set[i]];
            kv[i].id = set[i];
        }
        qsort(kv, (size_t)k, sizeof(keyed), cmp_keyed);
        for (i = 0; i < k; i++) set[i] = kv[i].id;
        free(kv);
    } else {
        /* graph growing: BFS from the lowest-index line finds a far line;
         * BFS again from there; the first half visited is the left part */
        int *ord = (int *)xcalloc((size_t)k, sizeof(int));
        int lo = set[0];
        for (i = 1; i < k; i++)
            if (set[i] < lo) lo = set[i];
        bfs_order(cx, set, k, lo, ord);
        bfs_order(cx, set, k, ord[k - 1], ord);
        memcpy(set, ord, (size_t)k * sizeof(int));
        free(ord);
    }
    {
        /* each half keeps ascending line order for reproducibility */
        qsort(set, (size_t)left, sizeof(int), cmp_int);
        qsort(set + left, (size_t)(k - left), sizeof(int), cmp_int);
    }
    bisect(cx, set, left, depth + 1);
    bisect(cx, set + left, k - left, depth + 1);
}

/*
 * Column-preserving partition.  Lines = connected components of the strong
 * couplings |a_ij| >= theta * max_{k != i} |a_ik| (either row's test).  The
 * line graph is bisected recursively (coordinates of each line's lowest DOF
 * when given, BFS graph growing otherwise) into 2^L leaves, L the smallest
 * with ceil(lines / 2^L) <= leaf_lines.  Leaf c's DOFs, ascending, occupy
 * perm[leaf_ptr[c] .. leaf_ptr[c+1]).
 */
int or_partition_extruded(int64_t n64, const int64_t *rowptr, const int32_t *col,
                          const double *val, const double *coords,
                          int32_t leaf_lines, double theta, int32_t *perm,
                          int32_t *leaf_ptr, int32_t *nleaf_out) {
    int n = (int)n64, i, nl = 0, L = 0, c;
    int *par, *line_of, *first, *cnt, *gptr, *gadj, *set, *tmp;
    double *lx = NULL, *ly = NULL;
    bisect_ctx cx;
    if (n <= 0 || leaf_lines <= 0) return OR_ERR_ARG;
    par = (int *)xcalloc((size_t)n, sizeof(int));
    for (i = 0; i < n; i++) par[i] = i;
    for (i = 0; i < n; i++) {
        double m = 0.0;
        int64_t e;
        for (e = rowptr[i]; e < rowptr[i + 1]; e++)
            if (col[e] != i && fabs(val[e]) > m) m = fabs(val[e]);
        if (m <= 0.0) continue;
        for (e = rowptr[i]; e < rowptr[i + 1]; e++) {
            int j = col[e];
            if (j != i && fabs(val[e]) >= theta * m) {
                int a = uf_find(par, i), b = uf_find(par, j);
                if (a != b) {
                    if (a < b) par[b] = a;
                    else par[a] = b;
                }
            }
        }
    }
    /* lines numbered in order of their lowest DOF */
    line_of = (int *)xcalloc((size_t)n, sizeof(int));
    first = (int *)xcalloc((size_t)n, sizeof(int));
    {
        int *root_line = (int *)xcalloc((size_t)n, sizeof(int));
        for (i = 0; i < n; i++) root_line[i] = -1;
        for (i = 0; i < n; i++) {
            int r = uf_find(par, i);
            if (root_line[r] < 0) {
                root_line[r] = nl;
                first[nl] = i;
                nl++;
            }
            line_of[i] = root_line[r];
        }
        free(root_line);
    }
    /* line graph */
    {
        int *deg = (int *)xcalloc((size_t)nl + 1, sizeof(int));
        int *lst = NULL, nlst = 0, cap = 0, l;
        /* collect (line_i, line_j) pairs then dedup per line */
        int **nb = (int **)xcalloc((size_t)nl, sizeof(int *));
        int *nbn = (int *)xcalloc((size_t)nl, sizeof(int));
        int *nbc = (int *)xcalloc((size_t)nl, sizeof(int));
        (void)lst; (void)nlst; (void)cap;
        for (i = 0; i < n; i++) {
            int64_t e;
            int li = line_of[i];
            for (e = rowptr[i]; e < rowptr[i + 1]; e++) {
                int lj = line_of[col[e]];
                if (lj == li) continue;
                if (nbn[li] == nbc[li]) {
                    nbc[li] = nbc[li] ? 2 * nbc[li] : 8;
                    nb[li] = (int *)realloc(nb[li], (size_t)nbc[li] * sizeof(int));
                }
                nb[li][nbn[li]++] = lj;
            }
        }
        gptr = (int *)xcalloc((size_t)nl + 1, sizeof(int));
        for (l = 0; l < nl; l++) {
            int k2 = 0, t;
            qsort(nb[l], (size_t)nbn[l], sizeof(int), cmp_int);
            for (t = 0; t < nbn[l]; t++)
                if (k2 == 0 || nb[l][t] != nb[l][k2 - 1]) nb[l][k2++] = nb[l][t];
            nbn[l] = k2;
            gptr[l + 1] = gptr[l] + k2;
        }
        gadj = (int *)xcalloc((size_t)gptr[nl], sizeof(int));
        for (l = 0; l < nl; l++) {
            if (nbn[l]) memcpy(gadj + gptr[l], nb[l], (size_t)nbn[l] * sizeof(int));
            free(nb[l]);
        }
        free(nb); free(nbn); free(nbc); free(deg);
    }
    if (coords) {
        lx = (double *)xcalloc((size_t)nl, sizeof(double));
        ly = (double *)xcalloc((size_t)nl, sizeof(double));
        for (i = 0; i < nl; i++) {
            lx[i] = coords[2 * (int64_t)first[i]];
            ly[i] = coords[2 * (int64_t)first[i] + 1];
        }
    }
    while (((int64_t)nl + (1LL << L) - 1) / (1LL << L) > leaf_lines && (1 << (L + 1)) <= nl) L++;
    cx.nl = nl; cx.lx = lx; cx.ly = ly; cx.gptr = gptr; cx.gadj = gadj; cx.L = L;
    cx.leaf_of = (int *)xcalloc((size_t)nl, sizeof(int));
    cx.next_leaf = 0;
    cx.mark = (int *)xcalloc((size_t)nl, sizeof(int));
    cx.queue = (int *)xcalloc((size_t)nl, sizeof(int));
    set = (int *)xcalloc((size_t)nl, sizeof(int));
    for (i = 0; i < nl; i++) set[i] = i;
    bisect(&cx, set, nl, 0);
    /* perm: leaves in order, DOFs ascending inside each leaf */
    cnt = (int *)xcalloc((size_t)cx.next_leaf + 1, sizeof(int));
    for (i = 0; i < n; i++) cnt[cx.leaf_of[line_of[i]] + 1]++;
    for (c = 0; c < cx.next_leaf; c++) cnt[c + 1] += cnt[c];
    tmp = (int *)xcalloc((size_t)cx.next_leaf + 1, sizeof(int));
    memcpy(tmp, cnt, (size_t)(cx.next_leaf + 1) * sizeof(int));
    for (i = 0; i < n; i++) perm[tmp[cx.leaf_of[line_of[i]]]++] = i;
    for (c = 0; c <= cx.next_leaf; c++) leaf_ptr[c] = cnt[c];
    *nleaf_out = cx.next_leaf;
    free(tmp); free(cnt); free(set); free(cx.mark); free(cx.queue);
    free(cx.leaf_of); free(lx); free(ly); free(gptr); free(gadj);
    free(line_of); free(first); free(par);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Dense kernels (row-major, plain loops)                                   */
/* ------------------------------------------------------------------------ */

/* A = G G^T, G lower (Sec. 2, Cholesky factorization).  Returns 0 or k+1
 * when the k-th pivot is not positive. */
static int chol_lower(int n, double *a) {
    int i, j, k;
    for (j = 0; j < n; j++) {
        double d = a[j * n + j];
        for (k = 0; k < j; k++) d -= a[j * n + k] * a[j * n + k];
        if (!(d > 0.0)) return j + 1;
        d = sqrt(d);
        a[j * n + j] = d;
        for (i = j + 1; i < n; i++) {
            double t = a[i * n + j];
            for (k = 0; k < j; k++) t -= a[i * n + k] * a[j * n + k];
            a[i * n + j] = t / d;
        }
        for (i = 0; i < j; i++) a[i * n + j] = 0.0;
    }
    return 0;
}

/* B <- G^-1 B, G lower n x n, B n x m (forward substitution). */
static void lower_solve(int n, const double *g, int m, double *b) {
    int i, k, j;
    for (i = 0; i < n; i++) {
        double *bi = b + (size_t)i * m;
        for (k = 0; k < i; k++) {
            double gik = g[i * n + k];
            const double *bk = b + (size_t)k * m;
            for (j = 0; j < m; j++) bi[j] -= gik * bk[j];
        }
        for (j = 0; j < m; j++) bi[j] /= g[i * n + i];
    }
}

/* x <- G^-T x */
static void lower_t_solve_vec(int n, const double *g, double *x) {
    int i, k;
    for (i = n - 1; i >= 0; i--) {
        double t = x[i];
        for (k = i + 1; k < n; k++) t -= g[k * n + i] * x[k];
        x[i] = t / g[i * n + i];
    }
}

static void lower_solve_vec(int n, const double *g, double *x) {
    int i, k;
    for (i = 0; i < n; i++) {
        double t = x[i];
        for (k = 0; k < i; k++) t -= g[i * n + k] * x[k];
        x[i] = t / g[i * n + i];
    }
}

/*
 * Column-pivoted Householder QR (Businger-Golub) of the nw columns
 * M[:, nn : nn+nw] of the s x W matrix M (W = nn + nw), stopping at the
 * smallest k with ||R[k:,k:]||_F <= eps; every reflector is applied to all W
 * columns, so on return rows 0..r-1 of M hold U^T M (coarse rows) and rows
 * r.. hold the rest.  V (s x s, column k = reflector k, v_k = 1) and tau.
 * Returns the rank r.  (Eq. offdiag_new.)
 */
static int cpqr_apply(int s, int nn, int nw, double *M, double eps, double *V,
                      double *tau, int *piv) {
    int W = nn + nw, k = 0, i, j;
    char *used = (char *)xcalloc((size_t)nw, 1);
    double *cn = (double *)xcalloc((size_t)nw, sizeof(double));
    for (;;) {
        double total = 0.0, cmax = 0.0, alpha, sig, nrm, beta, t;
        int p = -1, pc;
        if (k >= s) break;
        for (j = 0; j < nw; j++) {
            double c = 0.0;
            if (used[j]) continue;
            for (i = k; i < s; i++) {
                double m = M[(size_t)i * W + nn + j];
                c += m * m;
            }
            cn[j] = c;
            total += c;
            if (c > cmax) cmax = c;
        }
        if (total <= eps * eps) break;
        for (j = 0; j < nw; j++)
            if (!used[j] && cn[j] >= (1.0 - PIVOT_TIE) * cmax) {
                p = j;
                break;
            }
        used[p] = 1;
        piv[k] = p;
        pc = nn + p;
        alpha = M[(size_t)k * W + pc];
        sig = 0.0;
        for (i = k + 1; i < s; i++) sig += M[(size_t)i * W + pc] * M[(size_t)i * W + pc];
        nrm = sqrt(alpha * alpha + sig);
        beta = alpha >= 0.0 ? -nrm : nrm;
        for (i = 0; i < s; i++) V[(size_t)i * s + k] = 0.0;
        V[(size_t)k * s + k] = 1.0;
        for (i = k + 1; i < s; i++) V[(size_t)i * s + k] = M[(size_t)i * W + pc] / (alpha - beta);
        tau[k] = (beta - alpha) / beta;
        M[(size_t)k * W + pc] = beta;
        for (i = k + 1; i < s; i++) M[(size_t)i * W + pc] = 0.0;
        for (j = 0; j < W; j++) {
            if (j == pc) continue;
            if (j >= nn && used[j - nn]) continue; /* zero below its row */
            t = M[(size_t)k * W + j];
            for (i = k + 1; i < s; i++) t += V[(size_t)i * s + k] * M[(size_t)i * W + j];
            t *= tau[k];
            M[(size_t)k * W + j] -= t;
            for (i = k + 1; i < s; i++) M[(size_t)i * W + j] -= t * V[(size_t)i * s + k];
        }
        k++;
    }
    free(used);
    free(cn);
    return k;
}

/*
 * One scaled low-rank elimination step on a dense block row (Sec. 3.1).
 * In:  Ass (s x s), M = [A_sn | A_sw] (s x (nn+nw)).
 * Out: Ass <- G (lower), M <- U^T G^-1 M, V/tau reflectors, rank.
 * Returns 0 or OR_ERR_NOT_SPD.
 */
static int step_core(int s, int nn, int nw, double *Ass, double *M, double eps,
                     double *V, double *tau, int *rank) {
    int *piv = (int *)xcalloc((size_t)s + 1, sizeof(int));
    if (chol_lower(s, Ass)) {
        free(piv);
        return OR_ERR_NOT_SPD;
    }
    lower_solve(s, Ass, nn + nw, M);                      /* Eq. scaling */
    *rank = cpqr_apply(s, nn, nw, M, eps, V, tau, piv);   /* Eq. offdiag_new, sparse */
    free(piv);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Block store of one level                                                 */
/* ------------------------------------------------------------------------ */

typedef struct {
    int q;
    double *a; /* size[p] x size[q], row-major */
} blk;

typedef struct {
    int n, cap;
    blk *v; /* sorted by q */
} brow;

typedef struct {
    int nc;
    int *size;
    brow *rows;
} bmat;

static blk *bfind(bmat *m, int p, int q) {
    brow *r = &m->rows[p];
    int lo = 0, hi = r->n - 1;
    while (lo <= hi) {
        int mid = (lo + hi) / 2;
        if (r->v[mid].q == q) return &r->v[mid];
        if (r->v[mid].q < q) lo = mid + 1;
        else hi = mid - 1;
    }
    return NULL;
}

static blk *bensure(bmat *m, int p, int q) {
    brow *r = &m->rows[p];
    blk *b = bfind(m, p, q);
    int pos;
    if (b) return b;
    if (r->n == r->cap) {
        r->cap = r->cap ? 2 * r->cap : 8;
        r->v = (blk *)realloc(r->v, (size_t)r->cap * sizeof(blk));
    }
    pos = r->n;
    while (pos > 0 && r->v[pos - 1].q > q) {
        r->v[pos] = r->v[pos - 1];
        pos--;
    }
    r->v[pos].q = q;
    r->v[pos].a = (double *)xcalloc((size_t)m->size[p] * (size_t)m->size[q], sizeof(double));
    r->n++;
    return &r->v[pos];
}

static void bremove(bmat *m, int p, int q) {
    brow *r = &m->rows[p];
    int i;
    for (i = 0; i < r->n; i++)
        if (r->v[i].q == q) break;
    if (i == r->n) return;
    free(r->v[i].a);
    for (; i + 1 < r->n; i++) r->v[i] = r->v[i + 1];
    r->n--;
}

static void bfree(bmat *m) {
    int p, i;
    for (p = 0; p < m->nc; p++) {
        for (i = 0; i < m->rows[p].n; i++) free(m->rows[p].v[i].a);
        free(m->rows[p].v);
    }
    free(m->rows);
    free(m->size);
}

/* ------------------------------------------------------------------------ */
/* Factor                                                                   */
/* ------------------------------------------------------------------------ */

typedef struct {
    int c, s, r;   /* cluster, size when processed, rank */
    int nodc;      /* 1: step without deferred compression (step_nodc) */
    double *G;     /* s x s (with DC) */
    double *V;     /* s x s (first r columns used) */
    double *tau;   /* s */
    int nn;        /* number of n-neighbours */
    int *nq, *nm;  /* their ids and widths when processed */
    int ncols;     /* sum of nm */
    double *C;     /* (s - r) x ncols */
    double *Gf;    /* without DC: (s - r) x (s - r), Cholesky factor of the fine block */
    double *Kc;    /* without DC: (s - r) x r */
} fstep;

typedef struct {
    int nc;
    int *size0;      /* sizes at level start */
    int *final;      /* sizes at level end (rank, 0 if gone) */
    int *phase;      /* phase of each cluster (-1 if empty) */
    int64_t *off;    /* vector slot offsets */
    int64_t len;
    int nsteps;
    fstep *steps;    /* processing order */
    int nphases;
} flevel;

typedef struct or_factor {
    int n;
    int32_t *perm;
    int depth;
    double eps;
    flevel *lev;     /* depth levels */
    int ntop_c;      /* clusters at the top */
    int *top_size;
    int64_t *top_off;
    int ntop;        /* dense top size */
    double *Ltop;    /* ntop x ntop */
    int64_t factor_bytes;
} or_factor;

static void step_free(fstep *st) {
    free(st->G); free(st->V); free(st->tau); free(st->nq); free(st->nm); free(st->C);
    free(st->Gf); free(st->Kc);
}

void or_factor_free(or_factor *f) {
    int l, i;
    if (!f) return;
    for (l = 0; l < f->depth; l++) {
        flevel *lv = &f->lev[l];
        for (i = 0; i < lv->nsteps; i++) step_free(&lv->steps[i]);
        free(lv->steps); free(lv->size0); free(lv->final); free(lv->phase); free(lv->off);
    }
    free(f->lev); free(f->perm); free(f->top_size); free(f->top_off); free(f->Ltop);
    free(f);
}

static int in_sorted(const int *a, int n, int x) {
    int lo = 0, hi = n - 1;
    while (lo <= hi) {
        int mid = (lo + hi) / 2;
        if (a[mid] == x) return 1;
        if (a[mid] < x) lo = mid + 1;
        else hi = mid - 1;
    }
    return 0;
}

/*
 * One cluster of a phase in three parts.  Clusters of a phase share no block
 * (they are pairwise non-adjacent), so cluster_compute of one reads nothing
 * that another's Schur update or write-back of the same phase writes; the
 * Schur updates of a phase touch each target block in ascending cluster
 * order, as they would one cluster after another.  The results equal those
 * of processing the clusters of a phase strictly one after another.
 */
typedef struct {
    int nn, nw, ncol, W;
    int *nl, *wl; /* n-neighbours (blocks of the level input), fill blocks */
    double *M;    /* transformed block row (s x W): coarse rows 0..r-1 */
    double *Acc;  /* no DC: coarse diagonal block (r x r) after eliminating f */
} cwork;

static void cwork_free(cwork *w) {
    free(w->nl); free(w->wl); free(w->M); free(w->Acc);
    memset(w, 0, sizeof(*w));
}

/* Apply reflector k (column k of V, scalar tau) to rows k.. of the s x m
 * matrix X from the left (X <- H_k X, H_k = I - tau v v^T). */
static void reflect_rows(int s, const double *V, int k, double tau, int m, double *X) {
    int i, j;
    for (j = 0; j < m; j++) {
        double t = 0.0;
        for (i = k; i < s; i++) t += V[(size_t)i * s + k] * X[(size_t)i * m + j];
        t *= tau;
        for (i = k; i < s; i++) X[(size_t)i * m + j] -= t * V[(size_t)i * s + k];
    }
}

/*
 * Elimination step without deferred compression (plain LoRaSp, Sec. 2,
 * Eq. offdiag and Eq. sc_old, with the sparsification of Eq. sparse and the
 * elimination of the fine DOFs as in Sec. 3.1): A_sw itself is compressed,
 * A_sw ~ U_1 V_1^T with ||V_2|| <= eps (same column-pivoted QR and rank rule
 * as with DC, on the unscaled block); the block row and column are rotated by
 * U^T, so that the fine DOFs f = r..s-1 have no fill coupling; then f is
 * eliminated by Cholesky of (U^T A_ss U)_ff = G_f G_f^T, which updates the
 * coarse DOFs c = 0..r-1 (diagonal and coupling to n) and the neighbours n:
 *   K = G_f^-1 [ (U^T A_ss U)_fc | (U^T A_sn)_f ],
 *   A_cc <- (U^T A_ss U)_cc - K_c^T K_c,  A_cn <- (U^T A_sn)_c - K_c^T K_n,
 *   A_nn <- A_nn - K_n^T K_n,  A_cw <- V_1^T.
 * In: Ass (s x s), M = [A_sn | A_sw] (s x W).  Out: M rows 0..r-1 = the
 * coarse rows [A_cn | V_1^T], st->V / tau (r reflectors), st->Gf, st->Kc,
 * st->C = K_n, *Acc_out (r x r).  Returns 0 or OR_ERR_NOT_SPD.
 */
static int step_nodc(int s, int nn, int nw, double *Ass, double *M, double eps, fstep *st,
                     double **Acc_out) {
    int W = nn + nw, r, f, i, j, k;
    int *piv = (int *)xcalloc((size_t)s + 1, sizeof(int));
    double *At, *Kc, *Acc, dmax = 0.0;
    /* the threshold in the units of A: eps times the square root of the
     * largest diagonal entry of A_ss (the threshold DC applies when A_ss is
     * a multiple of the identity) */
    for (i = 0; i < s; i++)
        if (Ass[(size_t)i * s + i] > dmax) dmax = Ass[(size_t)i * s + i];
    r = cpqr_apply(s, nn, nw, M, eps * sqrt(dmax), st->V, st->tau, piv); /* Eq. offdiag on A_sw */
    free(piv);
    f = s - r;
    /* U^T A_ss U: the reflectors from the left, then (by symmetry) again on
     * the transpose, which applies them from the right */
    At = (double *)xcalloc((size_t)s * (size_t)s, sizeof(double));
    memcpy(At, Ass, (size_t)s * (size_t)s * sizeof(double));
    for (k = 0; k < r; k++) reflect_rows(s, st->V, k, st->tau[k], s, At);
    for (i = 0; i < s; i++)
        for (j = 0; j < i; j++) {
            double t = At[(size_t)i * s + j];
            At[(size_t)i * s + j] = At[(size_t)j * s + i];
            At[(size_t)j * s + i] = t;
        }
    for (k = 0; k < r; k++) reflect_rows(s, st->V, k, st->tau[k], s, At);
    /* G_f G_f^T = (U^T A_ss U)_ff */
    st->Gf = (double *)xcalloc((size_t)f * (size_t)f + 1, sizeof(double));
    for (i = 0; i < f; i++)
        for (j = 0; j < f; j++) st->Gf[(size_t)i * f + j] = At[(size_t)(r + i) * s + r + j];
    if (f > 0 && chol_lower(f, st->Gf)) {
        free(At);
        return OR_ERR_NOT_SPD;
    }
    /* K_c = G_f^-1 (U^T A_ss U)_fc, K_n = G_f^-1 (U^T A_sn)_f */
    Kc = (double *)xcalloc((size_t)f * (size_t)r + 1, sizeof(double));
    for (i = 0; i < f; i++)
        for (j = 0; j < r; j++) Kc[(size_t)i * r + j] = At[(size_t)(r + i) * s + j];
    lower_solve(f, st->Gf, r, Kc);
    st->C = (double *)xcalloc((size_t)f * (size_t)nn + 1, sizeof(double));
    for (i = 0; i < f; i++)
        for (j = 0; j < nn; j++) st->C[(size_t)i * nn + j] = M[(size_t)(r + i) * W + j];
    lower_solve(f, st->Gf, nn, st->C);
    /* the coarse DOFs after eliminating f */
    Acc = (double *)xcalloc((size_t)r * (size_t)r + 1, sizeof(double));
    for (i = 0; i < r; i++)
        for (j = 0; j < r; j++) {
            double acc = 0.0;
            for (k = 0; k < f; k++) acc += Kc[(size_t)k * r + i] * Kc[(size_t)k * r + j];
            Acc[(size_t)i * r + j] = At[(size_t)i * s + j] - acc;
        }
    for (i = 0; i < r; i++)
        for (j = 0; j < nn; j++) {
            double acc = 0.0;
            for (k = 0; k < f; k++) acc += Kc[(size_t)k * r + i] * st->C[(size_t)k * nn + j];
            M[(size_t)i * W + j] -= acc;
        }
    st->Kc = Kc;
    st->r = r;
    *Acc_out = Acc;
    free(At);
    return OR_OK;
}

/* Part 1: the cluster's own computation (Algorithm 1, inner call): n / w
 * lists, the block row, the elimination step (with or without DC) and the
 * stored operators.  Reads only the cluster's own block row. */
static int cluster_compute(bmat *m, int pi, const int *adj0, int nadj0, double eps, int nodc,
                           fstep *st, cwork *w) {
    brow *row = &m->rows[pi];
    int s = m->size[pi], i, j, t, rc, r = 0, wcol = 0;
    double *Ass;
    memset(w, 0, sizeof(*w));
    w->nl = (int *)xcalloc((size_t)row->n + 1, sizeof(int));
    w->wl = (int *)xcalloc((size_t)row->n + 1, sizeof(int));
    /* n = present neighbours (blocks of the level input), w = other blocks */
    for (t = 0; t < row->n; t++) {
        int q = row->v[t].q;
        if (q == pi) continue;
        if (in_sorted(adj0, nadj0, q)) w->nl[w->nn++] = q;
        else w->wl[w->nw++] = q;
    }
    for (t = 0; t < w->nn; t++) w->ncol += m->size[w->nl[t]];
    for (t = 0; t < w->nw; t++) wcol += m->size[w->wl[t]];
    w->W = w->ncol + wcol;
    st->ncols = w->ncol;
    w->M = (double *)xcalloc((size_t)s * (size_t)w->W + 1, sizeof(double));
    /* gather the block row [A_sn | A_sw] */
    {
        int c0 = 0;
        for (t = 0; t < w->nn + w->nw; t++) {
            int q = t < w->nn ? w->nl[t] : w->wl[t - w->nn];
            int wq = m->size[q];
            blk *b = bfind(m, pi, q);
            for (i = 0; i < s; i++)
                for (j = 0; j < wq; j++) w->M[(size_t)i * w->W + c0 + j] = b->a[(size_t)i * wq + j];
            c0 += wq;
        }
    }
    Ass = (double *)xcalloc((size_t)s * (size_t)s, sizeof(double));
    memcpy(Ass, bfind(m, pi, pi)->a, (size_t)s * (size_t)s * sizeof(double));
    st->V = (double *)xcalloc((size_t)s * (size_t)s, sizeof(double));
    st->tau = (double *)xcalloc((size_t)s + 1, sizeof(double));
    st->c = pi;
    st->s = s;
    st->nodc = nodc;
    if (nodc) {
        rc = step_nodc(s, w->ncol, wcol, Ass, w->M, eps, st, &w->Acc);
        free(Ass);
        if (rc) return rc;
        r = st->r;
    } else {
        rc = step_core(s, w->ncol, wcol, Ass, w->M, eps, st->V, st->tau, &r);
        if (rc) {
            free(Ass);
            return rc;
        }
        st->G = Ass;
        st->r = r;
        /* C = fine rows of U^T G^-1 A_sn */
        st->C = (double *)xcalloc((size_t)(s - r) * (size_t)w->ncol + 1, sizeof(double));
        for (i = r; i < s; i++)
            for (j = 0; j < w->ncol; j++) st->C[(size_t)(i - r) * w->ncol + j] = w->M[(size_t)i * w->W + j];
    }
    st->nn = w->nn;
    st->nq = (int *)xcalloc((size_t)w->nn + 1, sizeof(int));
    st->nm = (int *)xcalloc((size_t)w->nn + 1, sizeof(int));
    for (t = 0; t < w->nn; t++) {
        st->nq[t] = w->nl[t];
        st->nm[t] = m->size[w->nl[t]];
    }
    return OR_OK;
}

/* The blocks (p, q), p and q n-neighbours of the step, that its Schur update
 * touches (created empty if absent: fill between every pair of neighbours). */
static void cluster_schur_blocks(bmat *m, const cwork *w) {
    int t, u;
    for (t = 0; t < w->nn; t++)
        for (u = 0; u < w->nn; u++) bensure(m, w->nl[t], w->nl[u]);
}

/* Part 2 (Eq. elim): row p's share of the step's Schur update,
 * A(p, q) -= C(:, p)^T C(:, q) for every n-neighbour q; t = p's position. */
static void cluster_schur_row(bmat *m, const fstep *st, const cwork *w, int t) {
    int p = w->nl[t], mp = m->size[p], op = 0, oq = 0, u, i, j, k, f = st->s - st->r;
    for (u = 0; u < t; u++) op += m->size[w->nl[u]];
    for (u = 0; u < w->nn; u++) {
        int q = w->nl[u], mq = m->size[q];
        blk *b = bfind(m, p, q);
        for (i = 0; i < mp; i++)
            for (j = 0; j < mq; j++) {
                double acc = 0.0;
                for (k = 0; k < f; k++)
                    acc += st->C[(size_t)k * w->ncol + op + i] * st->C[(size_t)k * w->ncol + oq + j];
                b->a[(size_t)i * mq + j] -= acc;
            }
        oq += mq;
    }
}

/* Part 3: write back the coarse part (Eq. perm).  With DC its diagonal is the
 * identity (the scaled diagonal block); without DC it is the coarse block
 * left by eliminating the fine DOFs. */
static void cluster_writeback(bmat *m, int pi, const fstep *st, const cwork *w, char *gone) {
    brow *row = &m->rows[pi];
    int r = st->r, t, i, j;
    if (w->nw == 0) {
        /* no fill block: rank 0, the cluster leaves the matrix */
        for (t = 0; t < row->n; t++) {
            int q = row->v[t].q;
            if (q != pi) bremove(m, q, pi);
        }
        for (t = 0; t < row->n; t++) free(row->v[t].a);
        row->n = 0;
        m->size[pi] = 0;
        gone[pi] = 1;
        return;
    }
    {
        int c0 = 0;
        for (t = 0; t < w->nn + w->nw; t++) {
            int q = t < w->nn ? w->nl[t] : w->wl[t - w->nn];
            int wq = m->size[q];
            blk *b = bfind(m, pi, q), *bt = bfind(m, q, pi);
            double *a = (double *)xcalloc((size_t)r * (size_t)wq + 1, sizeof(double));
            double *at = (double *)xcalloc((size_t)wq * (size_t)r + 1, sizeof(double));
            for (i = 0; i < r; i++)
                for (j = 0; j < wq; j++) {
                    a[(size_t)i * wq + j] = w->M[(size_t)i * w->W + c0 + j];
                    at[(size_t)j * r + i] = w->M[(size_t)i * w->W + c0 + j];
                }
            free(b->a); b->a = a;
            free(bt->a); bt->a = at;
            c0 += wq;
        }
    }
    {
        blk *d = bfind(m, pi, pi);
        free(d->a);
        d->a = (double *)xcalloc((size_t)r * (size_t)r + 1, sizeof(double));
        for (i = 0; i < r; i++)
            for (j = 0; j < r; j++)
                d->a[(size_t)i * r + j] = w->Acc ? w->Acc[(size_t)i * r + j] : (i == j ? 1.0 : 0.0);
    }
    m->size[pi] = r;
}

/* Level-0 block matrix from CSR in partition order. */
static void build_level0(bmat *m, int n, const int64_t *rowptr, const int32_t *col,
                         const double *val, int nleaf, const int32_t *perm,
                         const int32_t *leaf_ptr) {
    int *clu = (int *)xcalloc((size_t)n, sizeof(int));
    int *loc = (int *)xcalloc((size_t)n, sizeof(int));
    int c, k;
    m->nc = nleaf;
    m->size = (int *)xcalloc((size_t)nleaf, sizeof(int));
    m->rows = (brow *)xcalloc((size_t)nleaf, sizeof(brow));
    for (c = 0; c < nleaf; c++) {
        m->size[c] = leaf_ptr[c + 1] - leaf_ptr[c];
        for (k = leaf_ptr[c]; k < leaf_ptr[c + 1]; k++) {
            clu[perm[k]] = c;
            loc[perm[k]] = k - leaf_ptr[c];
        }
    }
    for (c = 0; c < nleaf; c++) {
        for (k = leaf_ptr[c]; k < leaf_ptr[c + 1]; k++) {
            int i = perm[k];
            int64_t e;
            for (e = rowptr[i]; e < rowptr[i + 1]; e++) {
                int j = col[e], q = clu[j];
                blk *b = bensure(m, c, q);
                b->a[(size_t)loc[i] * m->size[q] + loc[j]] += val[e];
            }
        }
        bensure(m, c, c);
    }
    free(clu);
    free(loc);
}

/* A_c of the coarse DOFs: parent P merges children 2P, 2P+1 (Algorithm 1). */
static void build_parent(const bmat *m, bmat *pm) {
    int P, a, t;
    pm->nc = m->nc / 2;
    pm->size = (int *)xcalloc((size_t)pm->nc, sizeof(int));
    pm->rows = (brow *)xcalloc((size_t)pm->nc, sizeof(brow));
    for (P = 0; P < pm->nc; P++) pm->size[P] = m->size[2 * P] + m->size[2 * P + 1];
    for (a = 0; a < m->nc; a++) {
        int P2 = a / 2, ra = m->size[a], oa = (a & 1) ? m->size[a - 1] : 0;
        if (ra == 0) continue;
        for (t = 0; t < m->rows[a].n; t++) {
            int bq = m->rows[a].v[t].q, Q = bq / 2, rb = m->size[bq];
            int ob = (bq & 1) ? m->size[bq - 1] : 0, i, j;
            blk *dst;
            if (rb == 0) continue;
            dst = bensure(pm, P2, Q);
            for (i = 0; i < ra; i++)
                for (j = 0; j < rb; j++)
                    dst->a[(size_t)(oa + i) * pm->size[Q] + ob + j] = m->rows[a].v[t].a[(size_t)i * rb + j];
        }
    }
}

/*
 * Hierarchical_Factor (Algorithm 1) with `depth` levels of scaled low-rank
 * elimination, then dense Cholesky of the remaining coarse system.
 */
int or_factor_create_ex(int64_t n64, const int64_t *rowptr, const int32_t *col,
                        const double *val, int32_t nleaf, const int32_t *perm,
                        const int32_t *leaf_ptr, int32_t depth, double eps, int32_t nodc,
                        int32_t nthreads, or_factor **out, int32_t *fail_level,
                        int32_t *fail_cluster) {
    int n = (int)n64, l, i, c, k, t;
    bmat m;
    or_factor *f;
    *out = NULL;
    if (fail_level) *fail_level = -1;
    if (fail_cluster) *fail_cluster = -1;
    if (n <= 0 || nleaf <= 0 || depth < 0) return OR_ERR_ARG;
    if (depth > 0 && (nleaf % (1 << depth)) != 0) return OR_ERR_ARG;
    f = (or_factor *)xcalloc(1, sizeof(or_factor));
    f->n = n;
    f->depth = depth;
    f->eps = eps;
    f->perm = (int32_t *)xcalloc((size_t)n, sizeof(int32_t));
    memcpy(f->perm, perm, (size_t)n * sizeof(int32_t));
    f->lev = (flevel *)xcalloc((size_t)depth + 1, sizeof(flevel));
    build_level0(&m, n, rowptr, col, val, nleaf, perm, leaf_ptr);
    for (l = 0; l < depth; l++) {
        flevel *lv = &f->lev[l];
        int nc = m.nc, done = 0, ph = 0, nproc = 0;
        int **adj0 = (int **)xcalloc((size_t)nc, sizeof(int *));
        int *nadj0 = (int *)xcalloc((size_t)nc, sizeof(int));
        char *processed = (char *)xcalloc((size_t)nc, 1);
        char *gone = (char *)xcalloc((size_t)nc, 1);
        char *sel = (char *)xcalloc((size_t)nc, 1);
        int *order = (int *)xcalloc((size_t)nc, sizeof(int));
        lv->nc = nc;
        lv->size0 = (int *)xcalloc((size_t)nc, sizeof(int));
        lv->final = (int *)xcalloc((size_t)nc, sizeof(int));
        lv->phase = (int *)xcalloc((size_t)nc, sizeof(int));
        lv->off = (int64_t *)xcalloc((size_t)nc + 1, sizeof(int64_t));
        lv->steps = (fstep *)xcalloc((size_t)nc, sizeof(fstep));
        for (c = 0; c < nc; c++) {
            int t, k2 = 0;
            lv->size0[c] = m.size[c];
            lv->off[c + 1] = lv->off[c] + m.size[c];
            lv->phase[c] = -1;
            adj0[c] = (int *)xcalloc((size_t)m.rows[c].n, sizeof(int));
            for (t = 0; t < m.rows[c].n; t++)
                if (m.rows[c].v[t].q != c) adj0[c][k2++] = m.rows[c].v[t].q;
            nadj0[c] = k2;
            if (m.size[c] == 0) {
                processed[c] = 1; /* empty cluster: nothing to do */
                done++;
            }
        }
        lv->len = lv->off[nc];
        while (done < nc) {
            int cnt = 0;
            memset(sel, 0, (size_t)nc);
            for (c = 0; c < nc; c++) {
                int t, ok = 1;
                if (processed[c]) continue;
                for (t = 0; t < m.rows[c].n; t++)
                    if (sel[m.rows[c].v[t].q]) { ok = 0; break; }
                if (ok) { sel[c] = 1; order[cnt++] = c; }
            }
            {
                /* the phase: every cluster's own computation (in parallel
                 * when threads > 1), the first failure in cluster order
                 * reported; then the Schur updates, target row by target row
                 * (each row's blocks in ascending cluster order); then the
                 * write-backs in cluster order */
                cwork *wk = (cwork *)xcalloc((size_t)cnt + 1, sizeof(cwork));
                int *rcs = (int *)xcalloc((size_t)cnt + 1, sizeof(int));
                int fail = -1, nrow = 0, *rp, *rlist, *rpos, *tp;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
                for (i = 0; i < cnt; i++)
                    rcs[i] = cluster_compute(&m, order[i], adj0[order[i]], nadj0[order[i]], eps, nodc,
                                             &lv->steps[nproc + i], &wk[i]);
                for (i = 0; i < cnt && fail < 0; i++)
                    if (rcs[i]) fail = i;
                if (fail >= 0) {
                    int rc = rcs[fail];
                    if (fail_level) *fail_level = l;
                    if (fail_cluster) *fail_cluster = order[fail];
                    lv->nsteps = nproc + cnt; /* freed with the factor */
                    for (i = 0; i < cnt; i++) cwork_free(&wk[i]);
                    free(wk); free(rcs);
                    for (c = 0; c < nc; c++) free(adj0[c]);
                    free(adj0); free(nadj0); free(processed); free(gone); free(sel); free(order);
                    bfree(&m);
                    f->depth = l + 1;
                    or_factor_free(f);
                    return rc;
                }
                for (i = 0; i < cnt; i++) cluster_schur_blocks(&m, &wk[i]);
                /* per target row p: the (step, position of p) pairs, ascending step */
                rp = (int *)xcalloc((size_t)nc + 1, sizeof(int));
                for (i = 0; i < cnt; i++)
                    for (t = 0; t < wk[i].nn; t++) rp[wk[i].nl[t] + 1]++;
                for (c = 0; c < nc; c++) rp[c + 1] += rp[c];
                rlist = (int *)xcalloc((size_t)rp[nc] + 1, sizeof(int));
                rpos = (int *)xcalloc((size_t)rp[nc] + 1, sizeof(int));
                tp = (int *)xcalloc((size_t)nc + 1, sizeof(int));
                memcpy(tp, rp, (size_t)nc * sizeof(int));
                for (i = 0; i < cnt; i++)
                    for (t = 0; t < wk[i].nn; t++) {
                        int p = wk[i].nl[t];
                        rlist[tp[p]] = i;
                        rpos[tp[p]++] = t;
                    }
                for (c = 0; c < nc; c++)
                    if (rp[c + 1] > rp[c]) tp[nrow++] = c;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
                for (k = 0; k < nrow; k++) {
                    int e, p = tp[k];
                    for (e = rp[p]; e < rp[p + 1]; e++)
                        cluster_schur_row(&m, &lv->steps[nproc + rlist[e]], &wk[rlist[e]], rpos[e]);
                }
                for (i = 0; i < cnt; i++) {
                    cluster_writeback(&m, order[i], &lv->steps[nproc + i], &wk[i], gone);
                    processed[order[i]] = 1;
                    lv->phase[order[i]] = ph;
                    done++;
                    cwork_free(&wk[i]);
                }
                nproc += cnt;
                free(wk); free(rcs); free(rp); free(rlist); free(rpos); free(tp);
            }
            ph++;
        }
        lv->nsteps = nproc;
        lv->nphases = ph;
        for (c = 0; c < nc; c++) lv->final[c] = m.size[c];
        for (c = 0; c < nc; c++) free(adj0[c]);
        free(adj0); free(nadj0); free(processed); free(gone); free(sel); free(order);
        {
            bmat pm;
            build_parent(&m, &pm);
            bfree(&m);
            m = pm;
        }
    }
    /* top: dense Cholesky of the remaining coarse system */
    f->ntop_c = m.nc;
    f->top_size = (int *)xcalloc((size_t)m.nc, sizeof(int));
    f->top_off = (int64_t *)xcalloc((size_t)m.nc + 1, sizeof(int64_t));
    for (c = 0; c < m.nc; c++) {
        f->top_size[c] = m.size[c];
        f->top_off[c + 1] = f->top_off[c] + m.size[c];
    }
    f->ntop = (int)f->top_off[m.nc];
    f->Ltop = (double *)xcalloc((size_t)f->ntop * (size_t)f->ntop, sizeof(double));
    for (c = 0; c < m.nc; c++) {
        int t;
        for (t = 0; t < m.rows[c].n; t++) {
            int q = m.rows[c].v[t].q, ii, jj;
            for (ii = 0; ii < m.size[c]; ii++)
                for (jj = 0; jj < m.size[q]; jj++)
                    f->Ltop[(size_t)(f->top_off[c] + ii) * f->ntop + f->top_off[q] + jj] =
                        m.rows[c].v[t].a[(size_t)ii * m.size[q] + jj];
        }
    }
    bfree(&m);
    if (f->ntop > 0 && chol_lower(f->ntop, f->Ltop)) {
        if (fail_level) *fail_level = depth;
        if (fail_cluster) *fail_cluster = 0;
        or_factor_free(f);
        return OR_ERR_NOT_SPD;
    }
    {
        int64_t bytes = (int64_t)f->ntop * f->ntop * 8;
        for (l = 0; l < depth; l++)
            for (i = 0; i < f->lev[l].nsteps; i++) {
                fstep *st = &f->lev[l].steps[i];
                int64_t fs = st->s - st->r;
                bytes += 8 * ((st->nodc ? fs * fs + fs * st->r : (int64_t)st->s * st->s) +
                              (int64_t)st->s * st->r + fs * st->ncols);
            }
        f->factor_bytes = bytes;
    }
    *out = f;
    return OR_OK;
}

/* Hierarchical_Factor with deferred compression, one thread. */
int or_factor_create(int64_t n64, const int64_t *rowptr, const int32_t *col,
                     const double *val, int32_t nleaf, const int32_t *perm,
                     const int32_t *leaf_ptr, int32_t depth, double eps,
                     or_factor **out, int32_t *fail_level, int32_t *fail_cluster) {
    return or_factor_create_ex(n64, rowptr, col, val, nleaf, perm, leaf_ptr, depth, eps, 0, 1, out,
                               fail_level, fail_cluster);
}

/* ------------------------------------------------------------------------ */
/* Hierarchical_Solve (Algorithm 2)                                         */
/* ------------------------------------------------------------------------ */

static void apply_reflector(int s, const double *V, int k, double tau, double *y) {
    int i;
    double t = 0.0;
    for (i = k; i < s; i++) t += V[(size_t)i * s + k] * y[i];
    t *= tau;
    for (i = k; i < s; i++) y[i] -= t * V[(size_t)i * s + k];
}

/* z = M^-1 r, both in the original ordering. */
void or_apply(const or_factor *f, const double *r, double *z) {
    int l, i, k, t, c;
    double **y = (double **)xcalloc((size_t)f->depth + 1, sizeof(double *));
    int64_t len0 = f->depth > 0 ? f->lev[0].len : f->ntop;
    y[0] = (double *)xcalloc((size_t)len0 + 1, sizeof(double));
    for (i = 0; i < f->n; i++) y[0][i] = r[f->perm[i]];
    /* forward: y <- W_i y for every cluster, level by level */
    for (l = 0; l < f->depth; l++) {
        const flevel *lv = &f->lev[l];
        double *yl = y[l];
        int64_t nlen;
        for (t = 0; t < lv->nsteps; t++) {
            const fstep *st = &lv->steps[t];
            double *ys = yl + lv->off[st->c];
            int oc = 0, u;
            if (st->nodc) {
                /* rotate by U^T, then eliminate f: y_f <- G_f^-1 y_f,
                 * y_c <- y_c - K_c^T y_f (y_n below, with C = K_n) */
                int f = st->s - st->r, j;
                for (k = 0; k < st->r; k++) apply_reflector(st->s, st->V, k, st->tau[k], ys);
                lower_solve_vec(f, st->Gf, ys + st->r);
                for (j = 0; j < st->r; j++) {
                    double acc = 0.0;
                    for (k = 0; k < f; k++) acc += st->Kc[(size_t)k * st->r + j] * ys[st->r + k];
                    ys[j] -= acc;
                }
            } else {
                lower_solve_vec(st->s, st->G, ys);
                for (k = 0; k < st->r; k++) apply_reflector(st->s, st->V, k, st->tau[k], ys);
            }
            for (u = 0; u < st->nn; u++) {
                double *yq = yl + lv->off[st->nq[u]];
                int j;
                for (j = 0; j < st->nm[u]; j++) {
                    double acc = 0.0;
                    for (k = 0; k < st->s - st->r; k++) acc += st->C[(size_t)k * st->ncols + oc + j] * ys[st->r + k];
                    yq[j] -= acc;
                }
                oc += st->nm[u];
            }
        }
        /* gather the coarse parts into the parent ordering */
        nlen = 0;
        for (c = 0; c < lv->nc; c++) nlen += lv->final[c];
        y[l + 1] = (double *)xcalloc((size_t)nlen + 1, sizeof(double));
        {
            int64_t o = 0;
            for (c = 0; c < lv->nc; c++) {
                memcpy(y[l + 1] + o, yl + lv->off[c], (size_t)lv->final[c] * sizeof(double));
                o += lv->final[c];
            }
        }
    }
    /* top: dense solve */
    if (f->ntop > 0) {
        lower_solve_vec(f->ntop, f->Ltop, y[f->depth]);
        lower_t_solve_vec(f->ntop, f->Ltop, y[f->depth]);
    }
    /* backward: x <- W_i^T x in reverse */
    for (l = f->depth - 1; l >= 0; l--) {
        const flevel *lv = &f->lev[l];
        double *yl = y[l];
        {
            int64_t o = 0;
            for (c = 0; c < lv->nc; c++) {
                memcpy(yl + lv->off[c], y[l + 1] + o, (size_t)lv->final[c] * sizeof(double));
                o += lv->final[c];
            }
        }
        for (t = lv->nsteps - 1; t >= 0; t--) {
            const fstep *st = &lv->steps[t];
            double *ys = yl + lv->off[st->c];
            int oc = 0, u;
            for (u = 0; u < st->nn; u++) {
                const double *yq = yl + lv->off[st->nq[u]];
                int j;
                for (k = 0; k < st->s - st->r; k++) {
                    double acc = 0.0;
                    for (j = 0; j < st->nm[u]; j++) acc += st->C[(size_t)k * st->ncols + oc + j] * yq[j];
                    ys[st->r + k] -= acc;
                }
                oc += st->nm[u];
            }
            if (st->nodc) {
                /* x_f <- G_f^-T (x_f - K_c x_c), then rotate back by U */
                int f = st->s - st->r, j;
                for (k = 0; k < f; k++) {
                    double acc = 0.0;
                    for (j = 0; j < st->r; j++) acc += st->Kc[(size_t)k * st->r + j] * ys[j];
                    ys[st->r + k] -= acc;
                }
                lower_t_solve_vec(f, st->Gf, ys + st->r);
                for (k = st->r - 1; k >= 0; k--) apply_reflector(st->s, st->V, k, st->tau[k], ys);
            } else {
                for (k = st->r - 1; k >= 0; k--) apply_reflector(st->s, st->V, k, st->tau[k], ys);
                lower_t_solve_vec(st->s, st->G, ys);
            }
        }
        free(y[l + 1]);
    }
    for (i = 0; i < f->n; i++) z[f->perm[i]] = y[0][i];
    free(y[0]);
    free(y);
}

/* ------------------------------------------------------------------------ */
/* Krylov (Sec. 5)                                                          */
/* ------------------------------------------------------------------------ */

static void spmv(int n, const int64_t *rowptr, const int32_t *col, const double *val,
                 const double *x, double *y) {
    int i;
    for (i = 0; i < n; i++) {
        double t = 0.0;
        int64_t e;
        for (e = rowptr[i]; e < rowptr[i + 1]; e++) t += val[e] * x[col[e]];
        y[i] = t;
    }
}

static double dot(int n, const double *a, const double *b) {
    double t = 0.0;
    int i;
    for (i = 0; i < n; i++) t += a[i] * b[i];
    return t;
}

/*
 * Preconditioned CG, x0 = 0.  Stops when ||r||/||b|| <= rtol on the
 * recurrence residual and the true residual confirms it; otherwise the true
 * residual replaces the recurrence one and CG restarts.  iters = CG steps.
 */
int or_pcg(int64_t n64, const int64_t *rowptr, const int32_t *col, const double *val,
           const or_factor *f, const double *b, double *x, double rtol, int32_t maxit,
           int32_t *iters, double *relres) {
    int n = (int)n64, it = 0, i;
    double *r = (double *)xcalloc((size_t)n, sizeof(double));
    double *z = (double *)xcalloc((size_t)n, sizeof(double));
    double *p = (double *)xcalloc((size_t)n, sizeof(double));
    double *q = (double *)xcalloc((size_t)n, sizeof(double));
    double bn = sqrt(dot(n, b, b)), rz, rn;
    int rc = OR_ERR_NOCONV;
    for (i = 0; i < n; i++) { x[i] = 0.0; r[i] = b[i]; }
    if (bn == 0.0) {
        *iters = 0; *relres = 0.0;
        free(r); free(z); free(p); free(q);
        return OR_OK;
    }
    or_apply(f, r, z);
    memcpy(p, z, (size_t)n * sizeof(double));
    rz = dot(n, r, z);
    rn = bn;
    while (it < maxit) {
        double alpha, rzn, beta;
        spmv(n, rowptr, col, val, p, q);
        alpha = rz / dot(n, p, q);
        for (i = 0; i < n; i++) { x[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
        it++;
        rn = sqrt(dot(n, r, r));
        if (rn / bn <= rtol) {
            spmv(n, rowptr, col, val, x, q);
            for (i = 0; i < n; i++) q[i] = b[i] - q[i];
            rn = sqrt(dot(n, q, q));
            if (rn / bn <= rtol) { rc = OR_OK; break; }
            memcpy(r, q, (size_t)n * sizeof(double));
            or_apply(f, r, z);
            memcpy(p, z, (size_t)n * sizeof(double));
            rz = dot(n, r, z);
            continue;
        }
        or_apply(f, r, z);
        rzn = dot(n, r, z);
        beta = rzn / rz;
        rz = rzn;
        for (i = 0; i < n; i++) p[i] = z[i] + beta * p[i];
    }
    *iters = it;
    *relres = rn / bn;
    free(r); free(z); free(p); free(q);
    return rc;
}

/*
 * Right-preconditioned restarted GMRES(m), x0 = 0; each restart recomputes the
 * FP64 true residual (iterative refinement).  iters = inner steps in total.
 */
int or_gmres(int64_t n64, const int64_t *rowptr, const int32_t *col, const double *val,
             const or_factor *f, const double *b, double *x, double rtol, int32_t m,
             int32_t maxit, int32_t *iters, double *relres) {
    int n = (int)n64, it = 0, i, j, k;
    double bn = sqrt(dot(n, b, b)), rn;
    double *V = (double *)xcalloc((size_t)(m + 1) * n, sizeof(double));
    double *Z = (double *)xcalloc((size_t)m * n, sizeof(double));
    double *H = (double *)xcalloc((size_t)(m + 1) * m, sizeof(double));
    double *cs = (double *)xcalloc((size_t)m, sizeof(double));
    double *sn = (double *)xcalloc((size_t)m, sizeof(double));
    double *g = (double *)xcalloc((size_t)m + 1, sizeof(double));
    double *w = (double *)xcalloc((size_t)n, sizeof(double));
    double *yv = (double *)xcalloc((size_t)m, sizeof(double));
    int rc = OR_ERR_NOCONV;
    for (i = 0; i < n; i++) x[i] = 0.0;
    if (bn == 0.0) { *iters = 0; *relres = 0.0; rc = OR_OK; goto done; }
    for (;;) {
        double beta;
        int kk;
        spmv(n, rowptr, col, val, x, w);
        for (i = 0; i < n; i++) w[i] = b[i] - w[i];
        beta = sqrt(dot(n, w, w));
        rn = beta;
        if (beta / bn <= rtol) { rc = OR_OK; break; }
        if (it >= maxit) break;
        for (i = 0; i < n; i++) V[i] = w[i] / beta;
        memset(g, 0, (size_t)(m + 1) * sizeof(double));
        g[0] = beta;
        kk = 0;
        for (j = 0; j < m && it < maxit; j++) {
            double hn, t;
            or_apply(f, V + (size_t)j * n, Z + (size_t)j * n);
            spmv(n, rowptr, col, val, Z + (size_t)j * n, w);
            for (k = 0; k <= j; k++) {  /* modified Gram-Schmidt */
                double h = dot(n, w, V + (size_t)k * n);
                H[k * m + j] = h;
                for (i = 0; i < n; i++) w[i] -= h * V[(size_t)k * n + i];
            }
            hn = sqrt(dot(n, w, w));
            H[(j + 1) * m + j] = hn;
            if (hn > 0.0)
                for (i = 0; i < n; i++) V[(size_t)(j + 1) * n + i] = w[i] / hn;
            for (k = 0; k < j; k++) {   /* previous Givens rotations */
                double a = H[k * m + j], c2 = H[(k + 1) * m + j];
                H[k * m + j] = cs[k] * a + sn[k] * c2;
                H[(k + 1) * m + j] = -sn[k] * a + cs[k] * c2;
            }
            {
                double a = H[j * m + j], c2 = H[(j + 1) * m + j];
                double d = sqrt(a * a + c2 * c2);
                cs[j] = d > 0.0 ? a / d : 1.0;
                sn[j] = d > 0.0 ? c2 / d : 0.0;
                H[j * m + j] = d;
                H[(j + 1) * m + j] = 0.0;
                t = g[j];
                g[j] = cs[j] * t;
                g[j + 1] = -sn[j] * t;
            }
            it++;
            kk = j + 1;
            if (fabs(g[j + 1]) / bn <= rtol || hn == 0.0) break;
        }
        for (k = kk - 1; k >= 0; k--) {
            double t = g[k];
            for (j = k + 1; j < kk; j++) t -= H[k * m + j] * yv[j];
            yv[k] = t / H[k * m + k];
        }
        for (k = 0; k < kk; k++)
            for (i = 0; i < n; i++) x[i] += yv[k] * Z[(size_t)k * n + i];
    }
    *iters = it;
    *relres = rn / bn;
done:
    free(V); free(Z); free(H); free(cs); free(sn); free(g); free(w); free(yv);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Introspection for the tests                                              */
/* ------------------------------------------------------------------------ */

int32_t or_depth(const or_factor *f) { return f->depth; }
int32_t or_top_n(const or_factor *f) { return f->ntop; }
int64_t or_factor_bytes(const or_factor *f) { return f->factor_bytes; }
int32_t or_level_nc(const or_factor *f, int32_t l) { return f->lev[l].nc; }
int32_t or_level_nphases(const or_factor *f, int32_t l) { return f->lev[l].nphases; }

/* per cluster of level l: start size, final size (rank or 0), phase */
void or_level_info(const or_factor *f, int32_t l, int32_t *size0, int32_t *final,
                   int32_t *phase) {
    int c;
    for (c = 0; c < f->lev[l].nc; c++) {
        size0[c] = f->lev[l].size0[c];
        final[c] = f->lev[l].final[c];
        phase[c] = f->lev[l].phase[c];
    }
}

/* processing order of level l and each step's rank */
void or_level_steps(const or_factor *f, int32_t l, int32_t *cluster, int32_t *rank) {
    int t;
    for (t = 0; t < f->lev[l].nsteps; t++) {
        cluster[t] = f->lev[l].steps[t].c;
        rank[t] = f->lev[l].steps[t].r;
    }
}

int32_t or_level_nsteps(const or_factor *f, int32_t l) { return f->lev[l].nsteps; }

/* ------------------------------------------------------------------------ */
/* Dense entry points for the pins                                          */
/* ------------------------------------------------------------------------ */

int or_dense_chol(int32_t n, double *a) { return chol_lower(n, a) ? OR_ERR_NOT_SPD : OR_OK; }

void or_dense_lower_solve(int32_t n, const double *g, int32_t m, double *b) { lower_solve(n, g, m, b); }

/* CPQR of the whole s x w matrix M (no n part); returns rank, V, tau, piv. */
int32_t or_dense_cpqr(int32_t s, int32_t w, double *M, double eps, double *V, double *tau,
                      int32_t *piv) {
    return cpqr_apply(s, 0, w, M, eps, V, tau, piv);
}

/*
 * One scaled low-rank elimination on a dense SPD matrix ordered (s, n, w)
 * with sizes (s, nn, nw): returns, in out (d x d, d = r + nn + nw), the
 * matrix on (coarse DOFs, n, w) that the factorization keeps after the step
 * (Sec. 3.1): [[I, U1^T G^-1 A_sn, V1^T], [., X_nn, A_nw], [., A_wn, A_ww]].
 * out must hold (s + nn + nw)^2 doubles.  Returns the rank, or -1 if A_ss is
 * not SPD.
 */
int32_t or_dense_step(int32_t s, int32_t nn, int32_t nw, const double *A, double eps,
                      double *out) {
    int N = s + nn + nw, W = nn + nw, i, j, k, r, d;
    double *Ass = (double *)xcalloc((size_t)s * s, sizeof(double));
    double *M = (double *)xcalloc((size_t)s * W, sizeof(double));
    double *V = (double *)xcalloc((size_t)s * s, sizeof(double));
    double *tau = (double *)xcalloc((size_t)s + 1, sizeof(double));
    double *R = (double *)xcalloc((size_t)W * W, sizeof(double));
    for (i = 0; i < s; i++)
        for (j = 0; j < s; j++) Ass[i * s + j] = A[i * N + j];
    for (i = 0; i < s; i++)
        for (j = 0; j < W; j++) M[i * W + j] = A[i * N + s + j];
    if (step_core(s, nn, nw, Ass, M, eps, V, tau, &r)) {
        free(Ass); free(M); free(V); free(tau); free(R);
        return -1;
    }
    /* remaining block: A on (n, w) minus the fine elimination on n x n */
    for (i = 0; i < W; i++)
        for (j = 0; j < W; j++) R[i * W + j] = A[(s + i) * N + s + j];
    for (i = 0; i < nn; i++)
        for (j = 0; j < nn; j++) {
            double acc = 0.0;
            for (k = r; k < s; k++) acc += M[k * W + i] * M[k * W + j];
            R[i * W + j] -= acc;
        }
    d = r + W;
    for (i = 0; i < d * d; i++) out[i] = 0.0;
    for (i = 0; i < r; i++) out[i * d + i] = 1.0;
    for (i = 0; i < r; i++)
        for (j = 0; j < W; j++) {
            out[i * d + r + j] = M[i * W + j];
            out[(r + j) * d + i] = M[i * W + j];
        }
    for (i = 0; i < W; i++)
        for (j = 0; j < W; j++) out[(r + i) * d + r + j] = R[i * W + j];
    free(Ass); free(M); free(V); free(tau); free(R);
    return r;
}

/*
 * The same step without deferred compression (step_nodc, as the level loop
 * runs it) on a dense (s, n, w) matrix; out (d x d, d = r + nn + nw) is the
 * matrix on (coarse DOFs, n, w) afterwards: the coarse block left by
 * eliminating the fine DOFs, its coupling to n and V_1^T to w, A_nn minus
 * the fine elimination, A_nw, A_ww.  Returns the rank, or -1 if not SPD.
 */
int32_t or_dense_step_nodc(int32_t s, int32_t nn, int32_t nw, const double *A, double eps,
                           double *out) {
    int N = s + nn + nw, W = nn + nw, i, j, k, r, d, f;
    double *Ass = (double *)xcalloc((size_t)s * s, sizeof(double));
    double *M = (double *)xcalloc((size_t)s * W + 1, sizeof(double));
    double *Acc = NULL;
    fstep st;
    memset(&st, 0, sizeof(st));
    st.V = (double *)xcalloc((size_t)s * s, sizeof(double));
    st.tau = (double *)xcalloc((size_t)s + 1, sizeof(double));
    for (i = 0; i < s; i++)
        for (j = 0; j < s; j++) Ass[i * s + j] = A[i * N + j];
    for (i = 0; i < s; i++)
        for (j = 0; j < W; j++) M[i * W + j] = A[i * N + s + j];
    if (step_nodc(s, nn, nw, Ass, M, eps, &st, &Acc)) {
        free(Ass); free(M); free(Acc); step_free(&st);
        return -1;
    }
    r = st.r;
    f = s - r;
    d = r + W;
    for (i = 0; i < d * d; i++) out[i] = 0.0;
    for (i = 0; i < r; i++)
        for (j = 0; j < r; j++) out[i * d + j] = Acc[i * r + j];
    for (i = 0; i < r; i++)
        for (j = 0; j < W; j++) {
            out[i * d + r + j] = M[i * W + j];
            out[(r + j) * d + i] = M[i * W + j];
        }
    for (i = 0; i < W; i++)
        for (j = 0; j < W; j++) {
            double acc = 0.0;
            if (i < nn && j < nn)
                for (k = 0; k < f; k++) acc += st.C[(size_t)k * nn + i] * st.C[(size_t)k * nn + j];
            out[(r + i) * d + r + j] = A[(s + i) * N + s + j] - acc;
        }
    free(Ass); free(M); free(Acc); step_free(&st);
    return r;
}

/* ------------------------------------------------------------------------ */
/* Symbolic plan of one level (the phase rule and the fill pattern alone)   */
/* ------------------------------------------------------------------------ */

typedef struct {
    int *v;
    int n, cap;
} ilist;

static int il_find(const ilist *l, int x) { /* index of x, or -1 */
    int i;
    for (i = 0; i < l->n; i++)
        if (l->v[i] == x) return i;
    return -1;
}

static void il_add(ilist *l, int x) { /* sorted insert if absent */
    int i;
    if (il_find(l, x) >= 0) return;
    if (l->n == l->cap) {
        int *nv;
        l->cap = l->cap ? 2 * l->cap : 8;
        nv = (int *)xcalloc((size_t)l->cap, sizeof(int));
        if (l->n) memcpy(nv, l->v, (size_t)l->n * sizeof(int));
        free(l->v);
        l->v = nv;
    }
    i = l->n;
    while (i > 0 && l->v[i - 1] > x) {
        l->v[i] = l->v[i - 1];
        i--;
    }
    l->v[i] = x;
    l->n++;
}

static void il_remove(ilist *l, int x) {
    int i = il_find(l, x);
    if (i < 0) return;
    for (; i + 1 < l->n; i++) l->v[i] = l->v[i + 1];
    l->n--;
}

/*
 * The level plan of or_factor_create without the arithmetic: the block graph
 * over nc clusters (adj: symmetric CSR without self loops; a cluster of size
 * 0 has no blocks), phases by the phase rule, clusters of a phase eliminated
 * one at a time in ascending order.  Eliminating c couples every pair of its
 * neighbours in the level's input graph (Eq. elim); when none of c's blocks
 * is fill, c has rank 0 and leaves the graph.  Out: phase (-1 for size 0),
 * vanished, the blocks present at the end of the level (end_ptr[nc+1];
 * end_adj, sorted per cluster, with the cluster itself unless it left or has
 * size 0) and every block that existed at some point of the level (all_ptr,
 * all_adj: sorted, with the cluster itself unless it has size 0).  A NULL
 * list queries the size (the pointer array is filled either way).
 */
int or_plan_level(int32_t nc, const int64_t *adj_ptr, const int32_t *adj, const int32_t *size0,
                  int32_t *phase, int32_t *vanished, int64_t *end_ptr, int32_t *end_adj,
                  int64_t end_cap, int64_t *all_ptr, int32_t *all_adj, int64_t all_cap) {
    ilist *cur = (ilist *)xcalloc((size_t)nc + 1, sizeof(ilist));
    ilist *ever = (ilist *)xcalloc((size_t)nc + 1, sizeof(ilist));
    char *processed = (char *)xcalloc((size_t)nc + 1, 1);
    char *sel = (char *)xcalloc((size_t)nc + 1, 1);
    int *order = (int *)xcalloc((size_t)nc + 1, sizeof(int));
    int *nb = NULL;
    int c, done = 0, ph = 0, rc = OR_OK;
    int64_t e, tot = 0;
    for (c = 0; c < nc; c++) {
        for (e = adj_ptr[c]; e < adj_ptr[c + 1]; e++) {
            il_add(&cur[c], adj[e]);
            il_add(&ever[c], adj[e]);
        }
        if (size0[c] > 0) il_add(&ever[c], c);
        phase[c] = -1;
        vanished[c] = 0;
        if (size0[c] == 0) {
            processed[c] = 1;
            done++;
        }
    }
    nb = (int *)xcalloc((size_t)nc + 1, sizeof(int));
    while (done < nc) {
        int cnt = 0, i;
        memset(sel, 0, (size_t)nc);
        for (c = 0; c < nc; c++) {
            int t, ok = 1;
            if (processed[c]) continue;
            for (t = 0; t < cur[c].n; t++)
                if (sel[cur[c].v[t]]) { ok = 0; break; }
            if (ok) { sel[c] = 1; order[cnt++] = c; }
        }
        for (i = 0; i < cnt; i++) {
            int pi = order[i], nn = 0, nw = 0, t, a, b;
            /* n: current neighbours that are blocks of the input graph; w: fill */
            for (t = 0; t < cur[pi].n; t++) {
                int q = cur[pi].v[t], in0 = 0;
                for (e = adj_ptr[pi]; e < adj_ptr[pi + 1]; e++)
                    if (adj[e] == q) in0 = 1;
                if (in0) nb[nn++] = q;
                else nw++;
            }
            for (a = 0; a < nn; a++)
                for (b = 0; b < nn; b++)
                    if (a != b) {
                        il_add(&cur[nb[a]], nb[b]);
                        il_add(&ever[nb[a]], nb[b]);
                    }
            if (nw == 0) {
                vanished[pi] = 1;
                for (t = 0; t < cur[pi].n; t++) il_remove(&cur[cur[pi].v[t]], pi);
                cur[pi].n = 0;
            }
            processed[pi] = 1;
            phase[pi] = ph;
            done++;
        }
        ph++;
    }
    for (c = 0; c < nc; c++) {
        if (size0[c] > 0 && !vanished[c]) il_add(&cur[c], c);
        end_ptr[c] = tot;
        tot += cur[c].n;
    }
    end_ptr[nc] = tot;
    if (end_adj) {
        if (end_cap < tot) rc = OR_ERR_ARG;
        else
            for (c = 0; c < nc; c++)
                if (cur[c].n) memcpy(end_adj + end_ptr[c], cur[c].v, (size_t)cur[c].n * sizeof(int));
    }
    tot = 0;
    for (c = 0; c < nc; c++) {
        all_ptr[c] = tot;
        tot += ever[c].n;
    }
    all_ptr[nc] = tot;
    if (all_adj) {
        if (all_cap < tot) rc = OR_ERR_ARG;
        else
            for (c = 0; c < nc; c++)
                if (ever[c].n) memcpy(all_adj + all_ptr[c], ever[c].v, (size_t)ever[c].n * sizeof(int));
    }
    for (c = 0; c < nc; c++) {
        free(cur[c].v);
        free(ever[c].v);
    }
    free(cur); free(ever); free(processed); free(sel); free(order); free(nb);
    return rc;
}
