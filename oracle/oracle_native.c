/*
 * Oracle (test infrastructure only): plain, slow, obviously-correct FP64 CPU
 * routines for the graph reordering, the incomplete LU factorisation and the
 * triangular sweeps of Nation, Johansson, Blencowe & Rimberg,
 * "Iterative solutions to the steady state density matrix for optomechanical
 * systems" (arXiv:1411.4356).
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg may load
 * this code.  It shares nothing with the CUDA library under
 * paper_1411_4356_gb300/csrc and must never be linked into it.
 *
 * Matrices are CSR: int64 row pointers, int32 column indices and complex128
 * values stored as interleaved (re, im) doubles.  Row entries must be sorted by
 * column on input; outputs are sorted by column too.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* ------------------------------------------------------------------------ */
/* Cuthill-McKee / reverse Cuthill-McKee (Sec. III).                        */
/*                                                                          */
/* The paper: breadth-first search from a node of lowest degree, the degree */
/* of node i being the number of nonzeros in row i of the symmetric matrix, */
/* visiting the neighbours of each node from lowest to highest degree;      */
/* repeated per connected component; the CM order is then reversed.         */
/* Ties the paper leaves open are broken by the node index: the start node  */
/* of each component is the unvisited node with the smallest (degree,       */
/* index), and a node's unvisited neighbours are appended in increasing     */
/* (degree, index) order.  perm[new] = old.                                 */
/* ------------------------------------------------------------------------ */

static const int64_t *g_deg; /* degree table seen by the comparator */

static int cmp_deg_index(const void *pa, const void *pb) {
    int32_t a = *(const int32_t *)pa, b = *(const int32_t *)pb;
    if (g_deg[a] != g_deg[b]) return g_deg[a] < g_deg[b] ? -1 : 1;
    return (a > b) - (a < b);
}

/* ptr/idx: CSR of the SYMMETRIC pattern (structure of A + A^T).
 * Returns 0 on success, -1 on allocation failure. */
int oracle_rcm(int64_t n, const int64_t *ptr, const int32_t *idx, int32_t *perm) {
    int64_t *deg = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int32_t *by_degree = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    unsigned char *visited = (unsigned char *)calloc((size_t)(n > 0 ? n : 1), 1);
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    if (!deg || !by_degree || !visited || !order) {
        free(deg); free(by_degree); free(visited); free(order);
        return -1;
    }
    for (int64_t i = 0; i < n; ++i) {
        deg[i] = ptr[i + 1] - ptr[i];
        by_degree[i] = (int32_t)i;
    }
    g_deg = deg;
    qsort(by_degree, (size_t)n, sizeof(int32_t), cmp_deg_index);

    int64_t tail = 0; /* number of nodes placed in CM order so far */
    for (int64_t s = 0; s < n; ++s) {
        int32_t start = by_degree[s];
        if (visited[start]) continue;
        /* new connected component */
        visited[start] = 1;
        order[tail++] = start;
        int64_t head = tail - 1;
        while (head < tail) {
            int32_t u = order[head++];
            int64_t first_child = tail;
            for (int64_t e = ptr[u]; e < ptr[u + 1]; ++e) {
                int32_t v = idx[e];
                if (!visited[v]) {
                    visited[v] = 1;
                    order[tail++] = v;
                }
            }
            /* children of u in increasing (degree, index) */
            qsort(order + first_child, (size_t)(tail - first_child), sizeof(int32_t),
                  cmp_deg_index);
        }
    }
    /* reverse the Cuthill-McKee order */
    for (int64_t i = 0; i < n; ++i) perm[i] = order[n - 1 - i];
    free(deg); free(by_degree); free(visited); free(order);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* ILUT(d, p): dual-threshold incomplete LU (Sec. II, the iLUTP paragraph), */
/* computed row by row in the i-k-j order of Saad's ILUT.                   */
/*                                                                          */
/* Readings of the paper used here:                                         */
/*  - every entry of a factor row (original or fill) whose modulus is below */
/*    d * ||row i of A||_inf is dropped; the diagonal is never dropped.     */
/*    (Sec. IV: the 1e-15 thermal entries, which are original entries, are  */
/*    absent from the preconditioner.)                                      */
/*  - the fill cap p * NNZ(A) is honoured row by row: the strict L part of  */
/*    row i keeps at most floor(p*nnz_i/2) entries, and the U part (the     */
/*    diagonal included) at most floor(p*nnz_i/2); the largest moduli win,  */
/*    ties go to the smaller column.                                        */
/*  - no pivoting: after the reordering every diagonal of the augmented     */
/*    Liouvillian is nonzero.  A diagonal of U smaller than                 */
/*    1e-14 * ||row i of A||_inf is replaced by that value (a guard) and    */
/*    counted in *n_guarded.                                                */
/* L is unit lower triangular and stored without its diagonal.  U rows are  */
/* stored with the diagonal first (it is the smallest column >= i).          */
/* The caller provides capacity sum_i floor(p*nnz_i/2) for each factor.      */
/* Returns 0, or -1 on allocation failure, or -2 if a capacity is exceeded. */
/* ------------------------------------------------------------------------ */

typedef struct { int32_t col; double mag; } keep_t;

static int cmp_keep(const void *pa, const void *pb) {
    const keep_t *a = (const keep_t *)pa, *b = (const keep_t *)pb;
    if (a->mag != b->mag) return a->mag > b->mag ? -1 : 1; /* larger first */
    return (a->col > b->col) - (a->col < b->col);          /* then smaller column */
}

static int cmp_i32(const void *pa, const void *pb) {
    int32_t a = *(const int32_t *)pa, b = *(const int32_t *)pb;
    return (a > b) - (a < b);
}

/* binary min-heap of column indices */
static void heap_push(int32_t *h, int64_t *len, int32_t v) {
    int64_t i = (*len)++;
    h[i] = v;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (h[p] <= h[i]) break;
        int32_t t = h[p]; h[p] = h[i]; h[i] = t;
        i = p;
    }
}

static int32_t heap_pop(int32_t *h, int64_t *len) {
    int32_t top = h[0];
    h[0] = h[--(*len)];
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, m = i;
        if (l < *len && h[l] < h[m]) m = l;
        if (r < *len && h[r] < h[m]) m = r;
        if (m == i) break;
        int32_t t = h[m]; h[m] = h[i]; h[i] = t;
        i = m;
    }
    return top;
}

int oracle_ilut(int64_t n, const int64_t *ap, const int32_t *ai, const double *ax_,
                double droptol, double fill,
                int64_t cap_l, int64_t *lp, int32_t *li, double *lx_,
                int64_t cap_u, int64_t *up, int32_t *ui, double *ux_,
                int64_t *n_guarded) {
    const cplx *ax = (const cplx *)ax_;
    cplx *lx = (cplx *)lx_;
    cplx *ux = (cplx *)ux_;
    size_t nn = (size_t)(n > 0 ? n : 1);
    cplx *w = (cplx *)calloc(nn, sizeof(cplx));
    unsigned char *present = (unsigned char *)calloc(nn, 1);
    int32_t *cols = (int32_t *)malloc(sizeof(int32_t) * nn); /* columns present in w */
    int32_t *heap = (int32_t *)malloc(sizeof(int32_t) * nn);
    keep_t *cand = (keep_t *)malloc(sizeof(keep_t) * nn);
    int32_t *sel = (int32_t *)malloc(sizeof(int32_t) * nn);
    if (!w || !present || !cols || !heap || !cand || !sel) {
        free(w); free(present); free(cols); free(heap); free(cand); free(sel);
        return -1;
    }
    *n_guarded = 0;
    lp[0] = 0;
    up[0] = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t nnz_i = ap[i + 1] - ap[i];
        double row_inf = 0.0;
        for (int64_t e = ap[i]; e < ap[i + 1]; ++e) {
            double m = cabs(ax[e]);
            if (m > row_inf) row_inf = m;
        }
        double tau = droptol * row_inf;
        int64_t keep_cap = (int64_t)floor(fill * (double)nnz_i / 2.0);
        if (keep_cap < 1) keep_cap = 1;

        /* w := row i of A */
        int64_t ncols = 0, hlen = 0;
        for (int64_t e = ap[i]; e < ap[i + 1]; ++e) {
            int32_t j = ai[e];
            w[j] = ax[e];
            present[j] = 1;
            cols[ncols++] = j;
            if (j < i) heap_push(heap, &hlen, j);
        }
        if (!present[i]) { /* structural zero diagonal: make room for it */
            w[i] = 0.0;
            present[i] = 1;
            cols[ncols++] = (int32_t)i;
        }

        /* eliminate with the rows k < i, in increasing k */
        while (hlen > 0) {
            int32_t k = heap_pop(heap, &hlen);
            cplx wk = w[k] / ux[up[k]]; /* U row k: diagonal first */
            if (cabs(wk) < tau) {
                w[k] = 0.0; /* dropped: no elimination with row k */
                continue;
            }
            w[k] = wk;
            for (int64_t e = up[k] + 1; e < up[k + 1]; ++e) {
                int32_t j = ui[e];
                if (!present[j]) {
                    present[j] = 1;
                    w[j] = 0.0;
                    cols[ncols++] = j;
                    if (j < i) heap_push(heap, &hlen, j);
                }
                w[j] -= wk * ux[e];
            }
        }

        /* drop small entries, then keep the largest ones per part */
        int64_t nl = 0, nu = 0;
        for (int64_t t = 0; t < ncols; ++t) {
            int32_t j = cols[t];
            if (j < i) {
                double m = cabs(w[j]);
                if (w[j] != 0.0 && !(m < tau)) { cand[nl].col = j; cand[nl].mag = m; ++nl; }
            }
        }
        if (nl > keep_cap) {
            qsort(cand, (size_t)nl, sizeof(keep_t), cmp_keep);
            nl = keep_cap;
        }
        for (int64_t t = 0; t < nl; ++t) sel[t] = cand[t].col;
        qsort(sel, (size_t)nl, sizeof(int32_t), cmp_i32);
        if (lp[i] + nl > cap_l) return -2;
        for (int64_t t = 0; t < nl; ++t) {
            li[lp[i] + t] = sel[t];
            lx[lp[i] + t] = w[sel[t]];
        }
        lp[i + 1] = lp[i] + nl;

        for (int64_t t = 0; t < ncols; ++t) {
            int32_t j = cols[t];
            if (j > i) {
                double m = cabs(w[j]);
                if (w[j] != 0.0 && !(m < tau)) { cand[nu].col = j; cand[nu].mag = m; ++nu; }
            }
        }
        if (nu > keep_cap - 1) {
            qsort(cand, (size_t)nu, sizeof(keep_t), cmp_keep);
            nu = keep_cap - 1;
        }
        for (int64_t t = 0; t < nu; ++t) sel[t] = cand[t].col;
        qsort(sel, (size_t)nu, sizeof(int32_t), cmp_i32);
        if (up[i] + 1 + nu > cap_u) return -2;
        cplx piv = w[i];
        double guard = 1e-14 * row_inf;
        if (cabs(piv) < guard || piv == 0.0) {
            piv = guard > 0.0 ? guard : 1e-300;
            ++*n_guarded;
        }
        ui[up[i]] = (int32_t)i;
        ux[up[i]] = piv;
        for (int64_t t = 0; t < nu; ++t) {
            ui[up[i] + 1 + t] = sel[t];
            ux[up[i] + 1 + t] = w[sel[t]];
        }
        up[i + 1] = up[i] + 1 + nu;

        /* clear the work row */
        for (int64_t t = 0; t < ncols; ++t) {
            w[cols[t]] = 0.0;
            present[cols[t]] = 0;
        }
    }
    free(w); free(present); free(cols); free(heap); free(cand); free(sel);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* ILUT(d, p) with the fill cap read as a total: NNZ(L) + NNZ(U) <= p NNZ(A) */
/* (Sec. II), held as a running budget over the rows in elimination order.  */
/* Row i drops as oracle_ilut does, then keeps every surviving entry while  */
/* the entries kept so far, its own included (the diagonal apart), stay     */
/* within floor(p * NNZ(rows 0..i of A)); beyond that it keeps the largest  */
/* moduli that fit (ties: the smaller column).  Where the budget never      */
/* binds, the factors are plain threshold ILU(d).  The caller provides      */
/* capacity floor(p NNZ(A)) + n for each factor.  Same return codes.        */
/* ------------------------------------------------------------------------ */

int oracle_ilut_total(int64_t n, const int64_t *ap, const int32_t *ai, const double *ax_,
                      double droptol, double fill,
                      int64_t cap_l, int64_t *lp, int32_t *li, double *lx_,
                      int64_t cap_u, int64_t *up, int32_t *ui, double *ux_,
                      int64_t *n_guarded) {
    const cplx *ax = (const cplx *)ax_;
    cplx *lx = (cplx *)lx_;
    cplx *ux = (cplx *)ux_;
    size_t nn = (size_t)(n > 0 ? n : 1);
    cplx *w = (cplx *)calloc(nn, sizeof(cplx));
    unsigned char *present = (unsigned char *)calloc(nn, 1);
    int32_t *cols = (int32_t *)malloc(sizeof(int32_t) * nn); /* columns present in w */
    int32_t *heap = (int32_t *)malloc(sizeof(int32_t) * nn);
    keep_t *cand = (keep_t *)malloc(sizeof(keep_t) * nn);
    int32_t *sel = (int32_t *)malloc(sizeof(int32_t) * nn);
    if (!w || !present || !cols || !heap || !cand || !sel) {
        free(w); free(present); free(cols); free(heap); free(cand); free(sel);
        return -1;
    }
    *n_guarded = 0;
    lp[0] = 0;
    up[0] = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t nnz_i = ap[i + 1] - ap[i];
        double row_inf = 0.0;
        for (int64_t e = ap[i]; e < ap[i + 1]; ++e) {
            double m = cabs(ax[e]);
            if (m > row_inf) row_inf = m;
        }
        double tau = droptol * row_inf;
        int64_t keep_cap = (int64_t)floor(fill * (double)nnz_i / 2.0);
        if (keep_cap < 1) keep_cap = 1;

        /* w := row i of A */
        int64_t ncols = 0, hlen = 0;
        for (int64_t e = ap[i]; e < ap[i + 1]; ++e) {
            int32_t j = ai[e];
            w[j] = ax[e];
            present[j] = 1;
            cols[ncols++] = j;
            if (j < i) heap_push(heap, &hlen, j);
        }
        if (!present[i]) { /* structural zero diagonal: make room for it */
            w[i] = 0.0;
            present[i] = 1;
            cols[ncols++] = (int32_t)i;
        }

        /* eliminate with the rows k < i, in increasing k */
        while (hlen > 0) {
            int32_t k = heap_pop(heap, &hlen);
            cplx wk = w[k] / ux[up[k]]; /* U row k: diagonal first */
            if (cabs(wk) < tau) {
                w[k] = 0.0; /* dropped: no elimination with row k */
                continue;
            }
            w[k] = wk;
            for (int64_t e = up[k] + 1; e < up[k + 1]; ++e) {
                int32_t j = ui[e];
                if (!present[j]) {
                    present[j] = 1;
                    w[j] = 0.0;
                    cols[ncols++] = j;
                    if (j < i) heap_push(heap, &hlen, j);
                }
                w[j] -= wk * ux[e];
            }
        }

        /* drop small entries; then, if the running budget is exceeded, keep the
           largest ones of the row (L and U parts together, the diagonal apart) */
        int64_t nc = 0;
        for (int64_t t = 0; t < ncols; ++t) {
            int32_t j = cols[t];
            if (j == i) continue;
            double m = cabs(w[j]);
            if (w[j] != 0.0 && !(m < tau)) { cand[nc].col = j; cand[nc].mag = m; ++nc; }
        }
        int64_t budget = (int64_t)floor(fill * (double)ap[i + 1]) - (lp[i] + up[i]) - 1; /* off-diagonals */
        if (budget < 0) budget = 0;
        if (nc > budget) {
            qsort(cand, (size_t)nc, sizeof(keep_t), cmp_keep);
            nc = budget;
        }
        int64_t nl = 0, nu = 0;
        for (int64_t t = 0; t < nc; ++t) sel[t] = cand[t].col;
        qsort(sel, (size_t)nc, sizeof(int32_t), cmp_i32);
        for (int64_t t = 0; t < nc; ++t) {
            if (sel[t] < i) ++nl;
            else ++nu;
        }
        if (lp[i] + nl > cap_l) return -2;
        for (int64_t t = 0; t < nl; ++t) {
            li[lp[i] + t] = sel[t];
            lx[lp[i] + t] = w[sel[t]];
        }
        lp[i + 1] = lp[i] + nl;
        if (up[i] + 1 + nu > cap_u) return -2;
        cplx piv = w[i];
        double guard = 1e-14 * row_inf;
        if (cabs(piv) < guard || piv == 0.0) {
            piv = guard > 0.0 ? guard : 1e-300;
            ++*n_guarded;
        }
        ui[up[i]] = (int32_t)i;
        ux[up[i]] = piv;
        for (int64_t t = 0; t < nu; ++t) {
            ui[up[i] + 1 + t] = sel[nl + t];
            ux[up[i] + 1 + t] = w[sel[nl + t]];
        }
        up[i + 1] = up[i] + 1 + nu;

        /* clear the work row */
        for (int64_t t = 0; t < ncols; ++t) {
            w[cols[t]] = 0.0;
            present[cols[t]] = 0;
        }
    }
    free(w); free(present); free(cols); free(heap); free(cand); free(sel);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* ILUTP: ILUT with threshold column pivoting, the "P" of the iLUTP of      */
/* Sec. II.  Row i is eliminated as in oracle_ilut, but in the order of the */
/* current column positions: q[k] is the column at position k, qinv its     */
/* inverse.  After the drop rule and the fill cap, if                        */
/*   permtol * max |u_ij| (kept off-diagonal entries) > |u_ii|,              */
/* the column of that largest entry (ties: the smallest position) takes     */
/* position i and the old diagonal column takes its place.  The factors     */
/* satisfy A Q ~ L U with (A Q)_{ik} = a_{i, q[k]}; L and U are returned in */
/* position space (U rows diagonal first, then increasing position), and    */
/* M^{-1} = Q U^{-1} L^{-1}.  permtol = 0 never pivots and gives exactly    */
/* the factors of oracle_ilut.  Same capacities and return codes.           */
/* ------------------------------------------------------------------------ */

typedef struct { int32_t pos; double mag; int32_t col; } keepp_t;

static int cmp_keepp(const void *pa, const void *pb) {
    const keepp_t *a = (const keepp_t *)pa, *b = (const keepp_t *)pb;
    if (a->mag != b->mag) return a->mag > b->mag ? -1 : 1; /* larger first */
    return (a->pos > b->pos) - (a->pos < b->pos);          /* then smaller position */
}

static int cmp_keepp_pos(const void *pa, const void *pb) {
    const keepp_t *a = (const keepp_t *)pa, *b = (const keepp_t *)pb;
    return (a->pos > b->pos) - (a->pos < b->pos);
}

int oracle_ilutp(int64_t n, const int64_t *ap, const int32_t *ai, const double *ax_,
                 double droptol, double fill, double permtol,
                 int64_t cap_l, int64_t *lp, int32_t *li, double *lx_,
                 int64_t cap_u, int64_t *up, int32_t *ui, double *ux_,
                 int32_t *q, int64_t *n_guarded, int64_t *n_swaps) {
    const cplx *ax = (const cplx *)ax_;
    cplx *lx = (cplx *)lx_;
    cplx *ux = (cplx *)ux_;
    size_t nn = (size_t)(n > 0 ? n : 1);
    cplx *w = (cplx *)calloc(nn, sizeof(cplx));
    unsigned char *present = (unsigned char *)calloc(nn, 1);
    int32_t *cols = (int32_t *)malloc(sizeof(int32_t) * nn);
    int32_t *heap = (int32_t *)malloc(sizeof(int32_t) * nn); /* positions < i */
    int32_t *qinv = (int32_t *)malloc(sizeof(int32_t) * nn);
    keepp_t *cand = (keepp_t *)malloc(sizeof(keepp_t) * nn);
    if (!w || !present || !cols || !heap || !qinv || !cand) {
        free(w); free(present); free(cols); free(heap); free(qinv); free(cand);
        return -1;
    }
    for (int64_t k = 0; k < n; ++k) { q[k] = (int32_t)k; qinv[k] = (int32_t)k; }
    *n_guarded = 0;
    *n_swaps = 0;
    lp[0] = 0;
    up[0] = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t nnz_i = ap[i + 1] - ap[i];
        double row_inf = 0.0;
        for (int64_t e = ap[i]; e < ap[i + 1]; ++e) {
            double m = cabs(ax[e]);
            if (m > row_inf) row_inf = m;
        }
        double tau = droptol * row_inf;
        int64_t keep_cap = (int64_t)floor(fill * (double)nnz_i / 2.0);
        if (keep_cap < 1) keep_cap = 1;

        int64_t ncols = 0, hlen = 0;
        for (int64_t e = ap[i]; e < ap[i + 1]; ++e) {
            int32_t j = ai[e];
            w[j] = ax[e];
            present[j] = 1;
            cols[ncols++] = j;
            if (qinv[j] < i) heap_push(heap, &hlen, qinv[j]);
        }
        int32_t dcol = q[i];
        if (!present[dcol]) {
            w[dcol] = 0.0;
            present[dcol] = 1;
            cols[ncols++] = dcol;
        }

        /* eliminate with the rows at positions k < i, in increasing k */
        while (hlen > 0) {
            int32_t k = heap_pop(heap, &hlen);
            int32_t ck = q[k];
            cplx wk = w[ck] / ux[up[k]];
            if (cabs(wk) < tau) {
                w[ck] = 0.0;
                continue;
            }
            w[ck] = wk;
            for (int64_t e = up[k] + 1; e < up[k + 1]; ++e) {
                int32_t j = ui[e]; /* a column label until the end */
                if (!present[j]) {
                    present[j] = 1;
                    w[j] = 0.0;
                    cols[ncols++] = j;
                    if (qinv[j] < i) heap_push(heap, &hlen, qinv[j]);
                }
                w[j] -= wk * ux[e];
            }
        }

        /* L part: positions < i */
        int64_t nl = 0;
        for (int64_t t = 0; t < ncols; ++t) {
            int32_t j = cols[t];
            if (qinv[j] < i) {
                double m = cabs(w[j]);
                if (w[j] != 0.0 && !(m < tau)) { cand[nl].pos = qinv[j]; cand[nl].mag = m; cand[nl].col = j; ++nl; }
            }
        }
        if (nl > keep_cap) {
            qsort(cand, (size_t)nl, sizeof(keepp_t), cmp_keepp);
            nl = keep_cap;
        }
        qsort(cand, (size_t)nl, sizeof(keepp_t), cmp_keepp_pos);
        if (lp[i] + nl > cap_l) return -2;
        for (int64_t t = 0; t < nl; ++t) {
            li[lp[i] + t] = cand[t].pos;
            lx[lp[i] + t] = w[cand[t].col];
        }
        lp[i + 1] = lp[i] + nl;

        /* U part: positions > i */
        int64_t nu = 0;
        for (int64_t t = 0; t < ncols; ++t) {
            int32_t j = cols[t];
            if (qinv[j] > i) {
                double m = cabs(w[j]);
                if (w[j] != 0.0 && !(m < tau)) { cand[nu].pos = qinv[j]; cand[nu].mag = m; cand[nu].col = j; ++nu; }
            }
        }
        if (nu > keep_cap - 1) {
            qsort(cand, (size_t)nu, sizeof(keepp_t), cmp_keepp);
            nu = keep_cap - 1;
        }
        if (up[i] + 1 + nu > cap_u) return -2;
        /* threshold pivoting among the kept entries */
        int64_t best = -1;
        for (int64_t t = 0; t < nu; ++t)
            if (best < 0 || cand[t].mag > cand[best].mag ||
                (cand[t].mag == cand[best].mag && cand[t].pos < cand[best].pos))
                best = t;
        if (best >= 0 && permtol * cand[best].mag > cabs(w[dcol])) {
            int32_t newc = cand[best].col;
            int32_t p = qinv[newc];
            q[i] = newc; qinv[newc] = (int32_t)i;
            q[p] = dcol; qinv[dcol] = p;
            cand[best].col = dcol;
            cand[best].pos = p;
            cand[best].mag = cabs(w[dcol]);
            if (w[dcol] == 0.0) { cand[best] = cand[nu - 1]; --nu; }
            dcol = newc;
            ++*n_swaps;
        }
        cplx piv = w[dcol];
        double guard = 1e-14 * row_inf;
        if (cabs(piv) < guard || piv == 0.0) {
            piv = guard > 0.0 ? guard : 1e-300;
            ++*n_guarded;
        }
        ui[up[i]] = dcol;
        ux[up[i]] = piv;
        for (int64_t t = 0; t < nu; ++t) {
            ui[up[i] + 1 + t] = cand[t].col;
            ux[up[i] + 1 + t] = w[cand[t].col];
        }
        up[i + 1] = up[i] + 1 + nu;

        for (int64_t t = 0; t < ncols; ++t) {
            w[cols[t]] = 0.0;
            present[cols[t]] = 0;
        }
    }
    /* U columns to positions, each row's off-diagonal part in increasing position */
    for (int64_t i = 0; i < n; ++i) {
        int64_t b = up[i], e = up[i + 1];
        ui[b] = (int32_t)i;
        int64_t m = 0;
        for (int64_t t = b + 1; t < e; ++t) { cand[m].pos = qinv[ui[t]]; cand[m].col = (int32_t)(t - b - 1); cand[m].mag = 0; ++m; }
        qsort(cand, (size_t)m, sizeof(keepp_t), cmp_keepp_pos);
        for (int64_t t = 0; t < m; ++t) ((cplx *)w)[t] = ux[b + 1 + cand[t].col];
        for (int64_t t = 0; t < m; ++t) { ui[b + 1 + t] = cand[t].pos; ux[b + 1 + t] = w[t]; }
        for (int64_t t = 0; t < m; ++t) w[t] = 0.0;
    }
    free(w); free(present); free(cols); free(heap); free(qinv); free(cand);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Triangular sweeps with the ILUT factors (the preconditioner solve of     */
/* Eq. 6, M = L U) and with their conjugate transposes (M^H = U^H L^H).     */
/* ------------------------------------------------------------------------ */

/* x := L^{-1} b, L unit lower (strict part stored). b and x may alias. */
void oracle_lsolve(int64_t n, const int64_t *lp, const int32_t *li, const double *lx_,
                   const double *b_, double *x_) {
    const cplx *lx = (const cplx *)lx_;
    const cplx *b = (const cplx *)b_;
    cplx *x = (cplx *)x_;
    for (int64_t i = 0; i < n; ++i) {
        cplx s = b[i];
        for (int64_t e = lp[i]; e < lp[i + 1]; ++e) s -= lx[e] * x[li[e]];
        x[i] = s;
    }
}

/* x := U^{-1} b, U upper with the diagonal first in each row. */
void oracle_usolve(int64_t n, const int64_t *up, const int32_t *ui, const double *ux_,
                   const double *b_, double *x_) {
    const cplx *ux = (const cplx *)ux_;
    const cplx *b = (const cplx *)b_;
    cplx *x = (cplx *)x_;
    for (int64_t i = n - 1; i >= 0; --i) {
        cplx s = b[i];
        for (int64_t e = up[i] + 1; e < up[i + 1]; ++e) s -= ux[e] * x[ui[e]];
        x[i] = s / ux[up[i]];
    }
}

/* x := U^{-H} b  (U^H is lower triangular; column sweep over the rows of U).
 * x is overwritten in place; b and x may alias. */
void oracle_uhsolve(int64_t n, const int64_t *up, const int32_t *ui, const double *ux_,
                    const double *b_, double *x_) {
    const cplx *ux = (const cplx *)ux_;
    const cplx *b = (const cplx *)b_;
    cplx *x = (cplx *)x_;
    if (x != b) memcpy(x, b, sizeof(cplx) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        x[i] = x[i] / conj(ux[up[i]]);
        for (int64_t e = up[i] + 1; e < up[i + 1]; ++e) x[ui[e]] -= conj(ux[e]) * x[i];
    }
}

/* x := L^{-H} b  (L^H is unit upper triangular; column sweep over rows of L). */
void oracle_lhsolve(int64_t n, const int64_t *lp, const int32_t *li, const double *lx_,
                    const double *b_, double *x_) {
    const cplx *lx = (const cplx *)lx_;
    const cplx *b = (const cplx *)b_;
    cplx *x = (cplx *)x_;
    if (x != b) memcpy(x, b, sizeof(cplx) * (size_t)n);
    for (int64_t i = n - 1; i >= 0; --i)
        for (int64_t e = lp[i]; e < lp[i + 1]; ++e) x[li[e]] -= conj(lx[e]) * x[i];
}
