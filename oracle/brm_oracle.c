/*
 * CPU oracle for BRMerge SpGEMM (Du et al., "Accelerating CPU-Based Sparse
 * General Matrix Multiplication With Binary Row Merging", IEEE Access 2022).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls
 * this file; only the tests, the smoke check and the benchmark's CPU-baseline
 * leg do.  It shares no code with the CUDA library.
 *
 * Plain, single-threaded, slow and obvious.  Build with -O2 -ffp-contract=off
 * so that no multiply-add is ever fused (the products must be rounded before
 * they are added, as in the paper's multiplying phase).
 *
 * Every entry point works on an explicit list of output rows, so callers can
 * ask for a whole matrix (rows = 0..m-1) or for a sample of rows of a product
 * too large to hold.
 *
 * Inputs are CSR with int32 row pointers and columns, columns strictly
 * ascending inside each row (Section II-A notation: A is M x K, B is K x N).
 * Values are passed as double; float inputs are promoted exactly by the
 * caller, except in the Algorithm 1 single-precision modes, which take float.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

/* ------------------------------------------------------------------------ */
/* Intermediate-product count per output row:                                */
/*   nprod_i = sum over k in A_i* of |B_k*|                                  */
/* (Algorithm 1 line 1 and step 1 of both libraries, Section III-D).         */
/* ------------------------------------------------------------------------ */
void orc_row_nprod(int64_t nrows, const int64_t *rows,
                   const int32_t *arp, const int32_t *acol, const int32_t *brp,
                   int64_t *nprod_out)
{
    for (int64_t t = 0; t < nrows; ++t) {
        int64_t i = rows[t], s = 0;
        for (int32_t p = arp[i]; p < arp[i + 1]; ++p) {
            int32_t k = acol[p];
            s += (int64_t)(brp[k + 1] - brp[k]);
        }
        nprod_out[t] = s;
    }
}

/* ------------------------------------------------------------------------ */
/* Symbolic phase (Section II-B, precise allocation): the number of distinct */
/* columns of row i of C, i.e. |union over k in A_i* of cols(B_k*)|.  No     */
/* floating point.  A stamp array marks columns already seen in this row.    */
/* ------------------------------------------------------------------------ */
int orc_symbolic(int64_t nrows, const int64_t *rows,
                 const int32_t *arp, const int32_t *acol,
                 int32_t ncols, const int32_t *brp, const int32_t *bcol,
                 int64_t *nnz_out)
{
    int64_t *mark = (int64_t *)malloc(sizeof(int64_t) * (size_t)(ncols > 0 ? ncols : 1));
    if (!mark) return -1;
    for (int32_t j = 0; j < ncols; ++j) mark[j] = -1;
    for (int64_t t = 0; t < nrows; ++t) {
        int64_t i = rows[t], cnt = 0;
        for (int32_t p = arp[i]; p < arp[i + 1]; ++p) {
            int32_t k = acol[p];
            for (int32_t q = brp[k]; q < brp[k + 1]; ++q) {
                int32_t j = bcol[q];
                if (mark[j] != t) { mark[j] = t; ++cnt; }
            }
        }
        nnz_out[t] = cnt;
    }
    free(mark);
    return 0;
}

static int cmp_i32(const void *x, const void *y)
{
    int32_t a = *(const int32_t *)x, b = *(const int32_t *)y;
    return (a > b) - (a < b);
}

/* ------------------------------------------------------------------------ */
/* Gustavson's row-wise product, the plain definition of Eq. (2):            */
/*   C_i* = sum over k in A_i* of A_ik * B_k*                                */
/* evaluated in double with a dense accumulator, k taken in stored order,    */
/* each product rounded and then added.  Output columns sorted ascending.    */
/* crp[t] .. crp[t+1] is where row rows[t] goes in ccol/cval (the caller     */
/* sizes it with orc_symbolic).  If cabs is not NULL it receives the same    */
/* row of |A|*|B| (the scale of the summation error bound).                  */
/* ------------------------------------------------------------------------ */
int orc_gustavson(int64_t nrows, const int64_t *rows,
                  const int32_t *arp, const int32_t *acol, const double *aval,
                  int32_t ncols, const int32_t *brp, const int32_t *bcol, const double *bval,
                  const int64_t *crp, int32_t *ccol, double *cval, double *cabs)
{
    size_t n = (size_t)(ncols > 0 ? ncols : 1);
    double *acc = (double *)malloc(sizeof(double) * n);
    double *aab = (double *)malloc(sizeof(double) * n);
    int64_t *mark = (int64_t *)malloc(sizeof(int64_t) * n);
    int32_t *touched = (int32_t *)malloc(sizeof(int32_t) * n);
    if (!acc || !aab || !mark || !touched) { free(acc); free(aab); free(mark); free(touched); return -1; }
    for (size_t j = 0; j < n; ++j) mark[j] = -1;
    int rc = 0;
    for (int64_t t = 0; t < nrows; ++t) {
        int64_t i = rows[t];
        int64_t nt = 0;
        for (int32_t p = arp[i]; p < arp[i + 1]; ++p) {
            int32_t k = acol[p];
            double a = aval[p];
            for (int32_t q = brp[k]; q < brp[k + 1]; ++q) {
                int32_t j = bcol[q];
                double prod = a * bval[q];
                double aprod = fabs(a) * fabs(bval[q]);
                if (mark[j] != t) {
                    mark[j] = t;
                    touched[nt++] = j;
                    acc[j] = 0.0;
                    aab[j] = 0.0;
                }
                acc[j] += prod;
                aab[j] += aprod;
            }
        }
        if (nt != crp[t + 1] - crp[t]) { rc = -2; break; }
        qsort(touched, (size_t)nt, sizeof(int32_t), cmp_i32);
        for (int64_t s = 0; s < nt; ++s) {
            int32_t j = touched[s];
            ccol[crp[t] + s] = j;
            cval[crp[t] + s] = acc[j];
            if (cabs) cabs[crp[t] + s] = aab[j];
        }
    }
    free(acc); free(aab); free(mark); free(touched);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1 (BRMerge accumulation), taken step by step.                   */
/*                                                                           */
/* Multiplying phase: for each A_ik of the row, in stored order, the scaled  */
/* row A_ik * B_k* is appended to the destination buffer and the list's end  */
/* is recorded in the offset array -- also when B_k* is empty, so empty      */
/* lists keep their place in the tree.                                       */
/* Accumulating phase: while more than one list remains, lists are consumed  */
/* two at a time in order (0,1), (2,3), ... and merged like a merge sort,    */
/* adding the values of equal columns once; a last odd list is copied.  The  */
/* buffers then swap roles.  The result row is in the source buffer.         */
/* Section III-B, Fig. 2 (ceil(log2 L) rounds for L lists), Fig. 3.          */
/*                                                                           */
/* The buffers are allocated once for all rows from max_row_nprod_C and      */
/* max_row_nnz_A (the algorithm's first line) and released at the end.       */
/*                                                                           */
/* prec: 0 = double values; 1 = float values, float sums; 2 = float values   */
/* with TwoSum-compensated merge additions.  In mode 2 every list element    */
/* carries (s, e): a product starts as (a*b, 0); merging equal columns       */
/* (x, y) gives s = x.s + y.s rounded, t its exact rounding error (Knuth's   */
/* TwoSum), and e = (x.e + y.e) + t; the stored value is s + e.  Modes 1/2   */
/* read avf/bvf and write float results, widened exactly, to cval.          */
/* rounds_out (may be NULL) receives the number of merging rounds per row.   */
/* ------------------------------------------------------------------------ */
typedef struct { int32_t col; double v; float s; float e; } orc_elem;

static orc_elem merge_equal(orc_elem x, orc_elem y, int prec)
{
    orc_elem r;
    r.col = x.col;
    r.v = 0.0; r.s = 0.0f; r.e = 0.0f;
    if (prec == 0) {
        r.v = x.v + y.v;
    } else if (prec == 1) {
        r.s = x.s + y.s;
    } else {
        float s = x.s + y.s;                    /* Knuth's TwoSum */
        float bb = s - x.s;
        float t = (x.s - (s - bb)) + (y.s - bb);
        r.s = s;
        r.e = (x.e + y.e) + t;
    }
    return r;
}

int orc_alg1(int64_t nrows, const int64_t *rows, int prec,
             const int32_t *arp, const int32_t *acol, const double *avd, const float *avf,
             const int32_t *brp, const int32_t *bcol, const double *bvd, const float *bvf,
             const int64_t *crp, int32_t *ccol, double *cval, int32_t *rounds_out)
{
    /* line 1: buffer sizes */
    int64_t max_nprod = 0, max_nnz_a = 0;
    for (int64_t t = 0; t < nrows; ++t) {
        int64_t i = rows[t], s = 0;
        for (int32_t p = arp[i]; p < arp[i + 1]; ++p) s += brp[acol[p] + 1] - brp[acol[p]];
        if (s > max_nprod) max_nprod = s;
        if (arp[i + 1] - arp[i] > max_nnz_a) max_nnz_a = arp[i + 1] - arp[i];
    }
    /* lines 2-5: ping-pong buffers and their list offsets */
    orc_elem *ping = (orc_elem *)malloc(sizeof(orc_elem) * (size_t)(max_nprod + 1));
    orc_elem *pong = (orc_elem *)malloc(sizeof(orc_elem) * (size_t)(max_nprod + 1));
    int64_t *ping_off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(max_nnz_a + 1));
    int64_t *pong_off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(max_nnz_a + 1));
    if (!ping || !pong || !ping_off || !pong_off) {
        free(ping); free(pong); free(ping_off); free(pong_off); return -1;
    }
    int rc = 0;
    for (int64_t t = 0; t < nrows; ++t) {
        int64_t i = rows[t];
        orc_elem *dst = ping;
        int64_t *dst_off = ping_off;
        int64_t buf_incr = 0, list_incr = 0;
        dst_off[0] = 0;
        /* multiplying phase */
        for (int32_t p = arp[i]; p < arp[i + 1]; ++p) {
            int32_t k = acol[p];
            for (int32_t q = brp[k]; q < brp[k + 1]; ++q) {
                orc_elem e;
                e.col = bcol[q];
                e.v = 0.0; e.s = 0.0f; e.e = 0.0f;
                if (prec == 0) e.v = avd[p] * bvd[q];
                else e.s = avf[p] * bvf[q];
                dst[buf_incr++] = e;
            }
            dst_off[++list_incr] = buf_incr;
        }
        int64_t num_list = list_incr;
        orc_elem *src = dst;
        int64_t *src_off = dst_off;
        dst = pong;
        dst_off = pong_off;
        int32_t rounds = 0;
        /* accumulating phase */
        while (num_list > 1) {
            int64_t inner = num_list, li = 0, w = 0;
            num_list = 0;
            dst_off[0] = 0;
            while (inner) {
                if (inner >= 2) {
                    /* consume lists li and li+1 */
                    int64_t x = src_off[li], xe = src_off[li + 1];
                    int64_t y = src_off[li + 1], ye = src_off[li + 2];
                    while (x < xe && y < ye) {
                        if (src[x].col < src[y].col) dst[w++] = src[x++];
                        else if (src[y].col < src[x].col) dst[w++] = src[y++];
                        else dst[w++] = merge_equal(src[x++], src[y++], prec);
                    }
                    while (x < xe) dst[w++] = src[x++];
                    while (y < ye) dst[w++] = src[y++];
                    li += 2;
                    inner -= 2;
                } else {
                    /* copy the last list */
                    for (int64_t x = src_off[li]; x < src_off[li + 1]; ++x) dst[w++] = src[x];
                    li += 1;
                    inner -= 1;
                }
                ++num_list;
                dst_off[num_list] = w;
            }
            orc_elem *tb = src; src = dst; dst = tb;
            int64_t *to = src_off; src_off = dst_off; dst_off = to;
            ++rounds;
        }
        /* store the row (the single remaining list, in src) */
        int64_t len = (list_incr == 0) ? 0 : src_off[1];
        if (len != crp[t + 1] - crp[t]) { rc = -2; break; }
        for (int64_t s = 0; s < len; ++s) {
            ccol[crp[t] + s] = src[s].col;
            if (prec == 0) cval[crp[t] + s] = src[s].v;
            else if (prec == 1) cval[crp[t] + s] = (double)src[s].s;
            else cval[crp[t] + s] = (double)(float)(src[s].s + src[s].e);
        }
        if (rounds_out) rounds_out[t] = rounds;
    }
    free(ping); free(pong); free(ping_off); free(pong_off);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Gradients of loss = sum_ij C_ij * G_ij with C = A*B, G given on C's       */
/* pattern (entries of G outside it are zero):                               */
/*   dA_ik = sum over j in B_k* of G_ij * B_kj       (dC * B^T, on A's pattern) */
/*   dB_kj = sum over i with k in A_i* of A_ik * G_ij (A^T * dC, on B's pattern)*/
/* in double.  dB is accumulated over i in increasing order.  rows must be   */
/* all rows of A for dB to be complete; dA is written for the listed rows.   */
/* crp/ccol give C's pattern for the listed rows (as from orc_symbolic).     */
/* ------------------------------------------------------------------------ */
int orc_backward(int64_t nrows, const int64_t *rows,
                 const int32_t *arp, const int32_t *acol, const double *aval,
                 int32_t ncols, const int32_t *brp, const int32_t *bcol, const double *bval,
                 const int64_t *crp, const int32_t *ccol, const double *g,
                 double *da, double *db)
{
    size_t n = (size_t)(ncols > 0 ? ncols : 1);
    double *gd = (double *)calloc(n, sizeof(double));
    if (!gd) return -1;
    for (int64_t t = 0; t < nrows; ++t) {
        int64_t i = rows[t];
        for (int64_t s = crp[t]; s < crp[t + 1]; ++s) gd[ccol[s]] = g[s];
        for (int32_t p = arp[i]; p < arp[i + 1]; ++p) {
            int32_t k = acol[p];
            double acc = 0.0;
            for (int32_t q = brp[k]; q < brp[k + 1]; ++q) {
                acc += gd[bcol[q]] * bval[q];
                if (db) db[q] += aval[p] * gd[bcol[q]];
            }
            if (da) da[p] = acc;
        }
        for (int64_t s = crp[t]; s < crp[t + 1]; ++s) gd[ccol[s]] = 0.0;
    }
    free(gd);
    return 0;
}
