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
/* (step 1 of both allocation methods, Section III-D; the buffer sizing    */
/* that opens Algorithm 1).                                                 */
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
/* BRMerge accumulation (Section III-B, Fig. 2 and Fig. 3).                  */
/*                                                                           */
/* Row i of C is built from the scaled rows A_ik * B_k* of its entries k, in */
/* the stored order of A_i*.  Each scaled row is one sorted list; an empty   */
/* B_k* gives an empty list that still takes its place in the sequence.      */
/* The lists are then reduced in rounds: every round pairs neighbouring      */
/* lists -- the 1st with the 2nd, the 3rd with the 4th, and so on -- and     */
/* merges each pair like merge sort into one list, adding the values of a    */
/* column present in both (the left list's value first); an unpaired last   */
/* list goes to the next round as it is.  After ceil(log2 L) rounds one list */
/* is left: the row of C.  Two scratch buffers take turns as the source and  */
/* the destination of a round (the paper's ping-pong buffers).               */
/*                                                                           */
/* prec: 0 = double values; 1 = float values, float sums; 2 = float values   */
/* with TwoSum-compensated additions.  In mode 2 every list element carries  */
/* (s, e): a product starts as (a*b, 0); adding two elements (x, y) gives    */
/* s = x.s + y.s rounded, t its exact rounding error (Knuth's TwoSum), and   */
/* e = (x.e + y.e) + t; the stored value is s + e.  Modes 1/2 read avf/bvf   */
/* and write float results, widened exactly, to cval.                        */
/* rounds_out (may be NULL) receives the number of rounds of every row.      */
/* ------------------------------------------------------------------------ */
typedef struct { int32_t col; double v; float s; float e; } orc_elem;

static orc_elem add_elems(orc_elem x, orc_elem y, int prec)
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

/* Merges the sorted lists x[0..nx) and y[0..ny) into out; returns the length. */
static int64_t merge_pair(const orc_elem *x, int64_t nx, const orc_elem *y, int64_t ny, orc_elem *out, int prec)
{
    int64_t a = 0, b = 0, w = 0;
    while (a < nx && b < ny) {
        if (x[a].col < y[b].col) out[w++] = x[a++];
        else if (y[b].col < x[a].col) out[w++] = y[b++];
        else { out[w++] = add_elems(x[a], y[b], prec); ++a; ++b; }
    }
    while (a < nx) out[w++] = x[a++];
    while (b < ny) out[w++] = y[b++];
    return w;
}

/* One round: the n lists of src (list j is src[lo[j] .. lo[j+1])) become   */
/* ceil(n/2) lists in dst, bounds in dlo.  Returns their number.             */
static int64_t merge_round(const orc_elem *src, const int64_t *lo, int64_t n, orc_elem *dst, int64_t *dlo, int prec)
{
    int64_t m = 0;
    dlo[0] = 0;
    for (int64_t j = 0; j < n; j += 2) {
        int64_t w = dlo[m];
        if (j + 1 < n) {
            w += merge_pair(src + lo[j], lo[j + 1] - lo[j], src + lo[j + 1], lo[j + 2] - lo[j + 1], dst + w, prec);
        } else {
            for (int64_t q = lo[j]; q < lo[j + 1]; ++q) dst[w++] = src[q];
        }
        dlo[++m] = w;
    }
    return m;
}

int orc_alg1(int64_t nrows, const int64_t *rows, int prec,
             const int32_t *arp, const int32_t *acol, const double *avd, const float *avf,
             const int32_t *brp, const int32_t *bcol, const double *bvd, const float *bvf,
             const int64_t *crp, int32_t *ccol, double *cval, int32_t *rounds_out)
{
    /* scratch sized for the largest requested row: its products and lists */
    int64_t most = 0, most_lists = 0;
    for (int64_t t = 0; t < nrows; ++t) {
        int64_t i = rows[t], s = 0;
        for (int32_t p = arp[i]; p < arp[i + 1]; ++p) s += brp[acol[p] + 1] - brp[acol[p]];
        if (s > most) most = s;
        if (arp[i + 1] - arp[i] > most_lists) most_lists = arp[i + 1] - arp[i];
    }
    orc_elem *buf[2];
    int64_t *lo[2];
    buf[0] = (orc_elem *)malloc(sizeof(orc_elem) * (size_t)(most + 1));
    buf[1] = (orc_elem *)malloc(sizeof(orc_elem) * (size_t)(most + 1));
    lo[0] = (int64_t *)malloc(sizeof(int64_t) * (size_t)(most_lists + 2));
    lo[1] = (int64_t *)malloc(sizeof(int64_t) * (size_t)(most_lists + 2));
    if (!buf[0] || !buf[1] || !lo[0] || !lo[1]) {
        free(buf[0]); free(buf[1]); free(lo[0]); free(lo[1]); return -1;
    }
    int rc = 0;
    for (int64_t t = 0; t < nrows; ++t) {
        int64_t i = rows[t];
        /* the scaled rows A_ik * B_k*, one list per entry of A_i* */
        int64_t n = 0, w = 0;
        lo[0][0] = 0;
        for (int32_t p = arp[i]; p < arp[i + 1]; ++p) {
            int32_t k = acol[p];
            for (int32_t q = brp[k]; q < brp[k + 1]; ++q) {
                orc_elem e;
                e.col = bcol[q];
                e.v = 0.0; e.s = 0.0f; e.e = 0.0f;
                if (prec == 0) e.v = avd[p] * bvd[q];
                else e.s = avf[p] * bvf[q];
                buf[0][w++] = e;
            }
            lo[0][++n] = w;
        }
        /* rounds until one list is left */
        int cur = 0;
        int32_t rounds = 0;
        while (n > 1) {
            n = merge_round(buf[cur], lo[cur], n, buf[1 - cur], lo[1 - cur], prec);
            cur = 1 - cur;
            ++rounds;
        }
        int64_t len = n == 0 ? 0 : lo[cur][1];
        if (len != crp[t + 1] - crp[t]) { rc = -2; break; }
        for (int64_t s = 0; s < len; ++s) {
            const orc_elem *e = &buf[cur][s];
            ccol[crp[t] + s] = e->col;
            if (prec == 0) cval[crp[t] + s] = e->v;
            else if (prec == 1) cval[crp[t] + s] = (double)e->s;
            else cval[crp[t] + s] = (double)(float)(e->s + e->e);
        }
        if (rounds_out) rounds_out[t] = rounds;
    }
    free(buf[0]); free(buf[1]); free(lo[0]); free(lo[1]);
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
