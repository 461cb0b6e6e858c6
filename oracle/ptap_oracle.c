/*
 * Oracle for the sparse triple product C = P^T A P.
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, single-threaded FP64 CPU
 * implementation used to check the CUDA library.  Only the test suite, the
 * package smoke check and the benchmark's CPU-baseline leg may load it; the
 * product path never does, and this file shares no code with it.
 *
 * Matrices are CSR with int32 row pointers and column indices (sorted, unique
 * per row) and float64 values.  Every product here is STRUCTURAL: a column
 * that is reached keeps its entry even if the numeric sum cancels to zero,
 * because the paper's symbolic phase preallocates C with no floating point
 * (Section 2, Alg. 1-2) and the numeric phase only fills that space.
 *
 * Functions return 0 on success, -1 on allocation failure, -2 if an output
 * would have 2^31 or more entries, -3 on invalid input.  Output arrays are
 * allocated with malloc and released by oracle_free.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

void oracle_free(void* p) { free(p); }

static int cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

/* Grow-on-demand output buffers for one CSR result. */
typedef struct {
  int64_t cap, nnz;
  int32_t* col;
  double* val;
} obuf;

static int obuf_reserve(obuf* b, int64_t need) {
  if (need <= b->cap) return 0;
  int64_t cap = b->cap ? b->cap : 1024;
  while (cap < need) cap *= 2;
  int32_t* c = (int32_t*)realloc(b->col, (size_t)cap * sizeof(int32_t));
  if (!c) return -1;
  b->col = c;
  double* v = (double*)realloc(b->val, (size_t)cap * sizeof(double));
  if (!v) return -1;
  b->val = v;
  b->cap = cap;
  return 0;
}

/*
 * Row-wise product C = A * B (Section 2: Alg. 3 for one row, Alg. 4 over all
 * rows; Alg. 1-2 give the same pattern without values).  For each row i,
 * C(i,:) = sum_k A(i,k) B(k,:), accumulated in a dense array of length
 * ncols(B) with a marker per column and a list of the touched columns, which
 * is sorted before the row is emitted.
 */
int oracle_spgemm(int32_t an, int32_t am, const int32_t* Ap, const int32_t* Aj,
                  const double* Ax, int32_t bm, const int32_t* Bp, const int32_t* Bj,
                  const double* Bx, int32_t** Cp_out, int32_t** Cj_out,
                  double** Cx_out, int64_t* nnz_out) {
  (void)am;
  if (an < 0 || bm < 0) return -3;
  int32_t* Cp = (int32_t*)malloc(((size_t)an + 1) * sizeof(int32_t));
  double* acc = (double*)malloc(((size_t)bm + 1) * sizeof(double));
  int32_t* mark = (int32_t*)malloc(((size_t)bm + 1) * sizeof(int32_t));
  int32_t* touched = (int32_t*)malloc(((size_t)bm + 1) * sizeof(int32_t));
  obuf out = {0, 0, NULL, NULL};
  if (!Cp || !acc || !mark || !touched) goto oom;
  for (int32_t j = 0; j < bm; j++) mark[j] = -1;
  Cp[0] = 0;
  for (int32_t i = 0; i < an; i++) {
    int32_t nt = 0;
    for (int32_t a = Ap[i]; a < Ap[i + 1]; a++) {
      int32_t k = Aj[a];
      double aik = Ax ? Ax[a] : 0.0;
      for (int32_t b = Bp[k]; b < Bp[k + 1]; b++) {
        int32_t j = Bj[b];
        double t = aik * (Bx ? Bx[b] : 0.0);
        if (mark[j] != i) {
          mark[j] = i;
          acc[j] = t;
          touched[nt++] = j;
        } else {
          acc[j] += t;
        }
      }
    }
    qsort(touched, (size_t)nt, sizeof(int32_t), cmp_i32);
    if (out.nnz + nt >= ((int64_t)1 << 31)) goto overflow;
    if (obuf_reserve(&out, out.nnz + nt)) goto oom;
    for (int32_t t = 0; t < nt; t++) {
      out.col[out.nnz + t] = touched[t];
      out.val[out.nnz + t] = acc[touched[t]];
    }
    out.nnz += nt;
    Cp[i + 1] = (int32_t)out.nnz;
  }
  free(acc);
  free(mark);
  free(touched);
  if (obuf_reserve(&out, 1)) goto oom2;
  *Cp_out = Cp;
  *Cj_out = out.col;
  *Cx_out = out.val;
  *nnz_out = out.nnz;
  return 0;
overflow:
  free(Cp); free(acc); free(mark); free(touched); free(out.col); free(out.val);
  return -2;
oom:
  free(acc); free(mark); free(touched);
oom2:
  free(Cp); free(out.col); free(out.val);
  return -1;
}

/*
 * Explicit transpose of an n x m matrix (the "explicit transpose of P" of the
 * two-step method, Section 3, Alg. 5-6), by counting sort on the column index.
 * Rows of the result come out with ascending column indices because the
 * input rows are visited in order.
 */
int oracle_transpose(int32_t n, int32_t m, const int32_t* Pp, const int32_t* Pj,
                     const double* Px, int32_t** Tp_out, int32_t** Tj_out,
                     double** Tx_out) {
  if (n < 0 || m < 0) return -3;
  int64_t nnz = Pp[n];
  int32_t* Tp = (int32_t*)calloc((size_t)m + 1, sizeof(int32_t));
  int32_t* Tj = (int32_t*)malloc(((size_t)nnz + 1) * sizeof(int32_t));
  double* Tx = (double*)malloc(((size_t)nnz + 1) * sizeof(double));
  int32_t* next = (int32_t*)malloc(((size_t)m + 1) * sizeof(int32_t));
  if (!Tp || !Tj || !Tx || !next) {
    free(Tp); free(Tj); free(Tx); free(next);
    return -1;
  }
  for (int64_t e = 0; e < nnz; e++) Tp[Pj[e] + 1]++;
  for (int32_t j = 0; j < m; j++) Tp[j + 1] += Tp[j];
  for (int32_t j = 0; j < m; j++) next[j] = Tp[j];
  for (int32_t I = 0; I < n; I++) {
    for (int32_t e = Pp[I]; e < Pp[I + 1]; e++) {
      int32_t j = Pj[e];
      int32_t dst = next[j]++;
      Tj[dst] = I;
      Tx[dst] = Px ? Px[e] : 0.0;
    }
  }
  free(next);
  *Tp_out = Tp;
  *Tj_out = Tj;
  *Tx_out = Tx;
  return 0;
}

/*
 * Two-step triple product (Section 3, Eq. 6; Alg. 5 symbolic and Alg. 6
 * numeric): C~ = A P, then the explicit transpose P^T, then C = P^T C~.
 */
int oracle_ptap_two_step(int32_t n, int32_t m, const int32_t* Ap, const int32_t* Aj,
                         const double* Ax, const int32_t* Pp, const int32_t* Pj,
                         const double* Px, int32_t** Cp, int32_t** Cj, double** Cx,
                         int64_t* nnz) {
  int32_t *APp = NULL, *APj = NULL, *Tp = NULL, *Tj = NULL;
  double *APx = NULL, *Tx = NULL;
  int64_t apnnz = 0;
  int rc = oracle_spgemm(n, n, Ap, Aj, Ax, m, Pp, Pj, Px, &APp, &APj, &APx, &apnnz);
  if (rc) return rc;
  rc = oracle_transpose(n, m, Pp, Pj, Px, &Tp, &Tj, &Tx);
  if (rc) {
    free(APp); free(APj); free(APx);
    return rc;
  }
  rc = oracle_spgemm(m, n, Tp, Tj, Tx, m, APp, APj, APx, Cp, Cj, Cx, nnz);
  free(APp); free(APj); free(APx);
  free(Tp); free(Tj); free(Tx);
  return rc;
}

/*
 * Rows of C straight from the definition (Section 3, Eq. 7-8):
 *   C(i,:) = sum_I P(I,i) sum_J A(I,J) P(J,:)
 * for each requested coarse row i.  The fine rows I with P(I,i) in the
 * pattern are read from the transpose T = P^T supplied by the caller.
 * Output is CSR over the requested rows, columns sorted, structural.
 */
int oracle_ptap_rows(int32_t m, const int32_t* Ap, const int32_t* Aj, const double* Ax,
                     const int32_t* Pp, const int32_t* Pj, const double* Px,
                     const int32_t* Tp, const int32_t* Tj, const double* Tx,
                     int32_t nrows, const int32_t* rows, int32_t** Rp_out,
                     int32_t** Rj_out, double** Rx_out, int64_t* nnz_out) {
  int32_t* Rp = (int32_t*)malloc(((size_t)nrows + 1) * sizeof(int32_t));
  double* acc = (double*)malloc(((size_t)m + 1) * sizeof(double));
  int32_t* mark = (int32_t*)malloc(((size_t)m + 1) * sizeof(int32_t));
  int32_t* touched = (int32_t*)malloc(((size_t)m + 1) * sizeof(int32_t));
  obuf out = {0, 0, NULL, NULL};
  if (!Rp || !acc || !mark || !touched) goto oom;
  for (int32_t j = 0; j < m; j++) mark[j] = -1;
  Rp[0] = 0;
  for (int32_t r = 0; r < nrows; r++) {
    int32_t i = rows[r];
    if (i < 0 || i >= m) goto bad;
    int32_t nt = 0;
    for (int32_t e = Tp[i]; e < Tp[i + 1]; e++) {
      int32_t I = Tj[e];
      double pIi = Tx[e];
      for (int32_t a = Ap[I]; a < Ap[I + 1]; a++) {
        int32_t J = Aj[a];
        double w = pIi * Ax[a];
        for (int32_t b = Pp[J]; b < Pp[J + 1]; b++) {
          int32_t j = Pj[b];
          double t = w * Px[b];
          if (mark[j] != r) {
            mark[j] = r;
            acc[j] = t;
            touched[nt++] = j;
          } else {
            acc[j] += t;
          }
        }
      }
    }
    qsort(touched, (size_t)nt, sizeof(int32_t), cmp_i32);
    if (out.nnz + nt >= ((int64_t)1 << 31)) goto bad;
    if (obuf_reserve(&out, out.nnz + nt)) goto oom;
    for (int32_t t = 0; t < nt; t++) {
      out.col[out.nnz + t] = touched[t];
      out.val[out.nnz + t] = acc[touched[t]];
    }
    out.nnz += nt;
    Rp[r + 1] = (int32_t)out.nnz;
  }
  free(acc); free(mark); free(touched);
  if (obuf_reserve(&out, 1)) {
    free(Rp); free(out.col); free(out.val);
    return -1;
  }
  *Rp_out = Rp;
  *Rj_out = out.col;
  *Rx_out = out.val;
  *nnz_out = out.nnz;
  return 0;
bad:
  free(Rp); free(acc); free(mark); free(touched); free(out.col); free(out.val);
  return -3;
oom:
  free(Rp); free(acc); free(mark); free(touched); free(out.col); free(out.val);
  return -1;
}

/*
 * Restrict a CSR matrix M to the pattern of another matrix S of the same
 * shape: out[e] = M(I, S.col[e]) for every stored entry e of S, or 0 where M
 * has no entry there.  Used to sample the backward products onto the patterns
 * of A and P.
 */
int oracle_sample(int32_t n, const int32_t* Mp, const int32_t* Mj, const double* Mx,
                  const int32_t* Sp, const int32_t* Sj, double* out) {
  for (int32_t I = 0; I < n; I++) {
    int32_t lo0 = Mp[I], hi0 = Mp[I + 1];
    for (int32_t e = Sp[I]; e < Sp[I + 1]; e++) {
      int32_t j = Sj[e];
      int32_t lo = lo0, hi = hi0;
      double v = 0.0;
      while (lo < hi) {
        int32_t mid = lo + (hi - lo) / 2;
        if (Mj[mid] < j) lo = mid + 1;
        else hi = mid;
      }
      if (lo < hi0 && Mj[lo] == j) v = Mx[lo];
      out[e] = v;
    }
  }
  return 0;
}
