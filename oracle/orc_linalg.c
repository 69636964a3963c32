/* ORACLE (test infrastructure only): small dense linear algebra in FP64.
 * Gaussian elimination with partial pivoting, and least squares by Householder
 * QR. These are the library primitives the oracle's steps call. */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "orc.h"

/* Solve A x = b, A row-major n x n (not modified). Returns 0, or -1 if singular. */
int orc_lu_solve(int n, const double *A, const double *b, double *x) {
  double *M = (double *)malloc(sizeof(double) * n * (n + 1));
  for (int i = 0; i < n; i++) {
    for (int j = 0; j < n; j++) M[i * (n + 1) + j] = A[i * n + j];
    M[i * (n + 1) + n] = b[i];
  }
  for (int c = 0; c < n; c++) {
    int piv = c;
    double best = fabs(M[c * (n + 1) + c]);
    for (int r = c + 1; r < n; r++)
      if (fabs(M[r * (n + 1) + c]) > best) { best = fabs(M[r * (n + 1) + c]); piv = r; }
    if (best == 0.0) { free(M); return -1; }
    if (piv != c)
      for (int j = 0; j <= n; j++) {
        double t = M[c * (n + 1) + j]; M[c * (n + 1) + j] = M[piv * (n + 1) + j]; M[piv * (n + 1) + j] = t;
      }
    for (int r = c + 1; r < n; r++) {
      double f = M[r * (n + 1) + c] / M[c * (n + 1) + c];
      if (f == 0.0) continue;
      for (int j = c; j <= n; j++) M[r * (n + 1) + j] -= f * M[c * (n + 1) + j];
    }
  }
  for (int i = n - 1; i >= 0; i--) {
    double s = M[i * (n + 1) + n];
    for (int j = i + 1; j < n; j++) s -= M[i * (n + 1) + j] * x[j];
    x[i] = s / M[i * (n + 1) + i];
  }
  free(M);
  return 0;
}

int orc_inverse(int n, const double *A, double *Ainv) {
  double *e = (double *)calloc(n, sizeof(double)), *col = (double *)malloc(sizeof(double) * n);
  int rc = 0;
  for (int j = 0; j < n && rc == 0; j++) {
    memset(e, 0, sizeof(double) * n);
    e[j] = 1.0;
    rc = orc_lu_solve(n, A, e, col);
    for (int i = 0; i < n; i++) Ainv[i * n + j] = col[i];
  }
  free(e); free(col);
  return rc;
}

/* Least-squares map of a full-column-rank A (rows x cols, rows >= cols):
 * X (cols x rows) with x = X b minimising ||A x - b||_2, via Householder QR. */
int orc_lsq_pinv(int rows, int cols, const double *A, double *X) {
  if (rows < cols) return -1;
  double *R = (double *)malloc(sizeof(double) * rows * cols);
  double *Qt = (double *)calloc((size_t)rows * rows, sizeof(double));
  double *v = (double *)malloc(sizeof(double) * rows);
  memcpy(R, A, sizeof(double) * rows * cols);
  for (int i = 0; i < rows; i++) Qt[i * rows + i] = 1.0;
  for (int k = 0; k < cols; k++) {
    double nrm = 0.0;
    for (int i = k; i < rows; i++) nrm += R[i * cols + k] * R[i * cols + k];
    nrm = sqrt(nrm);
    if (nrm == 0.0) { free(R); free(Qt); free(v); return -1; }
    double alpha = R[k * cols + k] > 0 ? -nrm : nrm;
    for (int i = 0; i < rows; i++) v[i] = 0.0;
    v[k] = R[k * cols + k] - alpha;
    for (int i = k + 1; i < rows; i++) v[i] = R[i * cols + k];
    double vv = 0.0;
    for (int i = k; i < rows; i++) vv += v[i] * v[i];
    if (vv == 0.0) continue;
    for (int j = 0; j < cols; j++) {          /* R <- (I - 2vv^T/vv) R */
      double s = 0.0;
      for (int i = k; i < rows; i++) s += v[i] * R[i * cols + j];
      s = 2.0 * s / vv;
      for (int i = k; i < rows; i++) R[i * cols + j] -= s * v[i];
    }
    for (int j = 0; j < rows; j++) {          /* Qt <- (I - 2vv^T/vv) Qt */
      double s = 0.0;
      for (int i = k; i < rows; i++) s += v[i] * Qt[i * rows + j];
      s = 2.0 * s / vv;
      for (int i = k; i < rows; i++) Qt[i * rows + j] -= s * v[i];
    }
  }
  double rmax = 0.0;
  for (int i = 0; i < cols; i++) rmax = fmax(rmax, fabs(R[i * cols + i]));
  for (int i = 0; i < cols; i++) if (fabs(R[i * cols + i]) < 1e-12 * rmax) { free(R); free(Qt); free(v); return -1; }
  /* x = R1^{-1} (Qt b)[0:cols]: X = R1^{-1} Qt[0:cols, :] by back substitution */
  for (int j = 0; j < rows; j++) {
    for (int i = cols - 1; i >= 0; i--) {
      double s = Qt[i * rows + j];
      for (int l = i + 1; l < cols; l++) s -= R[i * cols + l] * X[l * rows + j];
      if (R[i * cols + i] == 0.0) { free(R); free(Qt); free(v); return -1; }
      X[i * rows + j] = s / R[i * cols + i];
    }
  }
  free(R); free(Qt); free(v);
  return 0;
}

/* sigma_min / sigma_max of A (rows x cols, cols <= 9) from the eigenvalues of
 * A^T A, found by cyclic Jacobi rotations. */
double orc_sv_ratio(int rows, int cols, const double *A) {
  double S[81];
  for (int a = 0; a < cols; a++)
    for (int b = 0; b < cols; b++) {
      double s = 0.0;
      for (int r = 0; r < rows; r++) s += A[r * cols + a] * A[r * cols + b];
      S[a * cols + b] = s;
    }
  for (int sweep = 0; sweep < 60; sweep++) {
    double off = 0.0;
    for (int p = 0; p < cols; p++) for (int q = p + 1; q < cols; q++) off += S[p * cols + q] * S[p * cols + q];
    if (off < 1e-300) break;
    for (int p = 0; p < cols; p++)
      for (int q = p + 1; q < cols; q++) {
        double apq = S[p * cols + q];
        if (apq == 0.0) continue;
        double th = 0.5 * (S[q * cols + q] - S[p * cols + p]) / apq;
        double t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
        double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < cols; k++) {   /* S <- S J (columns p, q) */
          double skp = S[k * cols + p], skq = S[k * cols + q];
          S[k * cols + p] = c * skp - s * skq; S[k * cols + q] = s * skp + c * skq;
        }
        for (int k = 0; k < cols; k++) {   /* S <- J^T S (rows p, q) */
          double spk = S[p * cols + k], sqk = S[q * cols + k];
          S[p * cols + k] = c * spk - s * sqk; S[q * cols + k] = s * spk + c * sqk;
        }
      }
  }
  double lo = S[0], hi = S[0];
  for (int a = 1; a < cols; a++) { double v = S[a * cols + a]; if (v < lo) lo = v; if (v > hi) hi = v; }
  if (hi <= 0.0) return 0.0;
  return sqrt(fmax(lo, 0.0) / hi);
}
