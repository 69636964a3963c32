// Least-squares solve of the GMRES Hessenberg system (Algorithm 1), one thread.
#pragma once
#include <cuda_runtime.h>

namespace hgks {

// y minimises || beta e1 - H y || for the (m+1) x m upper Hessenberg H
// (H[i*m + j] = h_ij), by Givens rotations applied column by column, in place:
// H's upper triangle holds R afterwards. Columns after the first zero
// subdiagonal entry (a breakdown) are left out. Returns |g_used|, the residual
// norm of the least-squares problem.
__device__ inline double givens_lsq(int m, double *__restrict__ H, double beta, double *__restrict__ y) {
  double cs[64], sn[64], gv[65];
  int used = m;
  for (int j = 0; j < m; j++)
    if (H[(j + 1) * m + j] == 0.0) { used = j + 1; break; }
  for (int j = 0; j < m; j++) y[j] = 0.0;
  if (beta == 0.0) return 0.0;
  for (int i = 0; i <= m; i++) gv[i] = 0.0;
  gv[0] = beta;
  for (int j = 0; j < used; j++) {
    for (int i = 0; i < j; i++) {
      const double h1 = H[i * m + j], h2 = H[(i + 1) * m + j];
      H[i * m + j] = cs[i] * h1 + sn[i] * h2;
      H[(i + 1) * m + j] = -sn[i] * h1 + cs[i] * h2;
    }
    const double a = H[j * m + j], b = H[(j + 1) * m + j], r = sqrt(a * a + b * b);
    const double c = a / r, s = b / r;
    cs[j] = c;
    sn[j] = s;
    H[j * m + j] = c * a + s * b;
    H[(j + 1) * m + j] = 0.0;
    const double g1 = gv[j], g2 = gv[j + 1];
    gv[j] = c * g1 + s * g2;
    gv[j + 1] = -s * g1 + c * g2;
  }
  for (int j = used - 1; j >= 0; j--) {
    double s = gv[j];
    for (int k = j + 1; k < used; k++) s -= H[j * m + k] * y[k];
    y[j] = s / H[j * m + j];
  }
  return fabs(gv[used]);
}

}  // namespace hgks
