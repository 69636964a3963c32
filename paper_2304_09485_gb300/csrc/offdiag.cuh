// Product form of the off-diagonal Jacobian blocks (mixed precision).
#pragma once
#include <cuda_runtime.h>

namespace hgks {

// acc += 1/2 (J(Q_j) n - lambda I) S x_j, the off-diagonal block of Eq. (deri-matrix)
// applied as a product (no stored 5x5 block): J(Q_j)(n S/2) x_j from j's primitives
// (jv rows 0-5) and the record of face p of cell i (rows 6 + 4p + k)
template <typename TV>
__device__ __forceinline__ void offdiag_product(const float *__restrict__ jv, int N, int i, int p, int j, const TV *x,
                                                TV *acc) {
  const TV u = jv[j], v = jv[(size_t)N + j], w = jv[2 * (size_t)N + j], H = jv[3 * (size_t)N + j];
  const TV phi = jv[4 * (size_t)N + j], g1 = jv[5 * (size_t)N + j];
  const float *f = jv + (size_t)(6 + 4 * p) * N + i;
  const TV nx = f[0], ny = f[N], nz = f[2 * (size_t)N], ls = f[3 * (size_t)N];
  const TV un = u * nx + v * ny + w * nz, nm = nx * x[1] + ny * x[2] + nz * x[3], um = u * x[1] + v * x[2] + w * x[3];
  const TV dp = g1 * (x[4] - um) + phi * x[0], t = nm - un * x[0];
  acc[0] += nm - ls * x[0];
  acc[1] += u * t + un * x[1] + nx * dp - ls * x[1];
  acc[2] += v * t + un * x[2] + ny * dp - ls * x[2];
  acc[3] += w * t + un * x[3] + nz * dp - ls * x[3];
  acc[4] += un * (x[4] + dp) + H * t - ls * x[4];
}

}  // namespace hgks
