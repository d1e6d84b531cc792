// The fine-grid operator H_h = -Lap_h - omega^2 kappa^2 (1 - i gamma) M_h at one node
// (Sec. 1 Eq. acousitcHelm; Sec. 3.1), shared by the cycle and the Krylov kernels.
#pragma once
#include "common.cuh"

namespace helm {

// Coefficient c = omega^2 kappa^2 (1 - i gamma) at node (i, j, k).
template <typename T>
__device__ __forceinline__ c2<T> fine_coef(const FineOp& op, const T* __restrict__ kap, long long idx, int i,
                                           int j, int k) {
  const T gam = (T)op.gam[0][i] + (T)op.gam[1][j] + (op.g.dim == 3 ? (T)op.gam[2][k] : T(0));
  const T cre = (T)op.omega2 * kap[idx];
  return mk<T>(cre, -cre * gam);
}

// Diagonal of the fine operator: 2d/h^2 - c (2nd order), or the centre of the compact
// 4th-order stencils, 20/(6h^2) - (8/12) c in 2D (Eq. disc4thCompact) and
// 24/(6h^2) - (6/12) c in 3D (Eq. disc4thCompact3D).
template <typename T>
__device__ __forceinline__ c2<T> fine_diag(const FineOp& op, const T* __restrict__ kap, long long idx,
                                           int i, int j, int k) {
  const c2<T> c = fine_coef<T>(op, kap, idx, i, j, k);
  const T ih2 = (T)op.inv_h2;
  if (op.order == 0) return mk<T>(T(2 * op.g.dim) * ih2 - c.x, -c.y);
  if (op.g.dim == 2) return mk<T>(T(20.0 / 6.0) * ih2 - T(8.0 / 12.0) * c.x, -T(8.0 / 12.0) * c.y);
  return mk<T>(T(4.0) * ih2 - T(0.5) * c.x, -T(0.5) * c.y);
}

// (H x) at flat position p of a vector x, node idx = (i, j, k); zero beyond the boundary.
// 4th order: Laplacian weights per offset class (centre / face / edge), mass weight 1/12
// on the faces with the coefficient mean (c_i + c_j) / 2 of the coupled nodes.
template <typename T, typename TX>
__device__ __forceinline__ c2<T> fine_apply_at(const FineOp& op, c2<T> diag, const c2<TX>* __restrict__ x,
                                               long long p, long long idx, int i, int j, int k,
                                               const T* __restrict__ kap) {
  const long long sy = op.g.N[0];
  const long long sz = (long long)op.g.N[0] * op.g.N[1];
  const T ih2 = (T)op.inv_h2;
  if (op.order == 0) {
    c2<T> s = mk<T>(0, 0);
    if (i > 0) s = s + cvt<T>(x[p - 1]);
    if (i < op.g.N[0] - 1) s = s + cvt<T>(x[p + 1]);
    if (j > 0) s = s + cvt<T>(x[p - sy]);
    if (j < op.g.N[1] - 1) s = s + cvt<T>(x[p + sy]);
    if (op.g.dim == 3) {
      if (k > 0) s = s + cvt<T>(x[p - sz]);
      if (k < op.g.N[2] - 1) s = s + cvt<T>(x[p + sz]);
    }
    return cmul(diag, cvt<T>(x[p])) - cscale(s, ih2);
  }
  const c2<T> ci = fine_coef<T>(op, kap, idx, i, j, k);
  c2<T> acc = cmul(diag, cvt<T>(x[p]));
  const bool is3 = op.g.dim == 3;
  const T wface = is3 ? T(-2.0 / 6.0) * ih2 : T(-4.0 / 6.0) * ih2;
  const T wedge = is3 ? T(-1.0 / 6.0) * ih2 : T(-1.0 / 6.0) * ih2;   // 2D: corners; 3D: edges
  const int zlo = is3 ? -1 : 0, zhi = is3 ? 1 : 0;
  for (int dz = zlo; dz <= zhi; ++dz) {
    const int kk = k + dz;
    if (kk < 0 || kk >= op.g.N[2]) continue;
    for (int dy = -1; dy <= 1; ++dy) {
      const int jj = j + dy;
      if (jj < 0 || jj >= op.g.N[1]) continue;
      for (int dx = -1; dx <= 1; ++dx) {
        const int ii = i + dx;
        if (ii < 0 || ii >= op.g.N[0]) continue;
        const int nz = (dx != 0) + (dy != 0) + (dz != 0);
        if (nz == 0 || (is3 && nz == 3) ) continue;
        const long long q = p + dx + dy * sy + dz * sz;
        const c2<T> xv = cvt<T>(x[q]);
        if (nz == 1) {
          // face: Laplacian weight and mass (1/12) (c_i + c_j) / 2
          const c2<T> cj = fine_coef<T>(op, kap, idx + (q - p), ii, jj, kk);
          const c2<T> m = mk<T>(wface - T(1.0 / 24.0) * (ci.x + cj.x), -T(1.0 / 24.0) * (ci.y + cj.y));
          acc = cmac(acc, m, xv);
        } else {
          acc = acc + cscale(xv, wedge);
        }
      }
    }
  }
  return acc;
}

}  // namespace helm
