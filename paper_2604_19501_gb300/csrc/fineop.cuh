// The fine-grid operator H_h = -Lap_h - omega^2 kappa^2 (1 - i gamma) M_h at one node
// (Sec. 1 Eq. acousitcHelm; Sec. 3.1), shared by the cycle and the Krylov kernels.
#pragma once
#include "common.cuh"

namespace helm {

// Diagonal 2d/h^2 - c of the 2nd-order operator, c = omega^2 kappa^2 (1 - i gamma).
template <typename T>
__device__ __forceinline__ c2<T> fine_diag(const FineOp& op, const T* __restrict__ kap, long long idx,
                                           int i, int j, int k) {
  const T gam = (T)op.gam[0][i] + (T)op.gam[1][j] + (op.g.dim == 3 ? (T)op.gam[2][k] : T(0));
  const T cre = (T)op.omega2 * kap[idx];
  return mk<T>(T(2 * op.g.dim) * (T)op.inv_h2 - cre, cre * gam);
}

// (H x) at flat position p (node (i, j, k)) of a vector x; zero beyond the boundary.
template <typename T, typename TX>
__device__ __forceinline__ c2<T> fine_apply_at(const FineOp& op, c2<T> diag, const c2<TX>* __restrict__ x,
                                               long long p, int i, int j, int k) {
  const long long sy = op.g.N[0];
  const long long sz = (long long)op.g.N[0] * op.g.N[1];
  c2<T> s = mk<T>(0, 0);
  if (i > 0) s = s + cvt<T>(x[p - 1]);
  if (i < op.g.N[0] - 1) s = s + cvt<T>(x[p + 1]);
  if (j > 0) s = s + cvt<T>(x[p - sy]);
  if (j < op.g.N[1] - 1) s = s + cvt<T>(x[p + sy]);
  if (op.g.dim == 3) {
    if (k > 0) s = s + cvt<T>(x[p - sz]);
    if (k < op.g.N[2] - 1) s = s + cvt<T>(x[p + sz]);
  }
  return cmul(diag, cvt<T>(x[p])) - cscale(s, (T)op.inv_h2);
}

}  // namespace helm
