// Adjoint-state gradient of a least-squares misfit with respect to the slowness squared
// m = kappa^2.  The paper has no adjoint; the derivation is the standard one for the
// discrete operator of Sec. 3.1, H(m) = -Lap_h - omega^2 M_h[m (1 - i gamma)]:
//   L = 1/2 sum_r ||P p_r - d_r||^2,  H p_r = q_r,
//   dL/dm_j = -Re(lambda_r^H dH/dm_j p_r),  H^H lambda_r = P^T (P p_r - d_r).
// H is complex-symmetric, so mu_r = conj(lambda_r) solves H mu_r = conj(P^T (P p_r - d_r))
// with the same preconditioned solver, and with the coefficient mean (c_i + c_j) / 2 on
// every mass coupling (mass weights w_o, w_0 the centre)
//   dL/dm_j = omega^2 sum_r Re((1 - i gamma_j) sum_o w_o (mu_j p_{j+o} + mu_{j+o} p_j) / 2).
#include "adjoint.cuh"
#include "fineop.cuh"
#include "timer.cuh"

namespace helm {

namespace {

__global__ void conj_kernel(long long n, const double2* __restrict__ a, double2* __restrict__ b) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double2 v = a[i];
    b[i] = make_double2(v.x, -v.y);
  }
}

// grad_j += omega^2 Re((1 - i gamma_j) acc_j), acc_j the mass-weighted products above.
__global__ void gradient_kernel(FineOp op, const double2* __restrict__ p, const double2* __restrict__ mu,
                                double* __restrict__ grad) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= op.g.size) return;
  int i, j, k;
  node_coords(op.g, idx, i, j, k);
  const double2 pj = p[idx], mj = mu[idx];
  double2 acc;
  if (op.order == 0) {
    acc = cmul(mj, pj);
  } else {
    const double wc = op.g.dim == 3 ? 6.0 / 12.0 : 8.0 / 12.0;
    acc = cscale(cmul(mj, pj), wc);
    const long long sy = op.g.N[0];
    const long long sz = (long long)op.g.N[0] * op.g.N[1];
    const long long off[6] = {-1, 1, -sy, sy, -sz, sz};
    const bool ok[6] = {i > 0, i < op.g.N[0] - 1, j > 0, j < op.g.N[1] - 1, op.g.dim == 3 && k > 0,
                        op.g.dim == 3 && k < op.g.N[2] - 1};
    for (int f = 0; f < 6; ++f) {
      if (!ok[f]) continue;
      const long long q = idx + off[f];
      // w_o (mu_j p_q + mu_q p_j) / 2 with w_o = 1/12
      const double2 t = cmul(mj, p[q]) + cmul(mu[q], pj);
      acc = acc + cscale(t, 1.0 / 24.0);
    }
  }
  const double gam = op.gam[0][i] + op.gam[1][j] + (op.g.dim == 3 ? op.gam[2][k] : 0.0);
  // Re((1 - i gam) acc) = acc.x + gam acc.y
  grad[idx] += op.omega2 * (acc.x + gam * acc.y);
}

}  // namespace

int launch_conj(long long n, const double2* a, double2* b, cudaStream_t s) {
  KernelTimer kt(HELM_K_KRYLOV_OTHER, s);
  const int th = 256;
  conj_kernel<<<(int)std::min<long long>(blocks_for(n, th), 152LL * 8), th, 0, s>>>(n, a, b);
  HELM_LAUNCH_CHECK();
  return 0;
}

int launch_gradient(const FineOp& op, const double2* p, const double2* mu, double* grad, cudaStream_t s) {
  KernelTimer kt(HELM_K_KRYLOV_OTHER, s);
  const int th = 256;
  gradient_kernel<<<blocks_for(op.g.size, th), th, 0, s>>>(op, p, mu, grad);
  HELM_LAUNCH_CHECK();
  return 0;
}

}  // namespace helm
