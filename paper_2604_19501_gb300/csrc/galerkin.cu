// Galerkin coarse operators (Eq. Galerkin) and the real-shifted coarsest operator
// (Eqs. realShift, CoarseRealShifted) assembled on the device, one thread per coarse
// node:
//   H_c(I, I + D) = sum_i sum_j R(I, i) A(i, j) P(j, I + D),
// i over the restriction support of I, j over the stencil of row i, with
// R(I, i) = prod_k w_R(i_k - 2 I_k) and P(j, J) = 2^d prod_k w_P(j_k - 2 J_k).
// The real part of the mass term, R (omega^2 kappa^2 M) P, is assembled alongside so
// that the coarsest shift can be applied by linearity:
//   H_4h^alpha = R2 (H_2h + (1 - alpha^2) R1 omega^2 kappa^2 M P1) P2   (Eq. realShiftMeaning).
#include "galerkin.cuh"
#include "timer.cuh"

namespace helm {

__constant__ double c_rap_w[2][5] = {{0.25, 0.5, 0.25, 0.0, 0.0},
                                     {1.0 / 16, 4.0 / 16, 6.0 / 16, 4.0 / 16, 1.0 / 16}};

// Rows of the fine operator, computed from kappa^2 and the absorbing profile: the
// 2nd-order 5/7-point stencil, or the compact 4th-order 9/19-point stencils of Eqs.
// disc4thCompact / disc4thCompact3D with the coefficient mean (c_i + c_j) / 2 on every
// mass coupling.  a: the operator entry; m: its real mass part omega^2 kappa^2 M.
struct FineRows {
  FineOp op;
  const double* kap;
  __device__ __forceinline__ double gam_at(int ii, int jj, int kk) const {
    return op.gam[0][ii] + op.gam[1][jj] + (op.g.dim == 3 ? op.gam[2][kk] : 0.0);
  }
  __device__ __forceinline__ void get(long long i, int ii, int jj, int kk, int bx, int by, int bz,
                                      double2& a, double& m) const {
    const int nz = abs(bx) + abs(by) + abs(bz);
    const bool is3 = op.g.dim == 3;
    double lap, mw;
    if (op.order == 0) {
      lap = nz == 0 ? 2.0 * op.g.dim * op.inv_h2 : (nz == 1 ? -op.inv_h2 : 0.0);
      mw = nz == 0 ? 1.0 : 0.0;
    } else if (nz == 0) {
      lap = (is3 ? 4.0 : 20.0 / 6.0) * op.inv_h2;
      mw = is3 ? 6.0 / 12.0 : 8.0 / 12.0;
    } else if (nz == 1) {
      lap = (is3 ? -2.0 / 6.0 : -4.0 / 6.0) * op.inv_h2;
      mw = 1.0 / 12.0;
    } else if (nz == 2) {
      lap = -op.inv_h2 / 6.0;
      mw = 0.0;
    } else {
      lap = 0.0;
      mw = 0.0;
    }
    if (mw == 0.0) {
      a = make_double2(lap, 0.0);
      m = 0.0;
      return;
    }
    const long long j = i + bx + (long long)by * op.g.N[0] + (long long)bz * op.g.N[0] * op.g.N[1];
    const double ki = op.omega2 * kap[i], kj = op.omega2 * kap[j];
    const double gi = gam_at(ii, jj, kk), gj = gam_at(ii + bx, jj + by, kk + bz);
    // c = k^2 (1 - i gamma); mean of the two coupled nodes
    const double cre = 0.5 * (ki + kj), cim = -0.5 * (ki * gi + kj * gj);
    a = make_double2(lap - mw * cre, -mw * cim);
    m = mw * cre;
  }
};

// Rows of an assembled stencil plus `shift` times its real mass part.
struct StoredRows {
  GridDims g;
  int r;
  const double2* coef;
  const double* mk;
  double shift;
  __device__ __forceinline__ void get(long long i, int, int, int, int bx, int by, int bz, double2& a,
                                      double& m) const {
    const int W = 2 * r + 1;
    if (abs(bx) > r || abs(by) > r || abs(bz) > r) { a = make_double2(0, 0); m = 0; return; }
    const int o = (bx + r) + W * ((by + r) + W * (g.dim == 3 ? bz + r : 0));
    a = coef[(long long)o * g.size + i];
    m = mk ? mk[(long long)o * g.size + i] : 0.0;
    a.x += shift * m;
  }
};

template <class Rows, int DIM, int RR, int RP, int RA, int RC>
__global__ void __launch_bounds__(128) rap_kernel(Rows rows, GridDims gf, GridDims gc,
                                                  double2* __restrict__ hout,
                                                  double* __restrict__ mout) {
  constexpr int WC = 2 * RC + 1;
  constexpr int NC = DIM == 3 ? WC * WC * WC : WC * WC;
  const long long I = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (I >= gc.size) return;
  int ci, cj, ck;
  node_coords(gc, I, ci, cj, ck);
  double2 H[NC];
  double M[NC];
  for (int o = 0; o < NC; ++o) { H[o] = make_double2(0, 0); M[o] = 0; }
  const double* wR = c_rap_w[RR - 1];
  const double* wP = c_rap_w[RP - 1];
  const long long sy = gf.N[0], sz = (long long)gf.N[0] * gf.N[1];
  const int zr = DIM == 3 ? 1 : 0;
  for (int az = -RR * zr; az <= RR * zr; ++az)
    for (int ay = -RR; ay <= RR; ++ay)
      for (int ax = -RR; ax <= RR; ++ax) {
        const int fi = 2 * ci + ax, fj = 2 * cj + ay, fk = 2 * ck + az;
        if (fi < 0 || fi >= gf.N[0] || fj < 0 || fj >= gf.N[1] || fk < 0 || fk >= gf.N[2]) continue;
        const double wr = wR[ax + RR] * wR[ay + RR] * (DIM == 3 ? wR[az + RR] : 1.0);
        const long long fidx = fi + fj * sy + fk * sz;
        for (int bz = -RA * zr; bz <= RA * zr; ++bz)
          for (int by = -RA; by <= RA; ++by)
            for (int bx = -RA; bx <= RA; ++bx) {
              const int gi = fi + bx, gj = fj + by, gk = fk + bz;
              if (gi < 0 || gi >= gf.N[0] || gj < 0 || gj >= gf.N[1] || gk < 0 || gk >= gf.N[2]) continue;
              double2 a;
              double m;
              rows.get(fidx, fi, fj, fk, bx, by, bz, a, m);
              if (a.x == 0.0 && a.y == 0.0 && m == 0.0) continue;
              // coarse J with |g - 2J| <= RP per axis
              const int i0 = max(0, (gi - RP + 1) >> 1), i1 = min(gc.N[0] - 1, (gi + RP) >> 1);
              const int j0 = max(0, (gj - RP + 1) >> 1), j1 = min(gc.N[1] - 1, (gj + RP) >> 1);
              int k0 = 0, k1 = 0;
              if (DIM == 3) { k0 = max(0, (gk - RP + 1) >> 1); k1 = min(gc.N[2] - 1, (gk + RP) >> 1); }
              for (int K = k0; K <= k1; ++K)
                for (int J = j0; J <= j1; ++J)
                  for (int Ii = i0; Ii <= i1; ++Ii) {
                    const double wp = 2.0 * wP[gi - 2 * Ii + RP] * 2.0 * wP[gj - 2 * J + RP] *
                                      (DIM == 3 ? 2.0 * wP[gk - 2 * K + RP] : 1.0);
                    const double f = wr * wp;
                    const int o = (Ii - ci + RC) + WC * ((J - cj + RC) + WC * (DIM == 3 ? K - ck + RC : 0));
                    H[o].x = fma(f, a.x, H[o].x);
                    H[o].y = fma(f, a.y, H[o].y);
                    M[o] = fma(f, m, M[o]);
                  }
            }
      }
  for (int o = 0; o < NC; ++o) {
    hout[(long long)o * gc.size + I] = H[o];
    if (mout) mout[(long long)o * gc.size + I] = M[o];
  }
}

// dinv = 1 / centre coefficient; c64 copies of the coefficients and of dinv.
__global__ void finalize_kernel(long long n, int ncoef, int centre, const double2* __restrict__ coef,
                                double2* __restrict__ dinv64, float2* __restrict__ coef32,
                                float2* __restrict__ dinv32, int* __restrict__ bad) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double2 d = coef[(long long)centre * n + i];
    const double m = d.x * d.x + d.y * d.y;
    if (!(m > 0.0) || !isfinite(m)) atomicExch(bad, 1);
    const double2 di = make_double2(d.x / m, -d.y / m);
    dinv64[i] = di;
    if (dinv32) dinv32[i] = make_float2((float)di.x, (float)di.y);
    if (coef32)
      for (int o = 0; o < ncoef; ++o) {
        const double2 c = coef[(long long)o * n + i];
        coef32[(long long)o * n + i] = make_float2((float)c.x, (float)c.y);
      }
  }
}

// out = coef + shift * mk (real mass part on the real component)
__global__ void shift_kernel(long long n, const double2* __restrict__ coef, const double* __restrict__ mk,
                             double shift, double2* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    double2 c = coef[i];
    c.x += shift * mk[i];
    out[i] = c;
  }
}

template <class Rows, int DIM, int RR, int RP, int RA, int RC>
static int rap_launch(const Rows& rows, const GridDims& gf, const GridDims& gc, double2* h, double* m,
                      cudaStream_t s) {
  const int th = 128;
  KernelTimer kt(HELM_K_SETUP, s);
  rap_kernel<Rows, DIM, RR, RP, RA, RC><<<blocks_for(gc.size, th), th, 0, s>>>(rows, gf, gc, h, m);
  HELM_LAUNCH_CHECK();
  return 0;
}

int assemble_level2(const FineOp& op, const double* kappa2, const GridDims& gc, int rR, int rP,
                    double2* h, double* mk, int* rc_out, cudaStream_t s) {
  FineRows rows{op, kappa2};
  const int rc = (rR + 1 + rP) / 2;
  *rc_out = rc;
  const bool d2 = op.g.dim == 2;
  if (rR == 1 && rP == 1)
    return d2 ? rap_launch<FineRows, 2, 1, 1, 1, 1>(rows, op.g, gc, h, mk, s)
              : rap_launch<FineRows, 3, 1, 1, 1, 1>(rows, op.g, gc, h, mk, s);
  if (rR == 2 && rP == 2)
    return d2 ? rap_launch<FineRows, 2, 2, 2, 1, 2>(rows, op.g, gc, h, mk, s)
              : rap_launch<FineRows, 3, 2, 2, 1, 2>(rows, op.g, gc, h, mk, s);
  set_error("transfer combination not built");
  return 1;
}

int assemble_level3(const GridDims& g2, int r2, const double2* h2, const double* mk2, double shift,
                    const GridDims& g3, int rR, int rP, double2* h3, int* rc_out, cudaStream_t s) {
  StoredRows rows{g2, r2, h2, mk2, shift};
  const int rc = (rR + r2 + rP) / 2;
  *rc_out = rc;
  const bool d2 = g2.dim == 2;
  if (rR == 1 && rP == 1 && r2 == 1)
    return d2 ? rap_launch<StoredRows, 2, 1, 1, 1, 1>(rows, g2, g3, h3, nullptr, s)
              : rap_launch<StoredRows, 3, 1, 1, 1, 1>(rows, g2, g3, h3, nullptr, s);
  if (rR == 2 && rP == 2 && r2 == 2 && d2)
    return rap_launch<StoredRows, 2, 2, 2, 2, 3>(rows, g2, g3, h3, nullptr, s);
  if (rR == 1 && rP == 2 && r2 == 2)
    return d2 ? rap_launch<StoredRows, 2, 1, 2, 2, 2>(rows, g2, g3, h3, nullptr, s)
              : rap_launch<StoredRows, 3, 1, 2, 2, 2>(rows, g2, g3, h3, nullptr, s);
  set_error("transfer combination not built");
  return 1;
}

int finalize_stencil(long long n, int ncoef, int centre, const double2* coef, double2* dinv64,
                     float2* coef32, float2* dinv32, int* bad, cudaStream_t s) {
  const int th = 256;
  const int bl = (int)std::min<long long>(blocks_for(n, th), 152LL * 16);
  finalize_kernel<<<bl, th, 0, s>>>(n, ncoef, centre, coef, dinv64, coef32, dinv32, bad);
  HELM_LAUNCH_CHECK();
  return 0;
}

int apply_shift(long long n, const double2* coef, const double* mk, double shift, double2* out,
                cudaStream_t s) {
  const int th = 256;
  const int bl = (int)std::min<long long>(blocks_for(n, th), 152LL * 16);
  shift_kernel<<<bl, th, 0, s>>>(n, coef, mk, shift, out);
  HELM_LAUNCH_CHECK();
  return 0;
}

}  // namespace helm
