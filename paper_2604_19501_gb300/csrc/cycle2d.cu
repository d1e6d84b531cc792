// Fused tile kernels of the 2D V(1,1) Jacobi cycle in FP32 (see cycle2d.cuh).
//
// Operators and weights are those of the separate kernels (gridops.cu):
//  * fine operator (Sec. 3.1): 2nd order  H x = D x - h^-2 (sum of the 4 face neighbours),
//    D = 4/h^2 - c;  4th order compact (Eq. disc4thCompact)  D = 20/(6h^2) - (8/12) c, face
//    weight -4/(6h^2) - (c_i + c_j)/24, corner weight -1/(6h^2); c = omega^2 kappa^2 (1 - i gamma);
//  * level-2 operator: the assembled Galerkin stencil (Eq. Galerkin), radius r2;
//  * transfers (Eqs. intergrid, levdep): R = tensor product of w (full weighting
//    [1 2 1]/4 or cubic [1 4 6 4 1]/16) centred on the even fine nodes, P = 4 R^T;
//    fine nodes outside the grid are left out.
// Values outside the grid are held as zero in the tiles, which reproduces the Dirichlet
// ghost of the operators and the transfers' omission of outside nodes.
#include "cycle2d.cuh"
#include "timer.cuh"

namespace helm {

namespace {

__constant__ float c_w[2][5] = {{0.25f, 0.5f, 0.25f, 0.f, 0.f},
                                {1.f / 16, 4.f / 16, 6.f / 16, 4.f / 16, 1.f / 16}};

constexpr int kThreads = 256;
constexpr int kFD = 16;              // fine down pass: coarse tile side
constexpr int kTX = 32, kTY = 8;     // level-2 passes: tile of level-2 nodes
constexpr int kFX = 32, kFY = 16;    // fine up pass: tile of fine nodes

__device__ __forceinline__ float2 z2() { return make_float2(0.f, 0.f); }
// 1 / d as conj(d) / |d|^2 with one IEEE round-to-nearest reciprocal
__device__ __forceinline__ float2 rcp_c(float2 d) {
  const float r = __frcp_rn(fmaf(d.x, d.x, d.y * d.y));
  return make_float2(d.x * r, -d.y * r);
}

// coefficient c = omega^2 kappa^2 (1 - i gamma) and diagonal of the fine operator at (x, y)
template <int ORDER>
__device__ __forceinline__ void fine_cd(const Cycle2D& c, long long idx, int x, int y, float2& cc, float2& diag) {
  const float cre = (float)c.fine.omega2 * c.kap[idx];
  const float gam = c.fine.gam32[0][x] + c.fine.gam32[1][y];
  cc = make_float2(cre, -cre * gam);
  const float ih2 = (float)c.fine.inv_h2;
  if (ORDER == 0) diag = make_float2(4.f * ih2 - cc.x, -cc.y);
  else diag = make_float2(float(20.0 / 6.0) * ih2 - float(8.0 / 12.0) * cc.x, -float(8.0 / 12.0) * cc.y);
}
template <int ORDER>
__device__ __forceinline__ float2 fine_diag_of(const Cycle2D& c, float2 cc) {
  const float ih2 = (float)c.fine.inv_h2;
  if (ORDER == 0) return make_float2(4.f * ih2 - cc.x, -cc.y);
  return make_float2(float(20.0 / 6.0) * ih2 - float(8.0 / 12.0) * cc.x, -float(8.0 / 12.0) * cc.y);
}

// (H x) at the centre of a 3 x 3 window of x and c held in registers ([row][column]), in
// the order of fine_apply_tile
template <int ORDER>
__device__ __forceinline__ float2 fine_apply_win(const float2 (&wx)[3][3], const float2 (&wc)[3][3], float ih2,
                                                 float2 diag) {
  if (ORDER == 0) {
    float2 s = wx[1][0] + wx[1][2];
    s = s + wx[0][1];
    s = s + wx[2][1];
    return cmul(diag, wx[1][1]) - cscale(s, ih2);
  }
  const float2 ci = wc[1][1];
  float2 acc = cmul(diag, wx[1][1]);
  const float wface = float(-4.0 / 6.0) * ih2, wedge = float(-1.0 / 6.0) * ih2;
#pragma unroll
  for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
    for (int dx = -1; dx <= 1; ++dx) {
      if (dx == 0 && dy == 0) continue;
      const float2 xv = wx[1 + dy][1 + dx];
      if (dx == 0 || dy == 0) {
        const float2 cj = wc[1 + dy][1 + dx];
        const float2 m = make_float2(wface - float(1.0 / 24.0) * (ci.x + cj.x), -float(1.0 / 24.0) * (ci.y + cj.y));
        acc = cmac(acc, m, xv);
      } else {
        acc = acc + cscale(xv, wedge);
      }
    }
  return acc;
}

// Entry (dx, dy) of the level-2 stencil at node idx.  The Galerkin operator R H P with
// P = 4 R^T of a complex-symmetric H is complex-symmetric, so an entry of the lower half
// of the stencil (dy < 0, or dy = 0 and dx < 0) is the mirrored entry stored at the
// neighbour; reading those from the neighbour keeps DRAM reads to the upper half of the
// planes (the shifted reads hit L1/L2).
template <int R>
__device__ __forceinline__ float2 coef2_sym(const Cycle2D& c, long long idx, int dx, int dy) {
  constexpr int W = 2 * R + 1;
  const long long n = c.g2.size;
  if (dy > 0 || (dy == 0 && dx >= 0)) return c.coef2[((dx + R) + W * (dy + R)) * n + idx];
  return c.coef2[((-dx + R) + W * (-dy + R)) * n + idx + dx + (long long)c.g2.N[0] * dy];
}

// (H x) at tile position li (row stride S) from tiles of x and c
template <int ORDER>
__device__ __forceinline__ float2 fine_apply_tile(const float2* __restrict__ sx, const float2* __restrict__ sc, int li,
                                                  int S, float ih2, float2 diag) {
  if (ORDER == 0) {
    float2 s = sx[li - 1] + sx[li + 1];
    s = s + sx[li - S];
    s = s + sx[li + S];
    return cmul(diag, sx[li]) - cscale(s, ih2);
  }
  const float2 ci = sc[li];
  float2 acc = cmul(diag, sx[li]);
  const float wface = float(-4.0 / 6.0) * ih2, wedge = float(-1.0 / 6.0) * ih2;
#pragma unroll
  for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
    for (int dx = -1; dx <= 1; ++dx) {
      if (dx == 0 && dy == 0) continue;
      const int q = li + dx + dy * S;
      const float2 xv = sx[q];
      if (dx == 0 || dy == 0) {
        const float2 cj = sc[q];
        const float2 m = make_float2(wface - float(1.0 / 24.0) * (ci.x + cj.x), -float(1.0 / 24.0) * (ci.y + cj.y));
        acc = cmac(acc, m, xv);
      } else {
        acc = acc + cscale(xv, wedge);
      }
    }
  return acc;
}

// ---------------------------------------------------------------- fine down pass
// One block: a kFD x kFD tile of level-2 nodes.  Fine region of x1: the tile's fine
// nodes widened by RW (restriction) + 1 (operator).
template <int ORDER, int RW>
__global__ void __launch_bounds__(kThreads) fine_down_kernel(const Cycle2D c, const float4* __restrict__ v,
                                                             float2* __restrict__ r2) {
  constexpr int NX = 2 * kFD + 2 * RW + 1;
  constexpr int NF = NX - 2;
  extern __shared__ float2 sm[];
  float2* sv = sm;
  float2* sc = sv + NX * NX;
  float2* sx = sc + NX * NX;
  float2* sr = sx + NX * NX;     // [NF][NF]
  float2* st = sr + NF * NF;     // [NF][kFD]
  const GridDims& g = c.fine.g;
  const int N0 = g.N[0], N1 = g.N[1];
  const int C0x = blockIdx.x * kFD, C0y = blockIdx.y * kFD, rhs = blockIdx.z;
  const int X0 = 2 * C0x - RW - 1, Y0 = 2 * C0y - RW - 1;
  const float4* vb = v + rhs * g.size;
  const float w1 = c.w1, ih2 = (float)c.fine.inv_h2;
  for (int q = threadIdx.x; q < NX * NX; q += kThreads) {
    const int gx = X0 + q % NX, gy = Y0 + q / NX;
    float2 vv = z2(), cc = z2(), xx = z2();
    if (gx >= 0 && gx < N0 && gy >= 0 && gy < N1) {
      const long long idx = gx + (long long)N0 * gy;
      const float4 t = vb[idx];
      vv = make_float2(t.x, t.y);
      float2 diag;
      fine_cd<ORDER>(c, idx, gx, gy, cc, diag);
      xx = cscale(cmul(rcp_c(diag), vv), w1);
    }
    sv[q] = vv;
    sc[q] = cc;
    sx[q] = xx;
  }
  __syncthreads();
  // residual on the NF x NF region: each thread walks RS consecutive rows of one column
  // with a three-row window of x and c in registers (a third of the shared-memory reads of
  // a gather per node)
  {
    constexpr int SEG = kThreads / NF;              // row segments per column
    constexpr int RS = (NF + SEG - 1) / SEG;        // rows per segment
    const int lx = threadIdx.x % NF + 1, sg = threadIdx.x / NF;
    if (sg < SEG) {
      const int y0 = 1 + sg * RS, y1 = min(NF + 1, y0 + RS);
      float2 wx[3][3], wc[3][3];   // [row - (ly - 1)][column - (lx - 1)]
#pragma unroll
      for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          wx[r][d] = sx[(lx - 1 + d) + NX * (y0 - 1 + r)];
          wc[r][d] = sc[(lx - 1 + d) + NX * (y0 - 1 + r)];
        }
      const int gx = X0 + lx;
      for (int ly = y0; ly < y1; ++ly) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          wx[2][d] = sx[(lx - 1 + d) + NX * (ly + 1)];
          wc[2][d] = sc[(lx - 1 + d) + NX * (ly + 1)];
        }
        const int gy = Y0 + ly;
        float2 r = z2();
        if (gx >= 0 && gx < N0 && gy >= 0 && gy < N1)
          r = sv[lx + NX * ly] - fine_apply_win<ORDER>(wx, wc, ih2, fine_diag_of<ORDER>(c, wc[1][1]));
        sr[(ly - 1) * NF + lx - 1] = r;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          wx[0][d] = wx[1][d];
          wx[1][d] = wx[2][d];
          wc[0][d] = wc[1][d];
          wc[1][d] = wc[2][d];
        }
      }
    }
  }
  __syncthreads();
  const float* w = c_w[RW - 1];
  for (int q = threadIdx.x; q < NF * kFD; q += kThreads) {
    const int fy = q / kFD, cx = q % kFD;
    float2 acc = z2();
#pragma unroll
    for (int a = 0; a <= 2 * RW; ++a) {
      const float2 t = sr[fy * NF + 2 * cx + a];
      acc.x = fmaf(w[a], t.x, acc.x);
      acc.y = fmaf(w[a], t.y, acc.y);
    }
    st[q] = acc;
  }
  __syncthreads();
  const GridDims& gc = c.g2;
  for (int q = threadIdx.x; q < kFD * kFD; q += kThreads) {
    const int cy = q / kFD, cx = q % kFD;
    const int Cx = C0x + cx, Cy = C0y + cy;
    if (Cx >= gc.N[0] || Cy >= gc.N[1]) continue;
    float2 acc = z2();
#pragma unroll
    for (int b = 0; b <= 2 * RW; ++b) {
      const float2 t = st[(2 * cy + b) * kFD + cx];
      acc.x = fmaf(w[b], t.x, acc.x);
      acc.y = fmaf(w[b], t.y, acc.y);
    }
    r2[rhs * gc.size + Cx + (long long)gc.N[0] * Cy] = acc;
  }
}

// ---------------------------------------------------------------- level 2
// A kTX x kTY tile of level-2 nodes; x2 = w2 D2^-1 r2 on the tile widened by R.
template <int R>
__global__ void __launch_bounds__(kThreads) l2_resid_kernel(const Cycle2D c, const float2* __restrict__ r2,
                                                            float2* __restrict__ s2) {
  constexpr int NX = kTX + 2 * R, NY = kTY + 2 * R;
  __shared__ float2 sx[NX * NY];
  const GridDims& g = c.g2;
  const int N0 = g.N[0], N1 = g.N[1];
  const int T0x = blockIdx.x * kTX, T0y = blockIdx.y * kTY, rhs = blockIdx.z;
  const float2* rb = r2 + rhs * g.size;
  for (int q = threadIdx.x; q < NX * NY; q += kThreads) {
    const int gx = T0x - R + q % NX, gy = T0y - R + q / NX;
    float2 xx = z2();
    if (gx >= 0 && gx < N0 && gy >= 0 && gy < N1) {
      const long long idx = gx + (long long)N0 * gy;
      xx = cscale(cmul(c.dinv2[idx], rb[idx]), c.w2);
    }
    sx[q] = xx;
  }
  __syncthreads();
  const int tx = threadIdx.x % kTX, ty = threadIdx.x / kTX;
  const int gx = T0x + tx, gy = T0y + ty;
  if (gx >= N0 || gy >= N1) return;
  const long long idx = gx + (long long)N0 * gy;
  float2 ax = z2();
#pragma unroll
  for (int dy = -R; dy <= R; ++dy) {
    if (gy + dy < 0 || gy + dy >= N1) continue;
#pragma unroll
    for (int dx = -R; dx <= R; ++dx) {
      if (gx + dx < 0 || gx + dx >= N0) continue;
      ax = cmac(ax, coef2_sym<R>(c, idx, dx, dy), sx[(tx + R + dx) + NX * (ty + R + dy)]);
    }
  }
  s2[rhs * g.size + idx] = rb[idx] - ax;
}

// b3 = R2 s2 in c128 (one thread per level-3 node)
template <int RW>
__global__ void __launch_bounds__(kThreads) l2_restrict_kernel(const Cycle2D c, const float2* __restrict__ s2,
                                                               double2* __restrict__ b3, int nrhs) {
  const GridDims& gf = c.g2;
  const GridDims& gc = c.g3;
  const long long I = blockIdx.x * (long long)kThreads + threadIdx.x;
  if (I >= gc.size) return;
  int ci, cj, ck;
  node_coords(gc, I, ci, cj, ck);
  const float* w = c_w[RW - 1];
  for (int r = 0; r < nrhs; ++r) {
    float2 acc = z2();
    const float2* sb = s2 + r * gf.size;
#pragma unroll
    for (int ay = -RW; ay <= RW; ++ay) {
      const int fy = 2 * cj + ay;
      if (fy < 0 || fy >= gf.N[1]) continue;
      const float wy = w[ay + RW];
#pragma unroll
      for (int ax = -RW; ax <= RW; ++ax) {
        const int fx = 2 * ci + ax;
        if (fx < 0 || fx >= gf.N[0]) continue;
        const float2 t = sb[fx + (long long)gf.N[0] * fy];
        const float wgt = wy * w[ax + RW];
        acc.x = fmaf(wgt, t.x, acc.x);
        acc.y = fmaf(wgt, t.y, acc.y);
      }
    }
    b3[r * gc.size + I] = make_double2(acc.x, acc.y);
  }
}

// Prolongation of a coarse field (held in a tile) to the fine tile positions
// [X0, X0 + NX) x [Y0, Y0 + NY): separable, P = 4 R^T, i.e. weights 2 w per axis.  Along
// an axis, fine node f = 2J takes 2w[PW] of J and, for cubic transfers, 2w[PW -+ 2] of J -+ 1;
// f = 2J + 1 takes 2w[PW - 1] = 2w[PW + 1] of J and J + 1:
//   full weighting:  even (1) of J;            odd (1/2, 1/2)
//   cubic:           even (1/8, 3/4, 1/8);     odd (1/2, 1/2)
//   ce: coarse tile with origin (J0x, J0y), size MX x MY; u: scratch [MY][NX]; out: [NY][NX]
template <int PW>
__device__ __forceinline__ float2 prolong_1d(const float2* __restrict__ e, int f, int J0, int stride) {
  const int J = f >> 1;   // floor division
  const float2* p = e + (J - J0) * stride;
  if (f & 1) return cscale(p[0] + p[stride], 0.5f);
  if (PW == 1) return p[0];
  float2 acc = cscale(p[0], 0.75f);
  acc.x = fmaf(0.125f, p[-stride].x + p[stride].x, acc.x);
  acc.y = fmaf(0.125f, p[-stride].y + p[stride].y, acc.y);
  return acc;
}
template <int PW>
__device__ __forceinline__ void prolong_tile(const float2* __restrict__ ce, int J0x, int J0y, int MX, int MY,
                                             float2* __restrict__ u, float2* __restrict__ out, int X0, int Y0,
                                             int NX, int NY) {
  for (int q = threadIdx.x; q < MY * NX; q += kThreads) {
    const int jy = q / NX, lx = q % NX;
    u[q] = prolong_1d<PW>(ce + jy * MX, X0 + lx, J0x, 1);
  }
  __syncthreads();
  for (int q = threadIdx.x; q < NY * NX; q += kThreads) {
    const int ly = q / NX, lx = q % NX;
    out[q] = prolong_1d<PW>(u + lx, Y0 + ly, J0y, NX);
  }
}

// level-2 post pass on a kTX x kTY tile: x2 = w2 D2^-1 r2 + P2 e3 on the tile widened by
// R, then one Jacobi step at the tile nodes
template <int R, int PW>
__global__ void __launch_bounds__(kThreads) l2_up_kernel(const Cycle2D c, const float2* __restrict__ r2,
                                                         const double2* __restrict__ e3, float2* __restrict__ y2) {
  constexpr int NX = kTX + 2 * R, NY = kTY + 2 * R;
  constexpr int MX = NX / 2 + PW + 2, MY = NY / 2 + PW + 2;   // coarse cover of the widened tile
  __shared__ float2 sx[NX * NY];
  __shared__ float2 sp[NX * NY];
  __shared__ float2 se[MX * MY];
  __shared__ float2 su[MY * NX];
  const GridDims& g = c.g2;
  const GridDims& g3 = c.g3;
  const int N0 = g.N[0], N1 = g.N[1];
  const int T0x = blockIdx.x * kTX, T0y = blockIdx.y * kTY, rhs = blockIdx.z;
  const int X0 = T0x - R, Y0 = T0y - R;
  const int J0x = (X0 - PW + 1) >> 1, J0y = (Y0 - PW + 1) >> 1;
  const float2* rb = r2 + rhs * g.size;
  const double2* eb = e3 + rhs * g3.size;
  for (int q = threadIdx.x; q < MX * MY; q += kThreads) {
    const int Jx = J0x + q % MX, Jy = J0y + q / MX;
    float2 e = z2();
    if (Jx >= 0 && Jx < g3.N[0] && Jy >= 0 && Jy < g3.N[1]) {
      const double2 d = eb[Jx + (long long)g3.N[0] * Jy];
      e = make_float2((float)d.x, (float)d.y);
    }
    se[q] = e;
  }
  __syncthreads();
  prolong_tile<PW>(se, J0x, J0y, MX, MY, su, sp, X0, Y0, NX, NY);
  __syncthreads();
  for (int q = threadIdx.x; q < NX * NY; q += kThreads) {
    const int gx = X0 + q % NX, gy = Y0 + q / NX;
    float2 xx = z2();
    if (gx >= 0 && gx < N0 && gy >= 0 && gy < N1) {
      const long long idx = gx + (long long)N0 * gy;
      xx = cscale(cmul(c.dinv2[idx], rb[idx]), c.w2) + sp[q];
    }
    sx[q] = xx;
  }
  __syncthreads();
  const int tx = threadIdx.x % kTX, ty = threadIdx.x / kTX;
  const int gx = T0x + tx, gy = T0y + ty;
  if (gx >= N0 || gy >= N1) return;
  const long long idx = gx + (long long)N0 * gy;
  float2 ax = z2();
#pragma unroll
  for (int dy = -R; dy <= R; ++dy) {
    if (gy + dy < 0 || gy + dy >= N1) continue;
#pragma unroll
    for (int dx = -R; dx <= R; ++dx) {
      if (gx + dx < 0 || gx + dx >= N0) continue;
      ax = cmac(ax, coef2_sym<R>(c, idx, dx, dy), sx[(tx + R + dx) + NX * (ty + R + dy)]);
    }
  }
  const float2 xc = sx[(tx + R) + NX * (ty + R)];
  y2[rhs * g.size + idx] = xc + cscale(cmul(c.dinv2[idx], rb[idx] - ax), c.w2);
}

// ---------------------------------------------------------------- fine up pass
// A kFX x kFY tile of fine nodes: x1 = w1 D1^-1 v + P1 y2 on the tile widened by 1, then
// z = x1 + w1 D1^-1 (v - H1 x1) at the tile nodes.
template <int ORDER, int PW>
__global__ void __launch_bounds__(kThreads) fine_up_kernel(const Cycle2D c, const float4* __restrict__ v,
                                                           const float2* __restrict__ y2, float2* __restrict__ z) {
  constexpr int NX = kFX + 2, NY = kFY + 2;
  constexpr int MX = NX / 2 + PW + 2, MY = NY / 2 + PW + 2;
  __shared__ float2 sv[NX * NY];
  __shared__ float2 sc[NX * NY];
  __shared__ float2 sx[NX * NY];
  __shared__ float2 sp[NX * NY];   // P y2, then 1 / diagonal
  __shared__ float2 se[MX * MY];
  __shared__ float2 su[MY * NX];
  const GridDims& g = c.fine.g;
  const GridDims& g2 = c.g2;
  const int N0 = g.N[0], N1 = g.N[1];
  const int T0x = blockIdx.x * kFX, T0y = blockIdx.y * kFY, rhs = blockIdx.z;
  const int X0 = T0x - 1, Y0 = T0y - 1;
  const int J0x = (X0 - PW + 1) >> 1, J0y = (Y0 - PW + 1) >> 1;
  const float4* vb = v + rhs * g.size;
  const float2* yb = y2 + rhs * g2.size;
  const float w1 = c.w1, ih2 = (float)c.fine.inv_h2;
  for (int q = threadIdx.x; q < MX * MY; q += kThreads) {
    const int Jx = J0x + q % MX, Jy = J0y + q / MX;
    se[q] = (Jx >= 0 && Jx < g2.N[0] && Jy >= 0 && Jy < g2.N[1]) ? yb[Jx + (long long)g2.N[0] * Jy] : z2();
  }
  __syncthreads();
  prolong_tile<PW>(se, J0x, J0y, MX, MY, su, sp, X0, Y0, NX, NY);
  __syncthreads();
  for (int q = threadIdx.x; q < NX * NY; q += kThreads) {
    const int gx = X0 + q % NX, gy = Y0 + q / NX;
    float2 vv = z2(), cc = z2(), xx = z2(), di = z2();
    if (gx >= 0 && gx < N0 && gy >= 0 && gy < N1) {
      const long long idx = gx + (long long)N0 * gy;
      const float4 t = vb[idx];
      vv = make_float2(t.x, t.y);
      float2 diag;
      fine_cd<ORDER>(c, idx, gx, gy, cc, diag);
      di = rcp_c(diag);
      xx = cscale(cmul(di, vv), w1) + sp[q];
    }
    sv[q] = vv;
    sc[q] = cc;
    sx[q] = xx;
    sp[q] = di;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < kFX * kFY; q += kThreads) {
    const int tx = q % kFX, ty = q / kFX;
    const int gx = T0x + tx, gy = T0y + ty;
    if (gx >= N0 || gy >= N1) continue;
    const int li = (tx + 1) + NX * (ty + 1);
    const float2 diag = fine_diag_of<ORDER>(c, sc[li]);
    const float2 res = sv[li] - fine_apply_tile<ORDER>(sx, sc, li, NX, ih2, diag);
    z[rhs * g.size + gx + (long long)N0 * gy] = sx[li] + cscale(cmul(sp[li], res), w1);
  }
}

inline dim3 tiles(const GridDims& g, int tx, int ty, int nrhs) {
  return dim3((g.N[0] + tx - 1) / tx, (g.N[1] + ty - 1) / ty, nrhs);
}

}  // namespace

int cycle2d_fine_down(const Cycle2D& c, const float4* v, float2* r2, int nrhs, cudaStream_t s) {
  KernelTimer kt(HELM_K_FINE, s);
  const dim3 grid = tiles(c.g2, kFD, kFD, nrhs);
  auto smem = [](int rw) {
    const int nx = 2 * kFD + 2 * rw + 1, nf = nx - 2;
    return (size_t)(3 * nx * nx + nf * nf + nf * kFD) * sizeof(float2);
  };
#define HELM_FD(O, RW)                                                                                  \
  if (c.fine.order == O && c.rw1 == RW) {                                                               \
    static bool attr = false;                                                                           \
    if (!attr) {                                                                                        \
      cudaFuncSetAttribute(fine_down_kernel<O, RW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem(RW)); \
      attr = true;                                                                                      \
    }                                                                                                   \
    fine_down_kernel<O, RW><<<grid, kThreads, smem(RW), s>>>(c, v, r2);                                 \
    HELM_LAUNCH_CHECK();                                                                                \
    return 0;                                                                                           \
  }
  HELM_FD(0, 1)
  HELM_FD(0, 2)
  HELM_FD(1, 1)
  HELM_FD(1, 2)
#undef HELM_FD
  set_error("fused fine pass: unsupported order or transfer");
  return HELM_EINVAL;
}

int cycle2d_l2_resid(const Cycle2D& c, const float2* r2, float2* s2, int nrhs, cudaStream_t s) {
  KernelTimer kt(HELM_K_STENCIL, s);
  const dim3 grid = tiles(c.g2, kTX, kTY, nrhs);
  if (c.r2 == 1) l2_resid_kernel<1><<<grid, kThreads, 0, s>>>(c, r2, s2);
  else if (c.r2 == 2) l2_resid_kernel<2><<<grid, kThreads, 0, s>>>(c, r2, s2);
  else { set_error("fused level-2 pass: unsupported stencil radius"); return HELM_EINVAL; }
  HELM_LAUNCH_CHECK();
  return 0;
}

int cycle2d_l2_restrict(const Cycle2D& c, const float2* s2, double2* b3, int nrhs, cudaStream_t s) {
  KernelTimer kt(HELM_K_TRANSFER, s);
  const int bl = blocks_for(c.g3.size, kThreads);
  if (c.rw2 == 1) l2_restrict_kernel<1><<<bl, kThreads, 0, s>>>(c, s2, b3, nrhs);
  else if (c.rw2 == 2) l2_restrict_kernel<2><<<bl, kThreads, 0, s>>>(c, s2, b3, nrhs);
  else { set_error("fused restriction: unsupported radius"); return HELM_EINVAL; }
  HELM_LAUNCH_CHECK();
  return 0;
}

int cycle2d_l2_up(const Cycle2D& c, const float2* r2, const double2* e3, float2* y2, int nrhs, cudaStream_t s) {
  KernelTimer kt(HELM_K_STENCIL, s);
  const dim3 grid = tiles(c.g2, kTX, kTY, nrhs);
#define HELM_L2U(R, PW)                                                                 \
  if (c.r2 == R && c.pw2 == PW) {                                                       \
    l2_up_kernel<R, PW><<<grid, kThreads, 0, s>>>(c, r2, e3, y2);                       \
    HELM_LAUNCH_CHECK();                                                                \
    return 0;                                                                           \
  }
  HELM_L2U(1, 1)
  HELM_L2U(1, 2)
  HELM_L2U(2, 1)
  HELM_L2U(2, 2)
#undef HELM_L2U
  set_error("fused level-2 pass: unsupported radius");
  return HELM_EINVAL;
}

int cycle2d_fine_up(const Cycle2D& c, const float4* v, const float2* y2, float2* z, int nrhs, cudaStream_t s) {
  KernelTimer kt(HELM_K_FINE, s);
  const dim3 grid = tiles(c.fine.g, kFX, kFY, nrhs);
#define HELM_FU(O, PW)                                                                  \
  if (c.fine.order == O && c.rw1 == PW) {                                               \
    fine_up_kernel<O, PW><<<grid, kThreads, 0, s>>>(c, v, y2, z);                       \
    HELM_LAUNCH_CHECK();                                                                \
    return 0;                                                                           \
  }
  HELM_FU(0, 1)
  HELM_FU(0, 2)
  HELM_FU(1, 1)
  HELM_FU(1, 2)
#undef HELM_FU
  set_error("fused fine pass: unsupported order or transfer");
  return HELM_EINVAL;
}

}  // namespace helm
