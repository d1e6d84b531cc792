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
#include <type_traits>

#include "cycle2d.cuh"
#include "timer.cuh"

namespace helm {

namespace {

__constant__ float c_w[2][5] = {{0.25f, 0.5f, 0.25f, 0.f, 0.f},
                                {1.f / 16, 4.f / 16, 6.f / 16, 4.f / 16, 1.f / 16}};

constexpr int kThreads = 256;
constexpr int kFD = 16;              // fine down pass: coarse tile side
constexpr int kL2Threads = 512;      // level-2 passes: threads per block, one per node
constexpr int kTX = 32, kTY = 16;    // level-2 passes: tile of level-2 nodes
constexpr int kFX = 32, kFY = 16;    // fine up pass: tile of fine nodes

__device__ __forceinline__ float2 z2() { return make_float2(0.f, 0.f); }

// asynchronous global -> shared copies (zero-filled when ok is false: source size 0, the
// source address then being the array's base, which is valid)
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, bool ok) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(ok ? 16 : 0) : "memory");
}
__device__ __forceinline__ void cp_async8(uint32_t dst, const void* src, bool ok) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(dst), "l"(src), "r"(ok ? 8 : 0) : "memory");
}
__device__ __forceinline__ void cp_async4(uint32_t dst, const void* src, bool ok) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src), "r"(ok ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
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

// Entry o = (dx + R) + W (dy + R) of the level-2 stencil at node idx.  The Galerkin
// operator R H P with P = 4 R^T of a complex-symmetric H is complex-symmetric, so an entry
// of the lower half of the stencil (dy < 0, or dy = 0 and dx < 0) is the mirrored entry
// stored at the neighbour; reading those from the neighbour keeps DRAM reads to the upper
// half of the planes (the shifted reads hit L1/L2).  Offsets are 32-bit (the launchers
// check ncoef x nodes < 2^31).  No bounds checks: an own entry is read at idx, and a
// mirrored entry at idx + dx + N0 dy, which for the lower-half offsets lies less than
// 2 N0 + 3 entries before idx and so inside the upper-half planes of lower index (all
// planes are allocated and hold finite values); a coefficient that belongs to no
// neighbour meets a zero x of the tile.
template <int R>
__device__ __forceinline__ float2 l2_coef(const Cycle2D& c, int idx, int o) {
  constexpr int W = 2 * R + 1;
  const int dx = o % W - R, dy = o / W - R;
  const bool up = dy > 0 || (dy == 0 && dx >= 0);
  const int plane = up ? o : (-dx + R) + W * (-dy + R);
  return c.coef2[plane * (int)c.g2.size + idx + (up ? 0 : dx + c.g2.N[0] * dy)];
}
// The whole stencil of node idx, loaded into registers (the up pass issues these loads
// when it starts, so that they are in flight while the block stages its tile).
template <int R>
__device__ __forceinline__ void l2_coefs(const Cycle2D& c, int idx, float2 (&cf)[(2 * R + 1) * (2 * R + 1)]) {
#pragma unroll
  for (int o = 0; o < (2 * R + 1) * (2 * R + 1); ++o) cf[o] = l2_coef<R>(c, idx, o);
}
// the launchers' check for the 32-bit offsets of l2_coef
inline bool l2_offsets_fit(const Cycle2D& c, long long ntiles) {
  return ntiles <= INT32_MAX && (long long)(2 * c.r2 + 1) * (2 * c.r2 + 1) * c.g2.size <= INT32_MAX;
}
// sum_{dx,dy} A2(idx; dx, dy) x(idx + (dx, dy)) with x from a tile (row stride NX, zero
// outside the grid) whose entry li is node idx, in the order of the rows and columns
template <int R, int NX>
__device__ __forceinline__ float2 l2_sum(const float2 (&cf)[(2 * R + 1) * (2 * R + 1)], const float2* __restrict__ sx,
                                         int li) {
  constexpr int W = 2 * R + 1;
  float2 ax = z2();
#pragma unroll
  for (int dy = -R; dy <= R; ++dy)
#pragma unroll
    for (int dx = -R; dx <= R; ++dx) ax = cmac(ax, cf[(dx + R) + W * (dy + R)], sx[li + dx + NX * dy]);
  return ax;
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
static_assert(kTX * kTY == kL2Threads, "one thread per level-2 node of the tile");

// Level-2 residual s2 = r2 - H2 x2, x2 = w2 D2^-1 r2, as a persistent kernel: block b walks
// the tiles b, b + G, b + 2G, ... (G resident blocks).  The next tile's inputs are in flight while the current tile is
// summed: its staged values (1 / diag and r2 on the widened tile) go by cp.async into
// the other half of a double buffer, and each stencil coefficient register is reloaded
// for the next tile right after its product with the current tile is formed.
// Coefficient offsets are 32-bit (the launcher checks ncoef x nodes < 2^31).  Tiles of
// kPX x kPY level-2 nodes, one per thread; tile t = (bx, by, rhs) in row-major order.
constexpr int kPThreads = 256;
constexpr int kPX = 32, kPY = 8;
static_assert(kPX * kPY == kPThreads, "one thread per level-2 node of the tile");
template <int R>
__global__ void __launch_bounds__(kPThreads, 2) l2_resid_pers_kernel(const Cycle2D c, const float2* __restrict__ r2,
                                                                      float2* __restrict__ s2, int ntx, int nty,
                                                                      int ntiles) {
  constexpr int W = 2 * R + 1, NC = W * W;
  constexpr int NX = kPX + 2 * R, NY = kPY + 2 * R, NS = NX * NY;
  constexpr int SPT = (NS + kPThreads - 1) / kPThreads;   // staged entries per thread
  __shared__ float2 sx[NS];
  __shared__ __align__(16) float2 sdr[2][2][NS];          // [buffer][1/diag, r2][entry]
  const GridDims& g = c.g2;
  const int N0 = g.N[0], N1 = g.N[1];
  const int tx = threadIdx.x % kPX, ty = threadIdx.x / kPX;
  const int li = (tx + R) + NX * (ty + R);
  // the node of tile t this thread sums: flat index within its right-hand side, and rhs
  auto node = [&](int t, int& idx, int& rhs, bool& in) {
    const int bx = t % ntx, by = (t / ntx) % nty;
    rhs = t / (ntx * nty);
    const int gx = bx * kPX + tx, gy = by * kPY + ty;
    in = gx < N0 && gy < N1;
    idx = in ? gx + N0 * gy : 0;
  };
  auto stage_copy = [&](int t, int buf) {   // cp.async of the staged inputs of tile t
    const int bx = t % ntx, by = (t / ntx) % nty, rhs = t / (ntx * nty);
    const float2* rb = r2 + rhs * g.size;
#pragma unroll
    for (int k = 0; k < SPT; ++k) {
      const int q = threadIdx.x + k * kPThreads;
      if (q < NS) {
        const int sxg = bx * kPX - R + q % NX, syg = by * kPY - R + q / NX;
        const bool ok = sxg >= 0 && sxg < N0 && syg >= 0 && syg < N1;
        const int j = ok ? sxg + N0 * syg : 0;
        cp_async8(smem_addr(&sdr[buf][0][q]), c.dinv2 + j, ok);
        cp_async8(smem_addr(&sdr[buf][1][q]), rb + j, ok);
      }
    }
    cp_commit();
  };
  int t = blockIdx.x;
  if (t >= ntiles) return;
  float2 cf[NC];
  int idx, rhs;
  bool in;
  node(t, idx, rhs, in);
#pragma unroll
  for (int o = 0; o < NC; ++o) cf[o] = l2_coef<R>(c, idx, o);
  float2 ro = r2[idx + rhs * g.size];
  stage_copy(t, 0);
  for (int buf = 0; t < ntiles; t += gridDim.x, buf ^= 1) {
    cp_wait<0>();   // this thread's copies of tile t have landed
#pragma unroll
    for (int k = 0; k < SPT; ++k) {
      const int q = threadIdx.x + k * kPThreads;
      if (q < NS) sx[q] = cscale(cmul(sdr[buf][0][q], sdr[buf][1][q]), c.w2);
    }
    const int tn = t + gridDim.x;
    const bool more = tn < ntiles;
    if (more) stage_copy(tn, buf ^ 1);
    int idxn = 0, rhsn = 0;
    bool inn = false;
    if (more) node(tn, idxn, rhsn, inn);
    __syncthreads();
    float2 ax = z2();
#pragma unroll
    for (int o = 0; o < NC; ++o) {
      const int dx = o % W - R, dy = o / W - R;
      ax = cmac(ax, cf[o], sx[li + dx + NX * dy]);
      if (more) cf[o] = l2_coef<R>(c, idxn, o);
    }
    if (in) s2[idx + rhs * g.size] = ro - ax;
    if (more) ro = r2[idxn + rhsn * g.size];
    idx = idxn;
    rhs = rhsn;
    in = inn;
    __syncthreads();
  }
}

// b3 = R2 s2 in c128 by tiles: a kRX x kRY tile of level-3 nodes per block, its level-2
// cover (widened by RW) staged in shared memory, then the restriction along x and along y
// with the weights in the per-node kernel's order (x first, then y).
constexpr int kRX = 32, kRY = 8;
template <int RW>
__global__ void __launch_bounds__(kThreads) l2_restrict_tile_kernel(const Cycle2D c, const float2* __restrict__ s2,
                                                                    double2* __restrict__ b3) {
  constexpr int NX = 2 * (kRX - 1) + 2 * RW + 1, NY = 2 * (kRY - 1) + 2 * RW + 1;
  __shared__ float2 sf[NY * NX];
  __shared__ float2 sx[NY * kRX];
  const GridDims& gf = c.g2;
  const GridDims& gc = c.g3;
  const int I0 = blockIdx.x * kRX, J0 = blockIdx.y * kRY, rhs = blockIdx.z;
  const int X0 = 2 * I0 - RW, Y0 = 2 * J0 - RW;
  const float2* sb = s2 + (long long)rhs * gf.size;
  // every staged value is loaded before any is stored (one memory round trip, not one per
  // pass of the loop)
  constexpr int NS = NX * NY, SPT = (NS + kThreads - 1) / kThreads;
  float2 v[SPT];
#pragma unroll
  for (int e = 0; e < SPT; ++e) {
    const int q = threadIdx.x + e * kThreads;
    const int fx = X0 + q % NX, fy = Y0 + q / NX;
    v[e] = (q < NS && fx >= 0 && fx < gf.N[0] && fy >= 0 && fy < gf.N[1]) ? sb[fx + (long long)gf.N[0] * fy] : z2();
  }
#pragma unroll
  for (int e = 0; e < SPT; ++e) {
    const int q = threadIdx.x + e * kThreads;
    if (q < NS) sf[q] = v[e];
  }
  __syncthreads();
  const float* w = c_w[RW - 1];
  for (int q = threadIdx.x; q < NY * kRX; q += kThreads) {
    const int ly = q / kRX, i = q % kRX;
    float2 acc = z2();
#pragma unroll
    for (int a = 0; a <= 2 * RW; ++a) {
      const float2 t = sf[ly * NX + 2 * i + a];
      acc.x = fmaf(w[a], t.x, acc.x);
      acc.y = fmaf(w[a], t.y, acc.y);
    }
    sx[q] = acc;
  }
  __syncthreads();
  const int i = threadIdx.x % kRX, j = threadIdx.x / kRX;
  const int I = I0 + i, J = J0 + j;
  if (I >= gc.N[0] || J >= gc.N[1]) return;
  float2 acc = z2();
#pragma unroll
  for (int b = 0; b <= 2 * RW; ++b) {
    const float2 t = sx[(2 * j + b) * kRX + i];
    acc.x = fmaf(w[b], t.x, acc.x);
    acc.y = fmaf(w[b], t.y, acc.y);
  }
  b3[(long long)rhs * gc.size + I + (long long)gc.N[0] * J] = make_double2(acc.x, acc.y);
}
static_assert(kRX * kRY == kThreads, "one thread per level-3 node of the tile");

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
template <int PW, int NT>
__device__ __forceinline__ void prolong_tile(const float2* __restrict__ ce, int J0x, int J0y, int MX, int MY,
                                             float2* __restrict__ u, float2* __restrict__ out, int X0, int Y0,
                                             int NX, int NY) {
  for (int q = threadIdx.x; q < MY * NX; q += NT) {
    const int jy = q / NX, lx = q % NX;
    u[q] = prolong_1d<PW>(ce + jy * MX, X0 + lx, J0x, 1);
  }
  __syncthreads();
  for (int q = threadIdx.x; q < NY * NX; q += NT) {
    const int ly = q / NX, lx = q % NX;
    out[q] = prolong_1d<PW>(u + lx, Y0 + ly, J0y, NX);
  }
}

// level-2 post pass on a kTX x kTY tile: x2 = w2 D2^-1 r2 + P2 e3 on the tile widened by
// R, then one Jacobi step at the tile nodes
template <int R, int PW>
__global__ void __launch_bounds__(kL2Threads, 2) l2_up_kernel(const Cycle2D c, const float2* __restrict__ r2,
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
  const int tx = threadIdx.x % kTX, ty = threadIdx.x / kTX;
  const int gx = T0x + tx, gy = T0y + ty;
  const bool in = gx < N0 && gy < N1;
  const int idx = in ? gx + N0 * gy : 0;
  float2 cf[(2 * R + 1) * (2 * R + 1)];
  l2_coefs<R>(c, idx, cf);
  for (int q = threadIdx.x; q < MX * MY; q += kL2Threads) {
    const int Jx = J0x + q % MX, Jy = J0y + q / MX;
    float2 e = z2();
    if (Jx >= 0 && Jx < g3.N[0] && Jy >= 0 && Jy < g3.N[1]) {
      const double2 d = eb[Jx + (long long)g3.N[0] * Jy];
      e = make_float2((float)d.x, (float)d.y);
    }
    se[q] = e;
  }
  __syncthreads();
  prolong_tile<PW, kL2Threads>(se, J0x, J0y, MX, MY, su, sp, X0, Y0, NX, NY);
  __syncthreads();
  {
    // the staged inputs are loaded before any staged value is formed (one round trip)
    constexpr int NS = NX * NY, SPT = (NS + kL2Threads - 1) / kL2Threads;
    float2 dv[SPT], rv[SPT];
    bool okv[SPT];
#pragma unroll
    for (int e = 0; e < SPT; ++e) {
      const int q = threadIdx.x + e * kL2Threads;
      const int sxg = X0 + q % NX, syg = Y0 + q / NX;
      okv[e] = q < NS && sxg >= 0 && sxg < N0 && syg >= 0 && syg < N1;
      const long long j = okv[e] ? sxg + (long long)N0 * syg : 0;
      dv[e] = okv[e] ? c.dinv2[j] : z2();
      rv[e] = okv[e] ? rb[j] : z2();
    }
#pragma unroll
    for (int e = 0; e < SPT; ++e) {
      const int q = threadIdx.x + e * kL2Threads;
      if (q < NS) sx[q] = okv[e] ? cscale(cmul(dv[e], rv[e]), c.w2) + sp[q] : z2();
    }
  }
  __syncthreads();
  if (!in) return;
  const float2 ax = l2_sum<R, NX>(cf, sx, (tx + R) + NX * (ty + R));
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
  prolong_tile<PW, kThreads>(se, J0x, J0y, MX, MY, su, sp, X0, Y0, NX, NY);
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

// ---------------------------------------------------------------- row-streaming fine passes
// The same two fine passes without shared memory: one warp per (strip, segment) of the
// fine grid.  Lane l holds coarse column I = I0 + l and the fine columns 2I and 2I + 1;
// the warp walks down the fine rows with a window of three rows of x1 and c in registers,
// takes the column neighbours of its two columns from the adjacent lanes (shuffles), and
// forms the restriction along x by shuffles and along y in a ring of three coarse-row
// accumulators.  The row loop is unrolled by six so that every ring slot is a compile-time
// register.  Lanes at the strip edges only supply halo values; neighbouring warps cover
// the next strip.  Values outside the grid are zero, as in the tile kernels, and the sums
// are taken in the tile kernels' order (restriction: x first, then y, weights in order).
constexpr int kRsWarps = 4;   // warps per block

__host__ __device__ constexpr int fdiv(int a, int b) { return (a >= 0) ? a / b : -((-a + b - 1) / b); }
__host__ __device__ constexpr int mod3(int a) { return ((a % 3) + 3) % 3; }

__device__ __forceinline__ float2 shup(float2 v) {
  return make_float2(__shfl_up_sync(0xffffffffu, v.x, 1), __shfl_up_sync(0xffffffffu, v.y, 1));
}
__device__ __forceinline__ float2 shdn(float2 v) {
  return make_float2(__shfl_down_sync(0xffffffffu, v.x, 1), __shfl_down_sync(0xffffffffu, v.y, 1));
}

// one fine row of a warp's two columns: x1, c (and the halo columns' from the neighbours)
struct RsRow {
  float2 xe, xo;           // x1 at columns 2I, 2I + 1
  float2 ue, uo;           // c x1 at 2I, 2I + 1 (4th order only)
  float2 ce, co;           // c at 2I, 2I + 1
  float2 de, dob;          // w1 / diagonal at 2I, 2I + 1 (fine up pass)
  float2 ve, vo;           // v at 2I, 2I + 1
};
// loaded values of one fine row
struct RsLoad {
  float4 ve, vo;
  float ke, ko, gy;
};

// Staging of the rows a warp streams: every lane copies its own entries (v at its two
// columns, 2 x 16 B; kappa, 2 x 4 B; the row's gamma_y, 4 B; in the up pass y2 at its
// coarse column, 8 B) with
// cp.async into a ring of kRing rows in shared memory, kAhead rows ahead of the row in
// use, so that each warp keeps about kAhead rows of loads in flight without holding them
// in registers.  A lane reads back only what it copied itself: its cp.async.wait_group
// makes the data visible to it.  Entries outside the grid are zero-filled (source size 0,
// the source address then being the array's base, which is valid).
constexpr int kRing = 6;                          // fine rows per warp ring (the unroll: slot = step)
constexpr int kAhead = 4;                         // rows in flight ahead of the current one
constexpr int kVRowBytes = 32 * 2 * 16;           // v: two float4 per lane
constexpr int kKRowBytes = 32 * 4 * 4;            // kappa at the two columns and gamma_y: four floats per lane
constexpr int kCRing = 4;                         // coarse rows per warp ring (fine up pass)
constexpr int kCRowBytes = 32 * 8;                // y2: one float2 per lane
constexpr int kRsDownWarpBytes = kRing * (kVRowBytes + kKRowBytes);
constexpr int kRsUpWarpBytes = kRsDownWarpBytes + kCRing * kCRowBytes;
static_assert(kRing >= kAhead + 2, "a ring slot is refilled two steps after its row was read");
static_assert(kRing == 6, "ring slots are the steps of the six-fold unroll");
constexpr int kRsMinBlocks = 5;                   // resident blocks per SM the kernels are shaped for


template <int ORDER>
__device__ __forceinline__ float2 diag_c(float2 cc, float ih2) {
  if (ORDER == 0) return make_float2(4.f * ih2 - cc.x, -cc.y);
  return make_float2(float(20.0 / 6.0) * ih2 - float(8.0 / 12.0) * cc.x, -float(8.0 / 12.0) * cc.y);
}

// (H x1) at a node from sums over its neighbours: sf, se the sums of x1 over the face and
// the corner neighbours, tf the sum of c x1 over the face neighbours.  Grouping the face
// weights wf - (c_m + c_f) / 24 of the 4th-order stencil (Eq. disc4thCompact) by term:
//   H x = d x_m + wf sf + we se - (c_m sf + tf) / 24,     d = 20 / (6 h^2) - (8 / 12) c_m;
// 2nd order (5 points): H x = (4 / h^2 - c_m) x_m - sf / h^2.  Each node's c x1 is formed
// once, when its row is formed, and used by the three rows around it.
template <int ORDER>
__device__ __forceinline__ float2 rs_apply(float2 cm, float2 xm, float2 sf, float2 se, float2 tf, float ih2) {
  const float2 diag = diag_c<ORDER>(cm, ih2);
  if (ORDER == 0) return cmul(diag, xm) - cscale(sf, ih2);
  const float wface = float(-4.0 / 6.0) * ih2, wedge = float(-1.0 / 6.0) * ih2;
  float2 acc = cmul(diag, xm);
  acc.x = fmaf(wface, sf.x, acc.x);
  acc.y = fmaf(wface, sf.y, acc.y);
  acc.x = fmaf(wedge, se.x, acc.x);
  acc.y = fmaf(wedge, se.y, acc.y);
  const float2 q = cmac(tf, cm, sf);
  acc.x = fmaf(float(-1.0 / 24.0), q.x, acc.x);
  acc.y = fmaf(float(-1.0 / 24.0), q.y, acc.y);
  return acc;
}

// c x1 of a freshly formed row (4th order)
template <int ORDER>
__device__ __forceinline__ void rs_row_prod(RsRow& R) {
  if (ORDER == 1) {
    R.ue = cmul(R.ce, R.xe);
    R.uo = cmul(R.co, R.xo);
  }
}

// H x1 at the two columns 2I, 2I + 1 of the middle row md, with rows up / dn above and
// below.  The column left of 2I is lane - 1's 2I + 1 and the one right of 2I + 1 is
// lane + 1's 2I, so the neighbour sums take one shuffle per column pair: faces of 2I are
// md(2I - 1), md(2I + 1), up(2I), dn(2I); its corners up / dn at 2I - 1 and 2I + 1.
template <int ORDER>
__device__ __forceinline__ void rs_apply_row(const RsRow& up, const RsRow& md, const RsRow& dn, float ih2, float2& he,
                                             float2& ho) {
  const float2 a = up.xo + dn.xo, b = up.xe + dn.xe;   // vertical pairs at 2I + 1, 2I
  const float2 sfe = (shup(md.xo) + md.xo) + b, sfo = (md.xe + shdn(md.xe)) + a;
  float2 see = z2(), seo = z2(), tfe = z2(), tfo = z2();
  if (ORDER == 1) {
    see = shup(a) + a;
    seo = b + shdn(b);
    tfe = (shup(md.uo) + md.uo) + (up.ue + dn.ue);
    tfo = (md.ue + shdn(md.ue)) + (up.uo + dn.uo);
  }
  he = rs_apply<ORDER>(md.ce, md.xe, sfe, see, tfe, ih2);
  ho = rs_apply<ORDER>(md.co, md.xo, sfo, seo, tfo, ih2);
}

template <int ORDER, int RW, int SEG>
struct RsDown {
  static constexpr int LO = RW;            // lanes [LO, 30] own their coarse column
  static constexpr int CS = 31 - LO;       // coarse columns per strip
  static constexpr int T = 2 * SEG + RW + 4;   // fine rows a warp visits: 2 J0 - 4 ...
};

template <int ORDER, int RW, int SEG>
__global__ void __launch_bounds__(32 * kRsWarps, kRsMinBlocks) fine_down_rs_kernel(const Cycle2D c, const float4* __restrict__ v,
                                                                     float2* __restrict__ r2) {
  using P = RsDown<ORDER, RW, SEG>;
  const GridDims& g = c.fine.g;
  const GridDims& g2 = c.g2;
  const int N0 = g.N[0], N1 = g.N[1];
  const int lane = threadIdx.x & 31;
  const int nstrip = (g2.N[0] + P::CS - 1) / P::CS;
  const int nseg = (g2.N[1] + SEG - 1) / SEG;
  const int wid = blockIdx.x * kRsWarps + (threadIdx.x >> 5);
  if (wid >= nstrip * nseg) return;   // a whole warp
  const int strip = wid % nstrip, seg = wid / nstrip;
  const int Ic = strip * P::CS - P::LO + lane;
  const int J0 = seg * SEG;
  const int xe = 2 * Ic, xo = xe + 1;
  const bool ine = xe >= 0 && xe < N0, ino = xo >= 0 && xo < N0;
  const bool own = lane >= P::LO && lane <= 30 && Ic < g2.N[0];
  const int Ybase = 2 * J0 - 4;
  const float4* vb = v + (long long)blockIdx.y * g.size;
  float2* rb = r2 + (long long)blockIdx.y * g2.size;
  const float omega2 = (float)c.fine.omega2, ih2 = (float)c.fine.inv_h2, w1 = c.w1;
  const float gxe = ine ? c.fine.gam32[0][xe] : 0.f, gxo = ino ? c.fine.gam32[0][xo] : 0.f;
  const float* __restrict__ gyt = c.fine.gam32[1];
  const float* __restrict__ kap = c.kap;
  const float* w = c_w[RW - 1];

  extern __shared__ __align__(16) unsigned char rs_smem[];
  unsigned char* const ring = rs_smem + (threadIdx.x >> 5) * kRsDownWarpBytes;
  const uint32_t vring = smem_addr(ring) + lane * 32, kring = smem_addr(ring + kRing * kVRowBytes) + lane * 16;
  RsRow W[3];
  float2 acc[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    acc[q] = z2();
    // zero rows before the first: the residual rows formed from them only feed coarse
    // rows above the segment, whose accumulators are cleared before they are reused
    W[q].xe = W[q].xo = W[q].ue = W[q].uo = W[q].ce = W[q].co = W[q].de = W[q].dob = W[q].ve = W[q].vo = z2();
  }

  // fine row t into ring slot t % kRing (zeros outside the grid, and for rows past the
  // warp's visit, `want` false)
  auto issue = [&](int t, bool want) {
    const int y = Ybase + t;
    const bool iny = want && y >= 0 && y < N1;
    const long long row = (long long)(iny ? y : 0) * N0;
    const int sl = t % kRing;
    cp_async16(vring + sl * kVRowBytes, iny && ine ? vb + row + xe : vb, iny && ine);
    cp_async16(vring + sl * kVRowBytes + 16, iny && ino ? vb + row + xo : vb, iny && ino);
    cp_async4(kring + sl * kKRowBytes, iny && ine ? kap + row + xe : kap, iny && ine);
    cp_async4(kring + sl * kKRowBytes + 4, iny && ino ? kap + row + xo : kap, iny && ino);
    cp_async4(kring + sl * kKRowBytes + 8, iny ? gyt + y : gyt, iny);
  };
  auto load = [&](int t, RsLoad& ld) {
    const int sl = t % kRing;
    const float4* vs = reinterpret_cast<const float4*>(ring + sl * kVRowBytes) + 2 * lane;
    const float* ks = reinterpret_cast<const float*>(ring + kRing * kVRowBytes + sl * kKRowBytes) + 4 * lane;
    ld.ve = vs[0];
    ld.vo = vs[1];
    ld.ke = ks[0];
    ld.ko = ks[1];
    ld.gy = ks[2];
  };
  auto node = [&](float4 vv, float kk, float gx, float gy, float2& x, float2& cc, float2& vo) {
    const float cre = omega2 * kk;
    cc = make_float2(cre, -cre * (gx + gy));
    vo = make_float2(vv.x, vv.y);
    x = cscale(cmul(rcp_c(diag_c<ORDER>(cc, ih2)), vo), w1);
  };
  // row t into window slot: own columns, then the neighbours' (zero outside the grid:
  // v = kappa = 0 there, and x1 = 0 with them; a zero kappa gives a finite diagonal)
  auto fill = [&](const RsLoad& ld, RsRow& R) {
    node(ld.ve, ld.ke, gxe, ld.gy, R.xe, R.ce, R.ve);
    node(ld.vo, ld.ko, gxo, ld.gy, R.xo, R.co, R.vo);
    rs_row_prod<ORDER>(R);
  };

  // fine row t = t0 + S of the warp's visit; S is a compile-time step of the six-fold
  // unroll.  Full groups of six steps run without branches (so that the scheduler can
  // overlap adjacent rows); only the last, partial group checks t < T.
  auto step = [&](int t0, auto Sc, auto Checked) {
    constexpr int S = decltype(Sc)::value;
    const int t = t0 + S;
    if constexpr (decltype(Checked)::value) {
      if (t >= P::T) return;
    }
    issue(t + kAhead, t + kAhead < P::T);
    cp_commit();
    cp_wait<kAhead>();   // row t has landed
    RsLoad ld;
    load(t, ld);
    RsRow& cur = W[S % 3];
    fill(ld, cur);
    const RsRow& up = W[(S + 1) % 3];   // row t - 2
    const RsRow& md = W[(S + 2) % 3];   // row t - 1 (the residual row)
    const int y = Ybase + t - 1;
    const bool iny = y >= 0 && y < N1;
    float2 he, ho;
    rs_apply_row<ORDER>(up, md, cur, ih2, he, ho);
    const float2 re = iny && ine ? md.ve - he : z2(), ro = iny && ino ? md.vo - ho : z2();
    // restriction along x, in weight order
    float2 rx = z2();
    if constexpr (RW == 2) {
      const float2 rel = shup(re), rol = shup(ro), rer = shdn(re);
      rx.x = fmaf(w[0], rel.x, rx.x); rx.y = fmaf(w[0], rel.y, rx.y);
      rx.x = fmaf(w[1], rol.x, rx.x); rx.y = fmaf(w[1], rol.y, rx.y);
      rx.x = fmaf(w[2], re.x, rx.x);  rx.y = fmaf(w[2], re.y, rx.y);
      rx.x = fmaf(w[3], ro.x, rx.x);  rx.y = fmaf(w[3], ro.y, rx.y);
      rx.x = fmaf(w[4], rer.x, rx.x); rx.y = fmaf(w[4], rer.y, rx.y);
    } else {
      const float2 rol = shup(ro);
      rx.x = fmaf(w[0], rol.x, rx.x); rx.y = fmaf(w[0], rol.y, rx.y);
      rx.x = fmaf(w[1], re.x, rx.x);  rx.y = fmaf(w[1], re.y, rx.y);
      rx.x = fmaf(w[2], ro.x, rx.x);  rx.y = fmaf(w[2], ro.y, rx.y);
    }
    // along y: residual row tm = t - 1 = 6k + u adds w[tm - 2 jr + RW] rx to the coarse
    // rows jr = 3k + q with |tm - 2 jr| <= RW (coarse row J = J0 - 2 + jr)
    constexpr int u = S - 1;
    constexpr int qlo = fdiv(u - RW + 1, 2), qhi = fdiv(u + RW, 2);
#pragma unroll
    for (int q = qlo; q <= qhi; ++q) {
      const float wq = w[u - 2 * q + RW];
      acc[mod3(q)].x = fmaf(wq, rx.x, acc[mod3(q)].x);
      acc[mod3(q)].y = fmaf(wq, rx.y, acc[mod3(q)].y);
    }
    // coarse row jr is complete once tm = 2 jr + RW
    if constexpr (((u - RW) & 1) == 0) {
      constexpr int qd = fdiv(u - RW, 2);
      const int J = J0 - 2 + t0 / 2 + qd;   // t0 = 6k: 3k = t0 / 2
      if (own && J >= J0 && J < J0 + SEG && J < g2.N[1]) rb[Ic + (long long)g2.N[0] * J] = acc[mod3(qd)];
      acc[mod3(qd)] = z2();
    }
  };

  for (int t = 0; t < kAhead; ++t) {
    issue(t, t < P::T);
    cp_commit();
  }
  using Ct = std::true_type;
  using Cf = std::false_type;
  int t0 = 0;
  for (; t0 + 6 <= P::T; t0 += 6) {
    step(t0, std::integral_constant<int, 0>{}, Cf{});
    step(t0, std::integral_constant<int, 1>{}, Cf{});
    step(t0, std::integral_constant<int, 2>{}, Cf{});
    step(t0, std::integral_constant<int, 3>{}, Cf{});
    step(t0, std::integral_constant<int, 4>{}, Cf{});
    step(t0, std::integral_constant<int, 5>{}, Cf{});
  }
  if (t0 < P::T) {
    step(t0, std::integral_constant<int, 0>{}, Ct{});
    step(t0, std::integral_constant<int, 1>{}, Ct{});
    step(t0, std::integral_constant<int, 2>{}, Ct{});
    step(t0, std::integral_constant<int, 3>{}, Ct{});
    step(t0, std::integral_constant<int, 4>{}, Ct{});
    step(t0, std::integral_constant<int, 5>{}, Ct{});
  }
  cp_wait<0>();
}

template <int ORDER, int PW, int SEG>
struct RsUp {
  static constexpr int CU = 29;            // lanes [1, 29] own both their fine columns
  static constexpr int RS = 2 * SEG;       // fine rows written per warp
  static constexpr int T = RS + 3;         // fine rows visited: Y0 - 2 ... Y0 + RS
};

template <int ORDER, int PW, int SEG>
__global__ void __launch_bounds__(32 * kRsWarps, kRsMinBlocks) fine_up_rs_kernel(const Cycle2D c, const float4* __restrict__ v,
                                                                   const float2* __restrict__ y2,
                                                                   float2* __restrict__ z) {
  using P = RsUp<ORDER, PW, SEG>;
  const GridDims& g = c.fine.g;
  const GridDims& g2 = c.g2;
  const int N0 = g.N[0], N1 = g.N[1];
  const int lane = threadIdx.x & 31;
  const int nstrip = (N0 + 2 * P::CU - 1) / (2 * P::CU);
  const int nseg = (N1 + P::RS - 1) / P::RS;
  const int wid = blockIdx.x * kRsWarps + (threadIdx.x >> 5);
  if (wid >= nstrip * nseg) return;   // a whole warp
  const int strip = wid % nstrip, seg = wid / nstrip;
  const int Ic = strip * P::CU - 1 + lane;
  const int Y0 = seg * P::RS, Ybase = Y0 - 2;
  const int cb = Ybase / 2 - 1;   // coarse row of ring index jc = 0 (Ybase is even)
  const int xe = 2 * Ic, xo = xe + 1;
  const bool ine = xe >= 0 && xe < N0, ino = xo >= 0 && xo < N0;
  const bool own = lane >= 1 && lane <= P::CU;
  const bool inc = Ic >= 0 && Ic < g2.N[0];
  const float4* vb = v + (long long)blockIdx.y * g.size;
  const float2* yb = y2 + (long long)blockIdx.y * g2.size;
  float2* zb = z + (long long)blockIdx.y * g.size;
  const float omega2 = (float)c.fine.omega2, ih2 = (float)c.fine.inv_h2, w1 = c.w1;
  const float gxe = ine ? c.fine.gam32[0][xe] : 0.f, gxo = ino ? c.fine.gam32[0][xo] : 0.f;
  const float* __restrict__ gyt = c.fine.gam32[1];
  const float* __restrict__ kap = c.kap;

  extern __shared__ __align__(16) unsigned char rs_smem[];
  unsigned char* const ring = rs_smem + (threadIdx.x >> 5) * kRsUpWarpBytes;
  const uint32_t vring = smem_addr(ring) + lane * 32, kring = smem_addr(ring + kRing * kVRowBytes) + lane * 16;
  const uint32_t cring = smem_addr(ring + kRsDownWarpBytes) + lane * 8;
  RsRow W[3];
  float2 pe[3], po[3];   // coarse rows prolongated along x to the columns 2I, 2I + 1
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    W[q].xe = W[q].xo = W[q].ue = W[q].uo = W[q].ce = W[q].co = W[q].de = W[q].dob = W[q].ve = W[q].vo = z2();
  }

  // fine row t into ring slot t % kRing, and with it (t even) coarse row t / 2 + 2 of y2
  // into coarse slot (t / 2 + 2) % kCRing; zeros outside the grids
  auto issue_coarse = [&](int jc) {
    const int J = cb + jc;
    const bool ok = inc && J >= 0 && J < g2.N[1];
    cp_async8(cring + (jc % kCRing) * kCRowBytes, ok ? yb + Ic + (long long)g2.N[0] * J : yb, ok);
  };
  auto issue = [&](int t, bool want) {
    const int y = Ybase + t;
    const bool iny = want && y >= 0 && y < N1;
    const long long row = (long long)(iny ? y : 0) * N0;
    const int sl = t % kRing;
    cp_async16(vring + sl * kVRowBytes, iny && ine ? vb + row + xe : vb, iny && ine);
    cp_async16(vring + sl * kVRowBytes + 16, iny && ino ? vb + row + xo : vb, iny && ino);
    cp_async4(kring + sl * kKRowBytes, iny && ine ? kap + row + xe : kap, iny && ine);
    cp_async4(kring + sl * kKRowBytes + 4, iny && ino ? kap + row + xo : kap, iny && ino);
    cp_async4(kring + sl * kKRowBytes + 8, iny ? gyt + y : gyt, iny);
    if ((t & 1) == 0 && want) issue_coarse(t / 2 + 2);
  };
  auto load = [&](int t, RsLoad& ld) {
    const int sl = t % kRing;
    const float4* vs = reinterpret_cast<const float4*>(ring + sl * kVRowBytes) + 2 * lane;
    const float* ks = reinterpret_cast<const float*>(ring + kRing * kVRowBytes + sl * kKRowBytes) + 4 * lane;
    ld.ve = vs[0];
    ld.vo = vs[1];
    ld.ke = ks[0];
    ld.ko = ks[1];
    ld.gy = ks[2];
  };
  // coarse row jc of y2 (staged) prolongated along x (the tile kernels' prolong_1d)
  auto coarse = [&](int jc, float2& e, float2& o) {
    const float2 yv = *(reinterpret_cast<const float2*>(ring + kRsDownWarpBytes + (jc % kCRing) * kCRowBytes) + lane);
    const float2 yl = shup(yv), yr = shdn(yv);
    o = cscale(yv + yr, 0.5f);
    if (PW == 1) {
      e = yv;
    } else {
      e = cscale(yv, 0.75f);
      e.x = fmaf(0.125f, yl.x + yr.x, e.x);
      e.y = fmaf(0.125f, yl.y + yr.y, e.y);
    }
  };
  auto node = [&](float4 vv, float kk, float gx, float gy, float2 py, float2& x, float2& cc, float2& di, float2& vo) {
    const float cre = omega2 * kk;
    cc = make_float2(cre, -cre * (gx + gy));
    vo = make_float2(vv.x, vv.y);
    di = cscale(rcp_c(diag_c<ORDER>(cc, ih2)), w1);
    x = cmul(di, vo) + py;
  };

  auto step = [&](int t0, auto Sc, auto Checked) {
    constexpr int S = decltype(Sc)::value;
    const int t = t0 + S;
    if constexpr (decltype(Checked)::value) {
      if (t >= P::T) return;
    }
    issue(t + kAhead, t + kAhead < P::T);
    cp_commit();
    cp_wait<kAhead>();   // fine row t (and for t even coarse row t / 2 + 2) has landed
    // prolongation along y to fine row t: coarse ring index jc = floor(t / 2) + 1 (t0 / 2 = 3k)
    float2 pye, pyo;
    if constexpr ((S & 1) == 0) {
      constexpr int jm = mod3(S / 2), j0 = mod3(S / 2 + 1), jp = mod3(S / 2 + 2);
      coarse(t / 2 + 2, pe[jp], po[jp]);
      if constexpr (PW == 1) {
        pye = pe[j0];
        pyo = po[j0];
      } else {
        pye = cscale(pe[j0], 0.75f);
        pye.x = fmaf(0.125f, pe[jm].x + pe[jp].x, pye.x);
        pye.y = fmaf(0.125f, pe[jm].y + pe[jp].y, pye.y);
        pyo = cscale(po[j0], 0.75f);
        pyo.x = fmaf(0.125f, po[jm].x + po[jp].x, pyo.x);
        pyo.y = fmaf(0.125f, po[jm].y + po[jp].y, pyo.y);
      }
    } else {
      constexpr int j0 = mod3((S - 1) / 2 + 1), j1 = mod3((S - 1) / 2 + 2);
      pye = cscale(pe[j0] + pe[j1], 0.5f);
      pyo = cscale(po[j0] + po[j1], 0.5f);
    }
    const int y = Ybase + t;
    const bool iny = y >= 0 && y < N1;
    RsRow& cur = W[S % 3];
    RsLoad ld;
    load(t, ld);
    cur.xe = cur.xo = cur.ce = cur.co = cur.de = cur.dob = cur.ve = cur.vo = z2();
    if (iny && ine) node(ld.ve, ld.ke, gxe, ld.gy, pye, cur.xe, cur.ce, cur.de, cur.ve);
    if (iny && ino) node(ld.vo, ld.ko, gxo, ld.gy, pyo, cur.xo, cur.co, cur.dob, cur.vo);
    rs_row_prod<ORDER>(cur);
    // z at fine row t - 1 (rows Y0 ... Y0 + RS - 1, i.e. 3 <= t <= RS + 2)
    const RsRow& up = W[(S + 1) % 3];
    const RsRow& md = W[(S + 2) % 3];
    const int ym = y - 1;
    const bool out = own && ym >= Y0 && ym < Y0 + P::RS && ym < N1;
    const long long row = (long long)ym * N0;
    float2 he, ho;
    rs_apply_row<ORDER>(up, md, cur, ih2, he, ho);
    if (out && ine) zb[row + xe] = md.xe + cmul(md.de, md.ve - he);
    if (out && ino) zb[row + xo] = md.xo + cmul(md.dob, md.vo - ho);
  };

  // coarse rows 0 and 1 travel with fine row 0
  issue_coarse(0);
  issue_coarse(1);
  for (int t = 0; t < kAhead; ++t) {
    issue(t, t < P::T);
    cp_commit();
  }
  cp_wait<kAhead - 1>();
  coarse(0, pe[0], po[0]);
  coarse(1, pe[1], po[1]);
  using Ct = std::true_type;
  using Cf = std::false_type;
  int t0 = 0;
  for (; t0 + 6 <= P::T; t0 += 6) {
    step(t0, std::integral_constant<int, 0>{}, Cf{});
    step(t0, std::integral_constant<int, 1>{}, Cf{});
    step(t0, std::integral_constant<int, 2>{}, Cf{});
    step(t0, std::integral_constant<int, 3>{}, Cf{});
    step(t0, std::integral_constant<int, 4>{}, Cf{});
    step(t0, std::integral_constant<int, 5>{}, Cf{});
  }
  if (t0 < P::T) {
    step(t0, std::integral_constant<int, 0>{}, Ct{});
    step(t0, std::integral_constant<int, 1>{}, Ct{});
    step(t0, std::integral_constant<int, 2>{}, Ct{});
    step(t0, std::integral_constant<int, 3>{}, Ct{});
    step(t0, std::integral_constant<int, 4>{}, Ct{});
    step(t0, std::integral_constant<int, 5>{}, Ct{});
  }
  cp_wait<0>();
}

// SMs of the current device (the persistent level-2 passes run two blocks on each)
inline int resident_sms() {
  static const int sms = [] {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
  }();
  return sms;
}

inline dim3 tiles(const GridDims& g, int tx, int ty, int nrhs) {
  return dim3((g.N[0] + tx - 1) / tx, (g.N[1] + ty - 1) / ty, nrhs);
}

template <int ORDER, int RW, int SEG>
int launch_down_rs(const Cycle2D& c, const float4* v, float2* r2, int nrhs, cudaStream_t s) {
  using P = RsDown<ORDER, RW, SEG>;
  const long long warps = (long long)((c.g2.N[0] + P::CS - 1) / P::CS) * ((c.g2.N[1] + SEG - 1) / SEG);
  const dim3 grid((unsigned)((warps + kRsWarps - 1) / kRsWarps), (unsigned)nrhs);
  static std::atomic<bool> attr{false};
  if (!attr) {
    cudaFuncSetAttribute(fine_down_rs_kernel<ORDER, RW, SEG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         kRsWarps * kRsDownWarpBytes);
    attr = true;
  }
  fine_down_rs_kernel<ORDER, RW, SEG><<<grid, 32 * kRsWarps, kRsWarps * kRsDownWarpBytes, s>>>(c, v, r2);
  HELM_LAUNCH_CHECK();
  return 0;
}

template <int ORDER, int PW, int SEG>
int launch_up_rs(const Cycle2D& c, const float4* v, const float2* y2, float2* z, int nrhs, cudaStream_t s) {
  using P = RsUp<ORDER, PW, SEG>;
  const long long warps =
      (long long)((c.fine.g.N[0] + 2 * P::CU - 1) / (2 * P::CU)) * ((c.fine.g.N[1] + P::RS - 1) / P::RS);
  const dim3 grid((unsigned)((warps + kRsWarps - 1) / kRsWarps), (unsigned)nrhs);
  static std::atomic<bool> attr{false};
  if (!attr) {
    cudaFuncSetAttribute(fine_up_rs_kernel<ORDER, PW, SEG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         kRsWarps * kRsUpWarpBytes);
    attr = true;
  }
  fine_up_rs_kernel<ORDER, PW, SEG><<<grid, 32 * kRsWarps, kRsWarps * kRsUpWarpBytes, s>>>(c, v, y2, z);
  HELM_LAUNCH_CHECK();
  return 0;
}

template <int SEG>
int down_rs(const Cycle2D& c, const float4* v, float2* r2, int nrhs, cudaStream_t s) {
  if (c.fine.order == 0 && c.rw1 == 1) return launch_down_rs<0, 1, SEG>(c, v, r2, nrhs, s);
  if (c.fine.order == 0 && c.rw1 == 2) return launch_down_rs<0, 2, SEG>(c, v, r2, nrhs, s);
  if (c.fine.order == 1 && c.rw1 == 1) return launch_down_rs<1, 1, SEG>(c, v, r2, nrhs, s);
  if (c.fine.order == 1 && c.rw1 == 2) return launch_down_rs<1, 2, SEG>(c, v, r2, nrhs, s);
  set_error("fused fine pass: unsupported order or transfer");
  return HELM_EINVAL;
}

template <int SEG>
int up_rs(const Cycle2D& c, const float4* v, const float2* y2, float2* z, int nrhs, cudaStream_t s) {
  if (c.fine.order == 0 && c.rw1 == 1) return launch_up_rs<0, 1, SEG>(c, v, y2, z, nrhs, s);
  if (c.fine.order == 0 && c.rw1 == 2) return launch_up_rs<0, 2, SEG>(c, v, y2, z, nrhs, s);
  if (c.fine.order == 1 && c.rw1 == 1) return launch_up_rs<1, 1, SEG>(c, v, y2, z, nrhs, s);
  if (c.fine.order == 1 && c.rw1 == 2) return launch_up_rs<1, 2, SEG>(c, v, y2, z, nrhs, s);
  set_error("fused fine pass: unsupported order or transfer");
  return HELM_EINVAL;
}

}  // namespace

int cycle2d_fine_down(const Cycle2D& c, const float4* v, float2* r2, int nrhs, cudaStream_t s) {
  KernelTimer kt(HELM_K_FINE, s);
  switch (c.fine_kind) {
    case HELM_FINE_ROWS8: return down_rs<8>(c, v, r2, nrhs, s);
    case HELM_FINE_ROWS16: return down_rs<16>(c, v, r2, nrhs, s);
    case HELM_FINE_ROWS32: return down_rs<32>(c, v, r2, nrhs, s);
    default: break;
  }
  const dim3 grid = tiles(c.g2, kFD, kFD, nrhs);
  auto smem = [](int rw) {
    const int nx = 2 * kFD + 2 * rw + 1, nf = nx - 2;
    return (size_t)(3 * nx * nx + nf * nf + nf * kFD) * sizeof(float2);
  };
#define HELM_FD(O, RW)                                                                                  \
  if (c.fine.order == O && c.rw1 == RW) {                                                               \
    static std::atomic<bool> attr{false};                                                               \
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
  const int ntx = (c.g2.N[0] + kPX - 1) / kPX, nty = (c.g2.N[1] + kPY - 1) / kPY;
  const long long nt = (long long)ntx * nty * nrhs;
  if (!l2_offsets_fit(c, nt)) {
    set_error("fused level-2 pass: grid too large for 32-bit coefficient offsets");
    return HELM_EINVAL;
  }
  const int grid = (int)std::min<long long>(nt, 2LL * resident_sms());
  if (c.r2 == 1) l2_resid_pers_kernel<1><<<grid, kPThreads, 0, s>>>(c, r2, s2, ntx, nty, (int)nt);
  else if (c.r2 == 2) l2_resid_pers_kernel<2><<<grid, kPThreads, 0, s>>>(c, r2, s2, ntx, nty, (int)nt);
  else { set_error("fused level-2 pass: unsupported stencil radius"); return HELM_EINVAL; }
  HELM_LAUNCH_CHECK();
  return 0;
}

int cycle2d_l2_restrict(const Cycle2D& c, const float2* s2, double2* b3, int nrhs, cudaStream_t s) {
  KernelTimer kt(HELM_K_TRANSFER, s);
  const dim3 grid = tiles(c.g3, kRX, kRY, nrhs);
  if (c.rw2 == 1) l2_restrict_tile_kernel<1><<<grid, kThreads, 0, s>>>(c, s2, b3);
  else if (c.rw2 == 2) l2_restrict_tile_kernel<2><<<grid, kThreads, 0, s>>>(c, s2, b3);
  else { set_error("fused restriction: unsupported radius"); return HELM_EINVAL; }
  HELM_LAUNCH_CHECK();
  return 0;
}

int cycle2d_l2_up(const Cycle2D& c, const float2* r2, const double2* e3, float2* y2, int nrhs, cudaStream_t s) {
  KernelTimer kt(HELM_K_STENCIL, s);
  const dim3 grid = tiles(c.g2, kTX, kTY, nrhs);
  if (!l2_offsets_fit(c, 0)) {
    set_error("fused level-2 pass: grid too large for 32-bit coefficient offsets");
    return HELM_EINVAL;
  }
#define HELM_L2U(R, PW)                                                                 \
  if (c.r2 == R && c.pw2 == PW) {                                                       \
    l2_up_kernel<R, PW><<<grid, kL2Threads, 0, s>>>(c, r2, e3, y2);                     \
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
  switch (c.fine_kind) {
    case HELM_FINE_ROWS8: return up_rs<8>(c, v, y2, z, nrhs, s);
    case HELM_FINE_ROWS16: return up_rs<16>(c, v, y2, z, nrhs, s);
    case HELM_FINE_ROWS32: return up_rs<32>(c, v, y2, z, nrhs, s);
    default: break;
  }
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
