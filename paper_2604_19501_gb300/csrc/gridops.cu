// Grid kernels of the RS-CGC cycle: the fine Helmholtz operator with the absorbing
// layer (Sec. 3.1), assembled coarse stencils (Eqs. Galerkin, CoarseRealShifted),
// damped-Jacobi and red-black point relaxation (Sec. 2), and the grid transfers
// (full weighting / bilinear; cubic Eq. intergrid).
//
// Every row kernel maps one thread to one node and loops over the right-hand sides
// of a batch inside the thread, so the coefficients of a node are read once per
// batch.
#include "gridops.cuh"
#include "fineop.cuh"
#include "timer.cuh"

namespace helm {

// 1D transfer weights by radius: full weighting 1/4 [1 2 1] (radius 1) and the cubic
// 1/16 [1 4 6 4 1] of Eq. intergrid (radius 2).
__constant__ double c_transfer_w[2][5] = {{0.25, 0.5, 0.25, 0.0, 0.0},
                                          {1.0 / 16, 4.0 / 16, 6.0 / 16, 4.0 / 16, 1.0 / 16}};
// The same weights in FP32 (exact: all are dyadic), read by the FP32 kernels.
__constant__ float c_transfer_wf[2][5] = {{0.25f, 0.5f, 0.25f, 0.0f, 0.0f},
                                          {1.0f / 16, 4.0f / 16, 6.0f / 16, 4.0f / 16, 1.0f / 16}};

template <typename T> struct TransferW;
template <> struct TransferW<double> {
  __device__ static const double* get(int rw) { return c_transfer_w[rw - 1]; }
};
template <> struct TransferW<float> {
  __device__ static const float* get(int rw) { return c_transfer_wf[rw - 1]; }
};

// --------------------------------------------------------------- fine operator
template <typename T, typename TX, typename SB, typename TY, int MODE>
__global__ void __launch_bounds__(256) fine_row_kernel(FineOp op, const T* __restrict__ kap,
                                                       const c2<TX>* __restrict__ x,
                                                       const SB* __restrict__ b,
                                                       c2<TY>* __restrict__ y, int nrhs, T w,
                                                       int colour) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= op.g.size) return;
  int i, j, k;
  node_coords(op.g, idx, i, j, k);
  const c2<T> diag = fine_diag<T>(op, kap, idx, i, j, k);
  const c2<T> dinv = crecip(diag);
  const long long N = op.g.size;
  const bool active = (MODE != MODE_RB) || (((i + j + k) & 1) == colour);
  for (int r = 0; r < nrhs; ++r) {
    const long long p = r * N + idx;
    c2<T> out;
    if (MODE == MODE_JACOBI0) {
      out = cscale(cmul(dinv, cvt<T>(b[p])), w);
    } else if (MODE == MODE_RB && !active) {
      out = cvt<T>(x[p]);
    } else {
      const c2<T> Ax = fine_apply_at<T, TX>(op, diag, x, p, idx, i, j, k, kap);
      if (MODE == MODE_APPLY) {
        out = Ax;
      } else {
        const c2<T> res = cvt<T>(b[p]) - Ax;
        if (MODE == MODE_RESID) out = res;
        else out = cvt<T>(x[p]) + cscale(cmul(dinv, res), w);
      }
    }
    y[p] = cvt<TY>(out);
  }
}

// FP32, 3D: the same row operations on a 32 x 4 x 2 tile of nodes whose x and coefficients
// c = omega^2 kappa^2 (1 - i gamma), widened by one node, are staged in shared memory (all
// of a thread's staging loads issued before any store), so that the 7- or 19-point
// stencil of each node reads shared memory instead of global memory behind bounds checks.
// Staged values outside the grid are zero: every skipped term of fine_apply_at becomes an
// exact zero added at the same place of the same sum, so the results are the same.
constexpr int kFTX = 32, kFTY = 4, kFTZ = 2;
template <typename TX, typename SB, typename TY, int MODE>
__global__ void __launch_bounds__(256) fine_tile3_kernel(FineOp op, const float* __restrict__ kap,
                                                         const c2<TX>* __restrict__ x, const SB* __restrict__ b,
                                                         c2<TY>* __restrict__ y, int nrhs, float w) {
  constexpr int HX = kFTX + 2, HY = kFTY + 2, HZ = kFTZ + 2, NS = HX * HY * HZ, SPT = (NS + 255) / 256;
  static_assert(kFTX * kFTY * kFTZ == 256, "one thread per node of the tile");
  __shared__ float2 sx[NS];
  __shared__ float2 sc[NS];
  const GridDims& g = op.g;
  const int tx = threadIdx.x % kFTX, ty = (threadIdx.x / kFTX) % kFTY, tz = threadIdx.x / (kFTX * kFTY);
  const int i0 = blockIdx.x * kFTX, j0 = blockIdx.y * kFTY, k0 = blockIdx.z * kFTZ;
  const int i = i0 + tx, j = j0 + ty, k = k0 + tz;
  const bool inside = i < g.N[0] && j < g.N[1] && k < g.N[2];
  const long long N = g.size, sy = g.N[0], sz = (long long)g.N[0] * g.N[1];
  const long long idx = inside ? i + sy * j + sz * k : 0;
  const float ih2 = (float)op.inv_h2;
  // staged entry e of this thread: its grid node, or -1 outside the grid (or the tile)
  auto staged = [&](int e) -> long long {
    const int q = threadIdx.x + e * 256;
    const int gi = i0 - 1 + q % HX, gj = j0 - 1 + (q / HX) % HY, gk = k0 - 1 + q / (HX * HY);
    const bool ok = q < NS && gi >= 0 && gi < g.N[0] && gj >= 0 && gj < g.N[1] && gk >= 0 && gk < g.N[2];
    return ok ? gi + sy * gj + sz * gk : -1;
  };
  {
    // c on the widened tile, as fine_coef forms it (the same for every right-hand side)
    float2 cs[SPT];
#pragma unroll
    for (int e = 0; e < SPT; ++e) {
      const long long gq = staged(e);
      cs[e] = make_float2(0.f, 0.f);
      if (gq >= 0) {
        const int q = threadIdx.x + e * 256;
        const int gi = i0 - 1 + q % HX, gj = j0 - 1 + (q / HX) % HY, gk = k0 - 1 + q / (HX * HY);
        const float gam = op.gam32[0][gi] + op.gam32[1][gj] + op.gam32[2][gk];
        const float cre = (float)op.omega2 * kap[gq];
        cs[e] = make_float2(cre, -cre * gam);
      }
    }
#pragma unroll
    for (int e = 0; e < SPT; ++e) {
      const int q = threadIdx.x + e * 256;
      if (q < NS) sc[q] = cs[e];
    }
  }
  const int c0 = (tx + 1) + HX * ((ty + 1) + HY * (tz + 1));
  for (int r = 0; r < nrhs; ++r) {
    const c2<TX>* xr = x + r * N;
    float2 xs[SPT];
#pragma unroll
    for (int e = 0; e < SPT; ++e) {
      const long long gq = staged(e);
      xs[e] = gq >= 0 ? cvt<float>(xr[gq]) : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int e = 0; e < SPT; ++e) {
      const int q = threadIdx.x + e * 256;
      if (q < NS) sx[q] = xs[e];
    }
    __syncthreads();
    if (inside) {
      const float2 ci = sc[c0], xc = sx[c0];
      // fine_diag and fine_apply_at, from the tile
      const float2 diag = op.order == 0 ? make_float2(6.f * ih2 - ci.x, -ci.y)
                                        : make_float2(4.f * ih2 - 0.5f * ci.x, -0.5f * ci.y);
      float2 Ax;
      if (op.order == 0) {
        float2 sm = make_float2(0.f, 0.f);
        sm = sm + sx[c0 - 1];
        sm = sm + sx[c0 + 1];
        sm = sm + sx[c0 - HX];
        sm = sm + sx[c0 + HX];
        sm = sm + sx[c0 - HX * HY];
        sm = sm + sx[c0 + HX * HY];
        Ax = cmul(diag, xc) - cscale(sm, ih2);
      } else {
        Ax = cmul(diag, xc);
        const float wface = float(-2.0 / 6.0) * ih2, wedge = float(-1.0 / 6.0) * ih2;
#pragma unroll
        for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
          for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) {
              const int nz = (dx != 0) + (dy != 0) + (dz != 0);
              if (nz == 0 || nz == 3) continue;
              const int q = c0 + dx + HX * (dy + HY * dz);
              const float2 xv = sx[q];
              if (nz == 1) {
                const float2 cj = sc[q];
                const float2 m = make_float2(wface - float(1.0 / 24.0) * (ci.x + cj.x),
                                             -float(1.0 / 24.0) * (ci.y + cj.y));
                Ax = cmac(Ax, m, xv);
              } else {
                Ax = Ax + cscale(xv, wedge);
              }
            }
      }
      const long long p = r * N + idx;
      float2 out;
      if (MODE == MODE_APPLY) {
        out = Ax;
      } else {
        const float2 res = cvt<float>(b[p]) - Ax;
        if (MODE == MODE_RESID) out = res;
        else out = xc + cscale(cmul(crecip(diag), res), w);
      }
      y[p] = cvt<TY>(out);
    }
    __syncthreads();   // the tile is reloaded for the next right-hand side
  }
}

template <typename T, typename TX, typename SB, typename TY>
static int fine_dispatch(const FineOp& op, int mode, const void* kap, const void* x, const void* b,
                         void* y, int nrhs, double w, int colour, cudaStream_t s) {
  const int th = 256;
  const int bl = blocks_for(op.g.size, th);
  auto K = (const T*)kap;
  auto X = (const c2<TX>*)x;
  auto B = (const SB*)b;
  auto Y = (c2<TY>*)y;
  KernelTimer kt(HELM_K_FINE, s);
  if constexpr (std::is_same<T, float>::value) {
    if (op.g.dim == 3 && (mode == MODE_APPLY || mode == MODE_RESID || mode == MODE_JACOBI)) {
      const dim3 tg((op.g.N[0] + kFTX - 1) / kFTX, (op.g.N[1] + kFTY - 1) / kFTY, (op.g.N[2] + kFTZ - 1) / kFTZ);
      if (tg.y > 65535u || tg.z > 65535u) { set_error("fine tile grid too large"); return 1; }
      if (mode == MODE_APPLY) fine_tile3_kernel<TX, SB, TY, MODE_APPLY><<<tg, 256, 0, s>>>(op, K, X, B, Y, nrhs, (T)w);
      else if (mode == MODE_RESID) fine_tile3_kernel<TX, SB, TY, MODE_RESID><<<tg, 256, 0, s>>>(op, K, X, B, Y, nrhs, (T)w);
      else fine_tile3_kernel<TX, SB, TY, MODE_JACOBI><<<tg, 256, 0, s>>>(op, K, X, B, Y, nrhs, (T)w);
      HELM_LAUNCH_CHECK();
      return 0;
    }
  }
  switch (mode) {
    case MODE_APPLY: fine_row_kernel<T, TX, SB, TY, MODE_APPLY><<<bl, th, 0, s>>>(op, K, X, B, Y, nrhs, (T)w, colour); break;
    case MODE_RESID: fine_row_kernel<T, TX, SB, TY, MODE_RESID><<<bl, th, 0, s>>>(op, K, X, B, Y, nrhs, (T)w, colour); break;
    case MODE_JACOBI: fine_row_kernel<T, TX, SB, TY, MODE_JACOBI><<<bl, th, 0, s>>>(op, K, X, B, Y, nrhs, (T)w, colour); break;
    case MODE_JACOBI0: fine_row_kernel<T, TX, SB, TY, MODE_JACOBI0><<<bl, th, 0, s>>>(op, K, X, B, Y, nrhs, (T)w, colour); break;
    case MODE_RB: fine_row_kernel<T, TX, SB, TY, MODE_RB><<<bl, th, 0, s>>>(op, K, X, B, Y, nrhs, (T)w, colour); break;
    default: set_error("bad row mode"); return 1;
  }
  HELM_LAUNCH_CHECK();
  return 0;
}

int launch_fine_row(const FineOp& op, int mode, Prec arith, Prec xs, Prec bs, Prec ys,
                    const void* kappa2, const void* x, const void* b, void* y, int nrhs,
                    double w, int colour, cudaStream_t s) {
  if (arith == P64) {
    if (xs != P64 || bs != P64 || ys != P64) { set_error("FP64 row kernel needs c128 storage"); return 1; }
    return fine_dispatch<double, double, double2, double>(op, mode, kappa2, x, b, y, nrhs, w, colour, s);
  }
  if (xs != P32 || ys != P32) { set_error("FP32 row kernel needs c64 x/y"); return 1; }
  if (bs == P64)
    return fine_dispatch<float, float, double2, float>(op, mode, kappa2, x, b, y, nrhs, w, colour, s);
  if (bs == P_DF)
    return fine_dispatch<float, float, float4, float>(op, mode, kappa2, x, b, y, nrhs, w, colour, s);
  return fine_dispatch<float, float, float2, float>(op, mode, kappa2, x, b, y, nrhs, w, colour, s);
}

// --------------------------------------------------------------- assembled stencils
template <int DIM, int R>
int stencil_rows(Prec arith, const GridDims& g, const void* coef, const void* dinv, int mode, Prec bs,
                 const void* x, const void* b, void* y, int nrhs, double w, int colour, cudaStream_t s);

int launch_stencil_row(const GridDims& g, int r, Prec arith, const void* coef, const void* dinv,
                       int mode, Prec xs, Prec bs, Prec ys, const void* x, const void* b, void* y,
                       int nrhs, double w, int colour, cudaStream_t s) {
  if (arith == P64) {
    if (xs != P64 || bs != P64 || ys != P64) { set_error("FP64 row kernel needs c128 storage"); return 1; }
  } else if (xs != P32 || ys != P32) {
    set_error("FP32 row kernel needs c64 x/y");
    return 1;
  }
#define HELM_STENCIL_CASE(D, RR) \
  if (g.dim == D && r == RR) return stencil_rows<D, RR>(arith, g, coef, dinv, mode, bs, x, b, y, nrhs, w, colour, s);
  HELM_STENCIL_CASE(2, 1)
  HELM_STENCIL_CASE(2, 2)
  HELM_STENCIL_CASE(2, 3)
  HELM_STENCIL_CASE(3, 1)
  HELM_STENCIL_CASE(3, 2)
#undef HELM_STENCIL_CASE
  set_error("stencil radius not built for this dimension");
  return 1;
}

// --------------------------------------------------------------- transfers
template <typename T, int RW>
__global__ void __launch_bounds__(256) restrict_kernel(GridDims gf, GridDims gc,
                                                       const c2<T>* __restrict__ rf,
                                                       c2<T>* __restrict__ rc, int nrhs) {
  const long long I = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (I >= gc.size) return;
  int ci, cj, ck;
  node_coords(gc, I, ci, cj, ck);
  const T* wt = TransferW<T>::get(RW);
  const long long sy = gf.N[0];
  const long long sz = (long long)gf.N[0] * gf.N[1];
  for (int r = 0; r < nrhs; ++r) {
    c2<T> acc = mk<T>(0, 0);
    const long long base = r * gf.size;
    for (int az = (gf.dim == 3 ? -RW : 0); az <= (gf.dim == 3 ? RW : 0); ++az) {
      const int fk = 2 * ck + az;
      if (fk < 0 || fk >= gf.N[2]) continue;
      const T wz = gf.dim == 3 ? (T)wt[az + RW] : T(1);
#pragma unroll
      for (int ay = -RW; ay <= RW; ++ay) {
        const int fj = 2 * cj + ay;
        if (fj < 0 || fj >= gf.N[1]) continue;
        const T wyz = wz * (T)wt[ay + RW];
#pragma unroll
        for (int ax = -RW; ax <= RW; ++ax) {
          const int fi = 2 * ci + ax;
          if (fi < 0 || fi >= gf.N[0]) continue;
          const c2<T> v = rf[base + fi + fj * sy + fk * sz];
          const T wgt = wyz * (T)wt[ax + RW];
          acc.x = fma(wgt, v.x, acc.x);
          acc.y = fma(wgt, v.y, acc.y);
        }
      }
    }
    rc[r * gc.size + I] = acc;
  }
}

template <typename T, int RW>
__global__ void __launch_bounds__(256) prolong_add_kernel(GridDims gf, GridDims gc,
                                                          const c2<T>* __restrict__ ec,
                                                          c2<T>* __restrict__ xf, int nrhs) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= gf.size) return;
  int fi, fj, fk;
  node_coords(gf, idx, fi, fj, fk);
  const T* wt = TransferW<T>::get(RW);
  const long long sy = gc.N[0];
  const long long sz = (long long)gc.N[0] * gc.N[1];
  // coarse J with |f - 2J| <= RW along each axis; weight 2 * w(f - 2J) per axis
  const int i0 = max(0, (fi - RW + 1) >> 1), i1 = min(gc.N[0] - 1, (fi + RW) >> 1);
  const int j0 = max(0, (fj - RW + 1) >> 1), j1 = min(gc.N[1] - 1, (fj + RW) >> 1);
  int k0 = 0, k1 = 0;
  if (gf.dim == 3) { k0 = max(0, (fk - RW + 1) >> 1); k1 = min(gc.N[2] - 1, (fk + RW) >> 1); }
  for (int r = 0; r < nrhs; ++r) {
    c2<T> acc = mk<T>(0, 0);
    const long long base = r * gc.size;
    for (int K = k0; K <= k1; ++K) {
      const T wz = gf.dim == 3 ? T(2) * (T)wt[fk - 2 * K + RW] : T(1);
      for (int J = j0; J <= j1; ++J) {
        const T wyz = wz * T(2) * (T)wt[fj - 2 * J + RW];
        for (int I = i0; I <= i1; ++I) {
          const T wgt = wyz * T(2) * (T)wt[fi - 2 * I + RW];
          const c2<T> v = ec[base + I + J * sy + K * sz];
          acc.x = fma(wgt, v.x, acc.x);
          acc.y = fma(wgt, v.y, acc.y);
        }
      }
    }
    const long long p = r * gf.size + idx;
    c2<T> o = xf[p];
    xf[p] = o + acc;
  }
}

int launch_restrict(const GridDims& gf, const GridDims& gc, const Transfer& t, Prec p,
                    const void* rf, void* rc, int nrhs, cudaStream_t s) {
  const int th = 256, bl = blocks_for(gc.size, th);
  KernelTimer kt(HELM_K_TRANSFER, s);
  if (p == P64) {
    if (t.radius == 1) restrict_kernel<double, 1><<<bl, th, 0, s>>>(gf, gc, (const double2*)rf, (double2*)rc, nrhs);
    else restrict_kernel<double, 2><<<bl, th, 0, s>>>(gf, gc, (const double2*)rf, (double2*)rc, nrhs);
  } else {
    if (t.radius == 1) restrict_kernel<float, 1><<<bl, th, 0, s>>>(gf, gc, (const float2*)rf, (float2*)rc, nrhs);
    else restrict_kernel<float, 2><<<bl, th, 0, s>>>(gf, gc, (const float2*)rf, (float2*)rc, nrhs);
  }
  HELM_LAUNCH_CHECK();
  return 0;
}

int launch_prolong_add(const GridDims& gf, const GridDims& gc, const Transfer& t, Prec p,
                       const void* ec, void* xf, int nrhs, cudaStream_t s) {
  const int th = 256, bl = blocks_for(gf.size, th);
  KernelTimer kt(HELM_K_TRANSFER, s);
  if (p == P64) {
    if (t.radius == 1) prolong_add_kernel<double, 1><<<bl, th, 0, s>>>(gf, gc, (const double2*)ec, (double2*)xf, nrhs);
    else prolong_add_kernel<double, 2><<<bl, th, 0, s>>>(gf, gc, (const double2*)ec, (double2*)xf, nrhs);
  } else {
    if (t.radius == 1) prolong_add_kernel<float, 1><<<bl, th, 0, s>>>(gf, gc, (const float2*)ec, (float2*)xf, nrhs);
    else prolong_add_kernel<float, 2><<<bl, th, 0, s>>>(gf, gc, (const float2*)ec, (float2*)xf, nrhs);
  }
  HELM_LAUNCH_CHECK();
  return 0;
}

// --------------------------------------------------------------- conversions
template <typename S, typename D>
__global__ void convert_kernel(const c2<S>* __restrict__ x, c2<D>* __restrict__ y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = cvt<D>(x[i]);
}

// c128 -> double-float (hi, lo) per component
__global__ void to_df_kernel(const double2* __restrict__ x, float4* __restrict__ y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double2 v = x[i];
    const float rh = __double2float_rn(v.x), ih = __double2float_rn(v.y);
    y[i] = make_float4(rh, ih, __double2float_rn(v.x - (double)rh), __double2float_rn(v.y - (double)ih));
  }
}

__global__ void add_c128_kernel(const double2* __restrict__ x, double2* __restrict__ y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double2 a = x[i];
    double2 b = y[i];
    b.x += a.x;
    b.y += a.y;
    y[i] = b;
  }
}

int launch_add_c128(const double2* x, double2* y, long long n, cudaStream_t s) {
  const int th = 256;
  const int bl = (int)std::min<long long>(blocks_for(n, th), 152LL * 16);
  KernelTimer kt(HELM_K_TRANSFER, s);
  add_c128_kernel<<<bl, th, 0, s>>>(x, y, n);
  HELM_LAUNCH_CHECK();
  return 0;
}

int launch_convert(Prec from, Prec to, const void* x, void* y, long long n, cudaStream_t s) {
  const int th = 256;
  const int bl = (int)std::min<long long>(blocks_for(n, th), 152LL * 16);
  KernelTimer kt(HELM_K_TRANSFER, s);
  if (from == P64 && to == P_DF) to_df_kernel<<<bl, th, 0, s>>>((const double2*)x, (float4*)y, n);
  else if (from == P_DF || to == P_DF) { set_error("unsupported conversion"); return 1; }
  else if (from == P64 && to == P32) convert_kernel<double, float><<<bl, th, 0, s>>>((const double2*)x, (float2*)y, n);
  else if (from == P32 && to == P64) convert_kernel<float, double><<<bl, th, 0, s>>>((const float2*)x, (double2*)y, n);
  else if (from == P64) convert_kernel<double, double><<<bl, th, 0, s>>>((const double2*)x, (double2*)y, n);
  else convert_kernel<float, float><<<bl, th, 0, s>>>((const float2*)x, (float2*)y, n);
  HELM_LAUNCH_CHECK();
  return 0;
}

}  // namespace helm
