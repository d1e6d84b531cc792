// Assembled-stencil (levels 2 and 3) row kernel, instantiated per (dimension, radius)
// in the stencil_rows_*.cu translation units.
#pragma once
#include "gridops.cuh"
#include "timer.cuh"

namespace helm {

template <typename T, typename TX, typename TB, typename TY, int MODE, int DIM, int R>
__global__ void __launch_bounds__(256) stencil_row_kernel(GridDims g, const c2<T>* __restrict__ coef,
                                                          const c2<T>* __restrict__ dinvp,
                                                          const c2<TX>* __restrict__ x,
                                                          const c2<TB>* __restrict__ b,
                                                          c2<TY>* __restrict__ y, int nrhs, T w,
                                                          int colour) {
  constexpr int W = 2 * R + 1;
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= g.size) return;
  int i, j, k;
  node_coords(g, idx, i, j, k);
  const long long N = g.size;
  const long long sy = g.N[0];
  const long long sz = (long long)g.N[0] * g.N[1];
  const c2<T> dinv = dinvp[idx];
  const bool active = (MODE != MODE_RB) || (((i + j + k) & 1) == colour);
  for (int r = 0; r < nrhs; ++r) {
    const long long p = r * N + idx;
    c2<T> out;
    if (MODE == MODE_JACOBI0) {
      out = cscale(cmul(dinv, cvt<T>(b[p])), w);
    } else if (MODE == MODE_RB && !active) {
      out = cvt<T>(x[p]);
    } else {
      c2<T> Ax = mk<T>(0, 0);
#pragma unroll
      for (int dz = (DIM == 3 ? -R : 0); dz <= (DIM == 3 ? R : 0); ++dz) {
        if (k + dz < 0 || k + dz >= g.N[2]) continue;
#pragma unroll
        for (int dy = -R; dy <= R; ++dy) {
          if (j + dy < 0 || j + dy >= g.N[1]) continue;
#pragma unroll
          for (int dx = -R; dx <= R; ++dx) {
            if (i + dx < 0 || i + dx >= g.N[0]) continue;
            const int o = (dx + R) + W * ((dy + R) + W * (DIM == 3 ? dz + R : 0));
            Ax = cmac(Ax, coef[o * N + idx], cvt<T>(x[p + dx + dy * sy + dz * sz]));
          }
        }
      }
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

template <typename T, typename TX, typename TB, typename TY, int DIM, int R>
int stencil_dispatch_mode(const GridDims& g, const void* coef, const void* dinv, int mode,
                                 const void* x, const void* b, void* y, int nrhs, double w,
                                 int colour, cudaStream_t s) {
  const int th = 256;
  const int bl = blocks_for(g.size, th);
  auto C = (const c2<T>*)coef;
  auto D = (const c2<T>*)dinv;
  auto X = (const c2<TX>*)x;
  auto B = (const c2<TB>*)b;
  auto Y = (c2<TY>*)y;
  KernelTimer kt(HELM_K_STENCIL, s);
  switch (mode) {
    case MODE_APPLY: stencil_row_kernel<T, TX, TB, TY, MODE_APPLY, DIM, R><<<bl, th, 0, s>>>(g, C, D, X, B, Y, nrhs, (T)w, colour); break;
    case MODE_RESID: stencil_row_kernel<T, TX, TB, TY, MODE_RESID, DIM, R><<<bl, th, 0, s>>>(g, C, D, X, B, Y, nrhs, (T)w, colour); break;
    case MODE_JACOBI: stencil_row_kernel<T, TX, TB, TY, MODE_JACOBI, DIM, R><<<bl, th, 0, s>>>(g, C, D, X, B, Y, nrhs, (T)w, colour); break;
    case MODE_JACOBI0: stencil_row_kernel<T, TX, TB, TY, MODE_JACOBI0, DIM, R><<<bl, th, 0, s>>>(g, C, D, X, B, Y, nrhs, (T)w, colour); break;
    case MODE_RB: stencil_row_kernel<T, TX, TB, TY, MODE_RB, DIM, R><<<bl, th, 0, s>>>(g, C, D, X, B, Y, nrhs, (T)w, colour); break;
    default: set_error("bad row mode"); return 1;
  }
  HELM_LAUNCH_CHECK();
  return 0;
}

template <int DIM, int R>
int stencil_rows(Prec arith, const GridDims& g, const void* coef, const void* dinv, int mode, Prec bs,
                 const void* x, const void* b, void* y, int nrhs, double w, int colour, cudaStream_t s) {
  if (arith == P64)
    return stencil_dispatch_mode<double, double, double, double, DIM, R>(g, coef, dinv, mode, x, b, y, nrhs, w, colour, s);
  if (bs == P64)
    return stencil_dispatch_mode<float, float, double, float, DIM, R>(g, coef, dinv, mode, x, b, y, nrhs, w, colour, s);
  return stencil_dispatch_mode<float, float, float, float, DIM, R>(g, coef, dinv, mode, x, b, y, nrhs, w, colour, s);
}

}  // namespace helm
