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

// The same row operations (apply, residual, Jacobi sweep) on a tile of nodes whose x,
// widened by the stencil radius, is staged in shared memory: every x value is read from
// memory once per tile instead of once per stencil entry, and the coefficient planes
// stream once (coalesced along x).  One node per thread; 2D tiles 32 x 8, 3D 32 x 4 x 2.
template <int DIM> struct TileShape;
template <> struct TileShape<2> { static constexpr int X = 32, Y = 8, Z = 1; };
template <> struct TileShape<3> { static constexpr int X = 32, Y = 4, Z = 2; };

template <typename T, typename TX, typename TB, typename TY, int MODE, int DIM, int R>
__global__ void __launch_bounds__(256, (DIM == 3 && sizeof(T) == sizeof(float)) ? 2 : 4) stencil_tile_kernel(GridDims g, const c2<T>* __restrict__ coef,
                                                           const c2<T>* __restrict__ dinvp,
                                                           const c2<TX>* __restrict__ x,
                                                           const c2<TB>* __restrict__ b,
                                                           c2<TY>* __restrict__ y, int nrhs, T w) {
  using S = TileShape<DIM>;
  constexpr int W = 2 * R + 1;
  constexpr int RZ = DIM == 3 ? R : 0;
  constexpr int HX = S::X + 2 * R, HY = S::Y + 2 * R, HZ = S::Z + 2 * RZ;
  __shared__ c2<T> sx[HX * HY * HZ];
  const int tx = threadIdx.x % S::X, ty = (threadIdx.x / S::X) % S::Y, tz = threadIdx.x / (S::X * S::Y);
  const int i0 = blockIdx.x * S::X, j0 = blockIdx.y * S::Y, k0 = blockIdx.z * S::Z;
  const int i = i0 + tx, j = j0 + ty, k = k0 + tz;
  const bool inside = i < g.N[0] && j < g.N[1] && (DIM == 2 || k < g.N[2]);
  const long long N = g.size;
  const long long sy = g.N[0];
  const long long sz = (long long)g.N[0] * g.N[1];
  const long long idx = inside ? i + sy * j + sz * k : 0;
  const c2<T> dinv = (inside && MODE == MODE_JACOBI) ? dinvp[idx] : mk<T>(0, 0);
  if constexpr (DIM == 3 && sizeof(T) == sizeof(float)) {
    // FP32 3D: latency-bound on its loads, so every load is issued as early as it can be.
    // The staged x values are loaded into registers before any of them is stored, the
    // first z-plane of coefficients is in flight during the staging, and each plane's
    // successor is loaded while the plane is summed.  Coefficients are read at the node
    // itself only (in bounds for any offset); an offset outside the grid meets a zero x in
    // the tile, so the sum needs no bounds checks and runs in the same order as below.
    constexpr int NS = HX * HY * HZ, SPT = (NS + 255) / 256, NP = W * W;
    static_assert(S::X * S::Y * S::Z == 256, "the launcher runs 256 threads per tile");
    const int c0 = (tx + R) + HX * ((ty + R) + HY * (tz + RZ));
    auto plane = [&](int dz, c2<T>(&cp)[NP]) {
#pragma unroll
      for (int q = 0; q < NP; ++q)
        cp[q] = coef[((q % W) + W * ((q / W) + W * (dz + R))) * N + idx];
    };
    for (int r = 0; r < nrhs; ++r) {
      const c2<TX>* xr = x + r * N;
      c2<T> ca[NP], cb[NP];
      plane(-R, ca);
      c2<T> xs[SPT];
#pragma unroll
      for (int e = 0; e < SPT; ++e) {
        const int q = threadIdx.x + e * 256;
        const int gi = i0 - R + q % HX, gj = j0 - R + (q / HX) % HY, gk = k0 - RZ + q / (HX * HY);
        const bool ok = q < NS && gi >= 0 && gi < g.N[0] && gj >= 0 && gj < g.N[1] && gk >= 0 && gk < g.N[2];
        xs[e] = ok ? cvt<T>(xr[gi + sy * gj + sz * gk]) : mk<T>(0, 0);
      }
#pragma unroll
      for (int e = 0; e < SPT; ++e) {
        const int q = threadIdx.x + e * 256;
        if (q < NS) sx[q] = xs[e];
      }
      __syncthreads();
      c2<T> Ax = mk<T>(0, 0);
      // planes alternate between ca and cb (the loop is unrolled by the plane count)
#pragma unroll
      for (int dz = -R; dz <= R; ++dz) {
        c2<T>(&cur)[NP] = ((dz + R) & 1) ? cb : ca;
        c2<T>(&nxt)[NP] = ((dz + R) & 1) ? ca : cb;
        if (dz < R) plane(dz + 1, nxt);
#pragma unroll
        for (int q = 0; q < NP; ++q) {
          const int dx = q % W - R, dy = q / W - R;
          Ax = cmac(Ax, cur[q], sx[c0 + dx + HX * (dy + HY * dz)]);
        }
      }
      if (inside) {
        const long long p = r * N + idx;
        c2<T> out;
        if (MODE == MODE_APPLY) {
          out = Ax;
        } else {
          const c2<T> res = cvt<T>(b[p]) - Ax;
          if (MODE == MODE_RESID) out = res;
          else out = sx[c0] + cscale(cmul(dinv, res), w);
        }
        y[p] = cvt<TY>(out);
      }
      __syncthreads();   // the tile is reloaded for the next right-hand side
    }
    return;
  }
  for (int r = 0; r < nrhs; ++r) {
    const c2<TX>* xr = x + r * N;
    for (int q = threadIdx.x; q < HX * HY * HZ; q += blockDim.x) {
      const int gi = i0 - R + q % HX, gj = j0 - R + (q / HX) % HY, gk = k0 - RZ + q / (HX * HY);
      c2<T> v = mk<T>(0, 0);
      if (gi >= 0 && gi < g.N[0] && gj >= 0 && gj < g.N[1] && (DIM == 2 || (gk >= 0 && gk < g.N[2])))
        v = cvt<T>(xr[gi + sy * gj + sz * gk]);
      sx[q] = v;
    }
    __syncthreads();
    if (inside) {
      const int c0 = (tx + R) + HX * ((ty + R) + HY * (tz + RZ));
      c2<T> Ax = mk<T>(0, 0);
      // one plane (3D) or the whole stencil (2D) of coefficient loads in flight at a time:
      // unrolling all 125 3D entries would hold them all in registers
#pragma unroll 1
      for (int dz = -RZ; dz <= RZ; ++dz) {
        if (k + dz < 0 || k + dz >= g.N[2]) continue;
#pragma unroll
        for (int dy = -R; dy <= R; ++dy) {
          if (j + dy < 0 || j + dy >= g.N[1]) continue;
#pragma unroll
          for (int dx = -R; dx <= R; ++dx) {
            if (i + dx < 0 || i + dx >= g.N[0]) continue;
            const int o = (dx + R) + W * ((dy + R) + W * (DIM == 3 ? dz + R : 0));
            Ax = cmac(Ax, coef[o * N + idx], sx[c0 + dx + HX * (dy + HY * dz)]);
          }
        }
      }
      const long long p = r * N + idx;
      c2<T> out;
      if (MODE == MODE_APPLY) {
        out = Ax;
      } else {
        const c2<T> res = cvt<T>(b[p]) - Ax;
        if (MODE == MODE_RESID) out = res;
        else out = sx[c0] + cscale(cmul(dinv, res), w);
      }
      y[p] = cvt<TY>(out);
    }
    __syncthreads();   // the tile is reloaded for the next right-hand side
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
  using SH = TileShape<DIM>;
  const dim3 tg((g.N[0] + SH::X - 1) / SH::X, (g.N[1] + SH::Y - 1) / SH::Y,
                DIM == 3 ? (g.N[2] + SH::Z - 1) / SH::Z : 1);
  switch (mode) {
    case MODE_APPLY: stencil_tile_kernel<T, TX, TB, TY, MODE_APPLY, DIM, R><<<tg, th, 0, s>>>(g, C, D, X, B, Y, nrhs, (T)w); break;
    case MODE_RESID: stencil_tile_kernel<T, TX, TB, TY, MODE_RESID, DIM, R><<<tg, th, 0, s>>>(g, C, D, X, B, Y, nrhs, (T)w); break;
    case MODE_JACOBI: stencil_tile_kernel<T, TX, TB, TY, MODE_JACOBI, DIM, R><<<tg, th, 0, s>>>(g, C, D, X, B, Y, nrhs, (T)w); break;
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
