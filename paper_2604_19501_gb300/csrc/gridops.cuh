// Host-side launchers of the grid kernels (operators, smoothers, transfers).
#pragma once
#include "common.cuh"

namespace helm {

// What a row kernel writes at every node (b: right-hand side, x: iterate, y: output):
enum RowMode {
  MODE_APPLY = 0,    // y = H x
  MODE_RESID = 1,    // y = b - H x
  MODE_JACOBI = 2,   // y = x + w D^-1 (b - H x)
  MODE_JACOBI0 = 3,  // y = w D^-1 b            (first sweep from x = 0)
  MODE_RB = 4        // y = x, except nodes of colour `colour`: x + w D^-1 (b - H x)
};

// Element types of a row kernel: arithmetic T, and the storage type of x, b, y.
// P_DF: double-float storage (float4 per complex entry), read-only input of the fine kernels.
enum Prec { P64 = 0, P32 = 1, P_DF = 2 };

// Fine-grid (level 1) row kernel.  kappa2 has the arithmetic type (double for P64).
int launch_fine_row(const FineOp& op, int mode, Prec arith, Prec xs, Prec bs, Prec ys,
                    const void* kappa2, const void* x, const void* b, void* y, int nrhs,
                    double w, int colour, cudaStream_t s);

// Assembled-stencil (levels 2, 3) row kernel.
int launch_stencil_row(const GridDims& g, int r, Prec arith, const void* coef, const void* dinv,
                       int mode, Prec xs, Prec bs, Prec ys, const void* x, const void* b, void* y,
                       int nrhs, double w, int colour, cudaStream_t s);

// rc = R rf (fine grid gf -> coarse grid gc); both in precision p.
int launch_restrict(const GridDims& gf, const GridDims& gc, const Transfer& t, Prec p,
                    const void* rf, void* rc, int nrhs, cudaStream_t s);

// xf += P ec, P = 2^d R^T.
int launch_prolong_add(const GridDims& gf, const GridDims& gc, const Transfer& t, Prec p,
                       const void* ec, void* xf, int nrhs, cudaStream_t s);

// y = convert(x) between c128 and c64 storage, n complex entries.
int launch_convert(Prec from, Prec to, const void* x, void* y, long long n, cudaStream_t s);

// y += x for n complex FP64 entries.
int launch_add_c128(const double2* x, double2* y, long long n, cudaStream_t s);

}  // namespace helm
