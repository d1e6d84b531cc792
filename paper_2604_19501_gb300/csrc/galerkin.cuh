// Host-side launchers of the Galerkin assembly kernels.
#pragma once
#include "common.cuh"

namespace helm {

// Level 2 from the fine operator: h = R1 H_h P1 (complex) and mk = R1 (omega^2 kappa^2 M) P1
// (real), both laid out [ncoef][nodes(2)].  rR / rP: transfer radii (1 = full weighting /
// linear, 2 = cubic).  *rc_out receives the coarse stencil radius.
int assemble_level2(const FineOp& op, const double* kappa2, const GridDims& gc, int rR, int rP,
                    double2* h, double* mk, int* rc_out, cudaStream_t s);

// Level 3: h3 = R2 (h2 + shift * mk2) P2 with shift = 1 - alpha3^2.
int assemble_level3(const GridDims& g2, int r2, const double2* h2, const double* mk2, double shift,
                    const GridDims& g3, int rR, int rP, double2* h3, int* rc_out, cudaStream_t s);

// dinv64 = 1 / coef[centre]; optional c64 copies of coef and dinv.  *bad set on a zero or
// non-finite diagonal.
int finalize_stencil(long long n, int ncoef, int centre, const double2* coef, double2* dinv64,
                     float2* coef32, float2* dinv32, int* bad, cudaStream_t s);

// out = coef + shift * mk over n entries (all coefficient planes).
int apply_shift(long long n, const double2* coef, const double* mk, double shift, double2* out,
                cudaStream_t s);

}  // namespace helm
