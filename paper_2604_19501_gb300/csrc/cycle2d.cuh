// Fused kernels of the 2D three-level V(1,1) cycle with damped Jacobi smoothing in FP32
// (Sec. 2, Algorithm TwoGrid applied on levels 1 and 2; Sec. 5: one pre- and one post-
// smoothing step, damped Jacobi).  Each pass keeps the intermediate fields of one tile in
// shared memory instead of writing them to HBM:
//   fine down    r2 = R1 (v - H1 x1),               x1 = w1 D1^-1 v        (v: double-float)
//   level-2 res  s2 = r2 - H2 x2,                   x2 = w2 D2^-1 r2
//   level-2 rst  b3 = R2 s2                          (c128, the coarsest right-hand side)
//   level-2 up   y2 = x2 + w2 D2^-1 (r2 - H2 x2),   x2 = w2 D2^-1 r2 + P2 e3   (e3: c128)
//   fine up      z  = x1 + w1 D1^-1 (v - H1 x1),    x1 = w1 D1^-1 v + P1 y2
// The arithmetic is that of the separate kernels (FP32, same operators and weights); only
// the order of some sums differs.
#pragma once
#include "common.cuh"

namespace helm {

// Kernels of the two fine passes: shared-memory tiles, or one warp per strip walking
// segments of 8, 16 or 32 coarse rows (16, 32, 64 fine rows) with a register window.
enum FineKind { HELM_FINE_TILES = 0, HELM_FINE_ROWS8 = 1, HELM_FINE_ROWS16 = 2, HELM_FINE_ROWS32 = 3 };

struct Cycle2D {
  FineOp fine;              // level-1 operator (FP32 tables in gam32)
  const float* kap;         // FP32 slowness squared, level-1 nodes
  GridDims g2, g3;          // level-2 and level-3 grids
  int r2;                   // stencil radius of the level-2 operator (1 or 2)
  const float2* coef2;      // level-2 stencil planes [(2 r2 + 1)^2][n2]
  const float2* dinv2;      // level-2 1 / diagonal
  int rw1, rw2, pw2;        // transfer radii: R1 = P1 (level 1-2), R2, P2 (level 2-3)
  float w1, w2;             // Jacobi weights
  int fine_kind;            // FineKind of the fine passes
};

// The passes above for nrhs right-hand sides stored back to back.
int cycle2d_fine_down(const Cycle2D& c, const float4* v, float2* r2, int nrhs, cudaStream_t s);
int cycle2d_l2_resid(const Cycle2D& c, const float2* r2, float2* s2, int nrhs, cudaStream_t s);
int cycle2d_l2_restrict(const Cycle2D& c, const float2* s2, double2* b3, int nrhs, cudaStream_t s);
int cycle2d_l2_up(const Cycle2D& c, const float2* r2, const double2* e3, float2* y2, int nrhs, cudaStream_t s);
int cycle2d_fine_up(const Cycle2D& c, const float4* v, const float2* y2, float2* z, int nrhs, cudaStream_t s);

}  // namespace helm
