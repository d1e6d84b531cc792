// Direct solver of the coarsest (level-3) operator: nested dissection with dense
// frontal matrices (multifrontal), factorised and applied on the device in complex FP64.
#pragma once
#include <vector>
#include "common.cuh"

namespace helm {

constexpr int kFwdCols = 256;    // columns per block of the forward sweep
constexpr int kFwdMinChunk = 16;   // rows per partial sum of the forward sweep: at least ...
constexpr int kFwdMaxChunk = 128;  // ... and at most
constexpr int kRhsGroup = 4;       // right-hand sides sharing each factor load in the sweeps

struct FrontDesc {
  int nS, nB;             // eliminated (separator / leaf) nodes, boundary (ancestor) nodes
  int S_off, B_off;       // offsets into the S / B node-index arrays
  long long M_off;        // forward matrix [nS][nS+nB], read as column sums (see coarse.cu)
  long long G_off;        // backward matrix F_SS^-1 F_SB, rows of stride g_ld
  int g_ld;
  int bsign;              // -1: M = [F_SS^-1 | G] (symmetric operator); +1: M = X^T
  long long aug_off;      // augmented front [nF][nF+nS] within the level work buffer
  long long U_off;        // update matrix   [nB][nB] = F_BB - F_BS F_SS^-1 F_SB
  int ent_off, ent_cnt;   // original matrix entries scattered into the front
  int kid_off, nkids;     // children (front ids)
  int cmap_off;           // this front's boundary positions inside its parent's front
  long long ctb_off;      // per front position: the children's update-vector entries added to it
  long long uv_off;       // solve scratch: update vector (nB entries)
};

struct FwdJob {
  int front, tile, s0, s1;           // column tile and rows [s0, s1) of one front
  int nchunks, chunk;                // row chunks of the tile and the index of this one
  int slot, pbase;                   // counter of the tile; first partial-sum slot of the tile
};

struct CoarseSolver {
  GridDims g;
  int r = 1;                          // stencil radius of the coarsest operator
  int nfronts = 0, nlevels = 0;
  std::vector<std::vector<int>> level_fronts;      // fronts by height (0 = leaves)
  // device arrays
  FrontDesc* d_desc = nullptr;
  int* d_S = nullptr;
  int* d_B = nullptr;
  int* d_kids = nullptr;
  int* d_cmap = nullptr;
  double2* d_factors = nullptr;       // M (and G) blocks of every front
  long long factor_entries = 0;
  long long bwd_entries = 0;          // entries of the G blocks (read again by the backward sweep)
  std::vector<int*> d_level_list;     // per level: front ids
  std::vector<FwdJob*> d_fwd_jobs;    // per level: forward-sweep blocks
  std::vector<int> n_fwd_jobs;
  std::vector<int*> big_list, small_list;   // per level: fronts by elimination path
  long long part_entries = 1;         // partial sums of the forward sweep (per right-hand side)
  int n_slots = 1;                    // column-tile counters
  double2* d_part = nullptr;
  unsigned* d_counters = nullptr;
  bool df = false;                    // factors stored and applied in double-float arithmetic
  float4* d_xd = nullptr;             // double-float copy of the backward-sweep result
  std::vector<int4*> d_bwd_rows;      // per level: (front, first row, end row) blocks
  std::vector<int> n_bwd_rows;
  long long uv_total = 0;
  int2* d_ctb = nullptr;              // children's contributions per front position
  double2* d_uv = nullptr;            // [nrhs][uv_total]
  double2* d_w = nullptr;             // [nrhs][nodes]
  int rhs_cap = 0;
  int max_nB = 0;                     // largest boundary of a front
  int* d_err = nullptr;
  long long* launches = nullptr;
};

// Symbolic analysis and numeric factorisation of the coarsest operator given by its
// assembled stencil coef (c128, [ncoef][nodes]) of radius r.  leaf_max: largest leaf box.
// symmetric: the operator is complex-symmetric (A = A^T), which halves the stored coupling.
// df: store the factors as double-float and apply them on the FP32 pipes.
int coarse_setup(CoarseSolver& cs, const GridDims& g, int r, const double2* coef, int leaf_max,
                 bool symmetric, bool df, cudaStream_t s);

// e = A^-1 b for nrhs vectors (c128, [nrhs][nodes]).
int coarse_solve(CoarseSolver& cs, const double2* b, double2* e, int nrhs, cudaStream_t s);

// The same solve with its scratch in a static device array of fixed size (no
// allocation); HELM_EINVAL when the problem needs more scratch than the array holds.
int coarse_solve_noalloc(const CoarseSolver& cs, const double2* b, double2* e, int nrhs, cudaStream_t s);

void coarse_free(CoarseSolver& cs);

}  // namespace helm
