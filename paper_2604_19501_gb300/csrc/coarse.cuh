// Direct solver of the coarsest (level-3) operator: nested dissection with dense
// frontal matrices (multifrontal), factorised on the device in complex FP64 and applied
// in FP64 or, in the mixed-precision mode, from double-float copies of the factors.
#pragma once
#include <vector>
#include "common.cuh"

namespace helm {

// The solve runs as one persistent kernel (coarse_sweep.cu): a list of jobs, forward
// (leaves to root) then backward (root to leaves), dealt round-robin to resident blocks.
// Each block streams its jobs' factor rows through a ring of shared-memory stages filled
// by bulk asynchronous copies, so a job's factors arrive while it waits for the fronts it
// depends on.
constexpr int kSweepThreads = 128;   // consumer threads per block
constexpr int kStageEntries = 1024;  // 16-byte factor entries per stage (16 KiB)
constexpr int kJobRows = 256;        // most factor rows of one job
constexpr int kTile = 128;           // output columns of one job (one thread each at most)
constexpr int kPartBlock = 128;      // partial-sum entries per chunk and right-hand side
constexpr int kRhsGroup = 4;         // right-hand sides sharing each staged factor entry

// Default limit on a wait of the solve kernel, in SM clock cycles (about 2 s at 2 GHz).
constexpr long long kDefaultWaitCycles = 4000000000LL;

// Error codes the solve kernel leaves in CoarseSolver::d_err.
constexpr int kErrPivot = 1;       // factorisation: zero or non-finite pivot
constexpr int kErrSweepWait = 2;   // solve: a dependency did not complete in time
constexpr int kErrSweepCopy = 3;   // solve: a factor copy did not complete in time

struct FrontDesc {
  int nS, nB;             // eliminated (separator / leaf) nodes, boundary (ancestor) nodes
  int S_off, B_off;       // offsets into the S / B node-index arrays
  long long M_off;        // forward matrix [nS][nS+nB], read as column sums (see coarse.cu)
  long long G_off;        // backward matrix (F_SS^-1 F_SB)^T [nB][nS], read as column sums
  int g_ld;               // its row stride (nS)
  int bsign;              // -1: M = [F_SS^-1 | G] (symmetric operator); +1: M = X^T
  long long aug_off;      // augmented front [nF][nF+nS] within the level work buffer
  long long U_off;        // update matrix   [nB][nB] = F_BB - F_BS F_SS^-1 F_SB
  int ent_off, ent_cnt;   // original matrix entries scattered into the front
  int kid_off, nkids;     // children (front ids)
  int cmap_off;           // this front's boundary positions inside its parent's front
  long long ctb_off;      // per front position: the children's update-vector entries added to it
  long long uv_off;       // solve scratch: update vector (nB entries)
  int parent;             // parent front, -1 for the root
  int fwd_units;          // forward output units (column tiles of M) of the front
  int bwd_units;          // backward output units (column tiles of G^T) of the front
};

// One job of the solve kernel: partial column sums over rows [r0, r1) of a front matrix,
// for its columns [c0, c1).  Kind 0 (forward): M, rows = eliminated positions s, columns =
// front positions t.  Kind 1 (backward): G^T, rows = boundary positions, columns =
// eliminated positions.  An output unit (a column tile) is split into nchunks jobs over
// the rows; their partial sums go to consecutive blocks of the partial buffer from pbase
// on and the last job to finish (counted in slot) adds them in chunk order.
struct SweepJob {
  int front, kind;
  int r0, r1, c0, c1;
  int srows;              // rows per stage (0: the job reads no factor entries)
  int nchunks, chunk, slot, pbase;
};

// Everything the solve kernel reads about one job, flattened on the host from the job and
// its front so that a job costs one 128-byte read; a block reads its next job's record
// while it runs the current one.
struct alignas(16) SweepMeta {
  int kind, r0, r1, c0;            // as SweepJob
  int c1, srows, nchunks, chunk;
  int slot, pbase, nS, nB;         // slot and pbase as SweepJob; the front's sizes
  int S_off, B_off, bsign, nwait;  // the front's node-index offsets and update sign; dependencies (0-2)
  int wait[2], target[2];          // counter indices and the counts they must reach before the job runs
  int done, ld;                    // counter the job's output unit completes; factor row stride
  long long src;                   // factor entry of row r0, column c0
  long long ctb_off, uv_off;       // the front's child-contribution map and update-vector offsets
  int front, pad[3];
};
static_assert(sizeof(SweepMeta) == 128, "one 128-byte record per job");

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
  std::vector<int*> big_list, small_list;   // per level: fronts by elimination path
  SweepMeta* d_meta = nullptr;        // the solve kernel's job list
  int njobs = 0;
  int grid = 0;                       // resident blocks of the solve kernel (one right-hand side)
  int grid_group = 0;                 // resident blocks for right-hand-side groups
  long long part_blocks = 1;          // partial-sum blocks (kPartBlock entries per right-hand side)
  int n_slots = 0;                    // output units split into several jobs
  long long n_counters = 0;           // forward and backward completion counts, then the slots
  double2* d_part = nullptr;
  unsigned* d_counters = nullptr;
  bool df = false;                    // factors stored and applied in double-float arithmetic
  float4* d_xd = nullptr;             // double-float copy of the backward-sweep result
  long long uv_total = 0;
  int2* d_ctb = nullptr;              // children's contributions per front position
  double2* d_uv = nullptr;            // [nrhs][uv_total]
  double2* d_w = nullptr;             // [nrhs][nodes]
  int rhs_cap = 0;
  int max_nB = 0;                     // largest boundary of a front
  int* d_err = nullptr;
  long long* launches = nullptr;
  int device = -1;                    // device current at set-up (the device of every buffer above)
  long long wait_cycles = kDefaultWaitCycles;   // limit on a dependency wait of the solve kernel
};

// Symbolic analysis and numeric factorisation of the coarsest operator given by its
// assembled stencil coef (c128, [ncoef][nodes]) of radius r.  leaf_max: largest leaf box.
// symmetric: the operator is complex-symmetric (A = A^T), which halves the stored coupling.
// df: store the factors as double-float and apply them on the FP32 pipes.
// blocks: resident blocks of the solve kernel (0: all that fit on the device).
// huge_min: fronts with at least this many eliminated nodes take the blocked elimination.
int coarse_setup(CoarseSolver& cs, const GridDims& g, int r, const double2* coef, int leaf_max,
                 bool symmetric, bool df, cudaStream_t s, int blocks = 0, int huge_min = 512);

// e = A^-1 b for nrhs vectors (c128, [nrhs][nodes]).
int coarse_solve(CoarseSolver& cs, const double2* b, double2* e, int nrhs, cudaStream_t s);

// The same solve with its scratch in a static device array of fixed size (no
// allocation); HELM_EINVAL when the problem needs more scratch than the array holds.
int coarse_solve_noalloc(const CoarseSolver& cs, const double2* b, double2* e, int nrhs, cudaStream_t s);

// Host only: the plan coarse_setup builds (tree, fronts, solve jobs for `grid` resident
// blocks), checked; stats as documented for helm_coarse_plan.
int coarse_plan_stats(const GridDims& g, int r, int leaf_max, bool symmetric, int grid, long long stats[8]);

// Failure-detection check: sets the dependency-wait limit and, for job >= 0 (-1: the last
// job with a dependency), raises that job's first completion target beyond anything the
// solve can reach, so that the next solve's wait runs out and reports kErrSweepWait.
int coarse_plant_unreachable_wait(CoarseSolver& cs, long long wait_cycles, int job, cudaStream_t s);

// Large fronts (by default at least kHugeFront eliminated nodes; coarse_blocked.cu; in 3D their
// boundaries reach thousands of nodes, where an elimination pass per pivot would stream
// the whole front once per pivot): grid-wide
// assembly of the augmented front [F | I_S], blocked Gauss-Jordan elimination of its first
// nS columns (panels of 64 columns: pivot rows chosen by partial pivoting, the rest updated
// by complex FP64 matrix products), and grid-wide extraction of M, G^T and the update
// matrix.  Workspaces: w32 (nS x 64 complex FP32), piv (64 ints), dinv (64 x 64 complex),
// xbuf (64 x ld complex).
constexpr int kHugeFront = 512;
int big_front_assemble(const FrontDesc& d, const std::vector<FrontDesc>& desc, const std::vector<int>& kids,
                       double2* aug, const int2* d_ents, const double2* coef, const double2* upool, const int* d_cmap,
                       cudaStream_t s);
int big_front_eliminate(const FrontDesc& d, double2* aug, float2* w32, int* piv, double2* dinv, double2* xbuf, int* err,
                        cudaStream_t s);
int big_front_extract(const FrontDesc& d, const double2* aug, double2* factors, double2* upool, bool df, cudaStream_t s);

// Waits for the stream and reports an error a solve kernel left in d_err.
int coarse_status(const CoarseSolver& cs, cudaStream_t s);

// Solve kernel (coarse_sweep.cu): resident blocks on this device, and one launch over
// the job list with the given scratch (counters cleared first).
int sweep_grid_size(int* grid, int* grid_group);
int sweep_launch(const CoarseSolver& cs, const double2* b, double2* e, int nrhs, double2* uv, double2* w,
                 double2* part, unsigned* counters, float4* xd, cudaStream_t s);

void coarse_free(CoarseSolver& cs);

}  // namespace helm
