/*
 * helm.h -- C ABI of the GB300 RS-CGC Helmholtz solver.
 *
 * Solves the finite-difference Helmholtz equation
 *     -Lap p - k^2(x) (1 - i gamma(x)) p = q,   k = omega * kappa,
 * on a regular 2D/3D node grid padded with an absorbing layer (Yovel & Treister,
 * Sec. 1 Eq. acousitcHelm; 20-cell absorbing padding, Sec. 5), by flexible GMRES
 * (Sec. 5) preconditioned with the 3-level real-shifted coarse grid correction
 * cycle (RS-CGC, Sec. 3: Galerkin level 2, Eq. Galerkin; real-shifted Galerkin
 * level 3, Eqs. realShift and CoarseRealShifted; exact coarsest solve and damped
 * Jacobi smoothing, Sec. 2, Algorithm TwoGrid).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Grid.  An axis with n cells has n + 1 nodes, every node is an unknown and
 *   values beyond the outermost nodes are zero.  Arrays are C-ordered with x
 *   fastest: node (i, j, k) sits at i + (nx+1) * (j + (ny+1) * k).  Level 2 is
 *   the grid of every second node (n/2 cells per axis), level 3 every fourth.
 * Complex vectors.  Interleaved (re, im) pairs: "c128" = two doubles per node
 *   (complex128), "c64" = two floats (complex64).  A batch of n_rhs vectors is
 *   stored back to back: vector r starts at node offset r * nodes(level).
 * Memory.  Unless stated otherwise, pointer arguments are caller-owned device
 *   memory (e.g. torch tensors), contiguous, not retained after the call.  The
 *   context owns only the buffers it allocates.  Work is issued on the stream
 *   given in helm_opts.stream (NULL = legacy default stream); a call returns
 *   after its work is queued, except where it says it synchronises.
 * Errors.  Every call returns an int status (helm_status).  No exception or
 *   abort crosses the ABI.  helm_last_error() describes the last failure of the
 *   calling thread.
 * Threads.  Calls on different contexts may come from different host threads at
 *   the same time; calls on one context must not overlap.  The process-wide state
 *   is the once-set kernel attributes (set under atomic flags) and the array of
 *   helm_coarse_solve_noalloc, whose own rule is stated there.
 */
#ifndef HELM_H
#define HELM_H

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
typedef enum {
  HELM_OK = 0,
  HELM_EINVAL = 1,          /* bad argument: sizes, enums, NaN/Inf input, null pointer */
  HELM_ENOMEM = 2,          /* device allocation failed */
  HELM_NOT_CONVERGED = 3,   /* solve stopped at maxit; the iterate is still written */
  HELM_ECUDA = 4,           /* a CUDA runtime call or kernel launch failed */
  HELM_ENUMERIC = 5         /* zero pivot in the coarsest factorisation, NaN in the iteration */
} helm_status;

typedef enum { HELM_STENCIL_2ND = 0, HELM_STENCIL_4TH = 1 } helm_stencil;
typedef enum { HELM_INTERGRID_FW = 0, HELM_INTERGRID_CUBIC = 1, HELM_INTERGRID_LEVDEP = 2 } helm_intergrid;
typedef enum { HELM_CYCLE_V = 0, HELM_CYCLE_W = 1 } helm_cycle_kind;
typedef enum { HELM_SMOOTHER_JACOBI = 0, HELM_SMOOTHER_REDBLACK = 1 } helm_smoother;
/* HELM_FP64: every step in complex FP64.  HELM_MIXED: the cycle on levels 1-2
 * (smoothing, residuals, transfers) in complex FP32; the coarsest solve, the FGMRES
 * basis and the Arnoldi kernels (outer matvec, orthogonalisation) in double-float
 * arithmetic (an unevaluated sum of two FP32 values, about 48 significant bits, on the
 * FP32 pipes), and so is the true residual q - H p (from a double-float copy of p; error
 * about 2^-46 |H| |p|); the Givens rotations and the solution in complex FP64.  The
 * coarsest factorisation itself is computed in FP64 in both modes. */
typedef enum { HELM_FP64 = 0, HELM_MIXED = 1 } helm_precision;
typedef enum { HELM_C128 = 0, HELM_C64 = 1 } helm_dtype;
/* HELM_SOLVER_FGMRES: FGMRES(restart) preconditioned by the cycle (Sec. 5).
 * HELM_SOLVER_CYCLE: RS-CGC as a solver (Sec. 5, the iteration counts Table 3 gives
 * in parentheses): p <- p + M^-1 (q - H p) from p = 0, M^-1 one cycle, the correction
 * added and the true residual formed in FP64; helm_stats.iterations counts cycles and
 * est_relres equals relres. */
typedef enum { HELM_SOLVER_FGMRES = 0, HELM_SOLVER_CYCLE = 1 } helm_solver;

/* Problem and method options; fill with helm_default_opts() first. */
typedef struct {
  int dim;                /* 2 or 3 */
  int n[3];               /* cells per axis (x, y, z) incl. the absorbing layer; each a multiple of 4 */
  double h;               /* grid spacing */
  double omega;           /* angular frequency; k = omega * kappa */
  int abc_width[6];       /* absorbing-layer width in cells per face: x-lo, x-hi, y-lo, y-hi, z-lo, z-hi */
  double abc_gamma_max;   /* gamma = gamma_max * sum_axes (d/L)^2, d = depth into the layer */
  double alpha2;          /* real shift of level 2 (1 = plain Galerkin, the paper's method) */
  double alpha3;          /* real shift of the coarsest level (Eq. CoarseRealShifted) */
  int stencil;            /* helm_stencil; HELM_STENCIL_2ND = 5-point (2D) / 7-point (3D);
                             HELM_STENCIL_4TH = compact 9-point / 19-point (Eqs. disc4thCompact(3D)) */
  int intergrid;          /* helm_intergrid; HELM_INTERGRID_FW = full weighting + (bi/tri)linear;
                             CUBIC = Eq. intergrid on both levels (2D only); LEVDEP = Eq. levdep */
  int cycle;              /* helm_cycle_kind */
  int nu1, nu2;           /* pre- / post-smoothing sweeps */
  int smoother;           /* helm_smoother */
  double jacobi_w[2];     /* Jacobi damping on levels 1 and 2 */
  double rb_w;            /* relaxation weight of the red-black sweep */
  int precision;          /* helm_precision used by helm_solve / helm_cycle */
  int restart;            /* FGMRES restart length m (>= 1) */
  int max_rhs;            /* right-hand sides per FGMRES block: helm_solve / helm_adjoint_grad run
                             n_rhs in blocks of this size, each block sharing one cycle and one
                             coarsest solve per iteration (operators read once per block) */
  void* stream;           /* cudaStream_t for all work of this context */
  int fuse_cycle;         /* 1: the 2D mixed-precision V(1,1) Jacobi cycle runs as fused tile
                             passes (fine down, level-2 residual, restriction to level 3,
                             level-2 up, fine up); 0: one kernel per step.  Other
                             configurations always take one kernel per step. */
  int graphs;             /* 1: helm_solve / helm_adjoint_grad replay each FGMRES iteration (the
                             block's cycle, Arnoldi kernels and the read-back of the
                             convergence scalars) as a CUDA graph, captured on the second
                             use of each (iteration, block, active set); 0 (default): plain
                             launches.  The launch timer reads the events a graph records
                             after each replay.  If capture fails the context keeps plain
                             launches (HELM_INFO_GRAPHS = -1). */
  double cslp_beta;       /* RS-CGC + CSLP (Sec. 5: a complex shift of 0.03 k^2 with RS-CGC for 10
                             points per wavelength): the cycle's operators are built from
                             H_h + i cslp_beta k^2 M_h (the shift enters like the absorbing
                             term), the outer FGMRES operator stays H_h.  Level-1 component
                             calls (helm_apply, helm_residual, helm_smooth) use the cycle's
                             operator.  Default 0: plain RS-CGC. */
  int solver;             /* helm_solver used by helm_solve / helm_adjoint_grad */
  int coarse_blocks;      /* resident thread blocks of the coarsest-solve kernel: 0 (default) =
                             every block that fits on the device (fastest for one solve at a
                             time); a smaller count leaves the rest of the GPU to contexts
                             solving at the same time on other streams.  Results do not
                             depend on it. */
  int coarse_refine;      /* steps of iterative refinement after every coarsest direct solve
                             (helm_coarse_solve and the cycle): e <- e + A3^-1 (b - A3 e), the
                             residual formed in FP64 with the assembled level-3 stencil.  The
                             direct solve eliminates the nested-dissection fronts with row
                             pivoting inside each front only and stores the eliminated
                             blocks' explicit inverses; separator and leaf blocks of the
                             indefinite real-shifted operator that are close to singular
                             (condition numbers near 4e5) amplify rounding through those
                             inverses, so its backward error grows with the grid (on
                             529^2 coarsest nodes 2e-8 to 5e-8 with FP64 factors and 4e-7 to
                             7e-7 with double-float factors, measured) although the operator
                             itself is well conditioned.  One step brings the residual to the level of the
                             arithmetic.  Each step costs a second solve.  Default 0. */
  int coarse_block_min;   /* coarsest fronts with at least this many eliminated nodes are
                             eliminated in panels of 64 columns (pivot rows by partial
                             pivoting, the rest of the front updated by complex FP64 matrix
                             products), smaller ones one pivot per pass; 0 (default) = 512.
                             The two orders give the same factors up to rounding. */
  int arnoldi_passes;     /* Gram-Schmidt passes of the mixed-precision Arnoldi step: 2 = CGS2
                             (a first pass in FP32 on the high parts inside the matvec, a
                             second in double-float in a separate kernel), 1 = one pass in
                             double-float inside the matvec, the new vector's norm from
                             ||w||^2 - ||h||^2 (one kernel and one read of the basis fewer
                             per iteration); 0 (default) = 2.  FP64 contexts always use
                             CGS2.  On the 2112^2 benchmark one pass is 1.6% faster at a
                             1e-6 tolerance; at 1e-10 its single projection leaves the
                             basis less orthogonal, and the adjoint gradients lose digits
                             that CGS2 keeps. */
} helm_opts;

/* Per-solve statistics, one entry per right-hand side. */
typedef struct {
  int iterations;         /* preconditioner applications (FGMRES iterations) */
  int converged;          /* 1 if the true relative residual is below tol */
  double relres;          /* true relative residual ||q - H p|| / ||q|| in FP64 */
  double est_relres;      /* last Givens estimate |g_{j+1}| / ||q|| */
} helm_stats;

typedef struct helm_ctx helm_ctx;

/* Fills *o with defaults: 2D, h = 1, gamma_max = 1, alpha2 = alpha3 = 1,
 * 2nd-order stencil, FW transfers, V(1,1), Jacobi w = (0.8, 0.8), rb_w = 1,
 * FP64, restart 10, max_rhs 1, default stream, fuse_cycle 1, graphs 0,
 * cslp_beta 0, solver FGMRES, coarse_blocks 0, coarse_refine 0, coarse_block_min 0,
 * arnoldi_passes 0.  The caller sets dim, n,
 * omega, abc_width and the shifts. */
int helm_default_opts(helm_opts* o);

/* Builds the operator hierarchy for slowness squared kappa2 (real FP64, one
 * value per fine node, device OR host pointer; copied, not retained):
 * level-2 Galerkin stencils H_2h = R H_h P (Eq. Galerkin) and the real mass
 * part R (omega^2 kappa^2 M) P, the real-shifted level-3 stencil
 * H_4h^alpha = R (H_2h + (1 - alpha3^2) R omega^2 kappa^2 M P) P (Eqs. realShift,
 * CoarseRealShifted, by the linearity of Eq. realShiftMeaning), and the
 * direct factorisation of the level-3 operator (Sec. 3.1: the coarsest level is
 * solved directly).  Synchronises the stream.  On success *out owns device
 * memory until helm_destroy. */
int helm_setup(const helm_opts* o, const double* kappa2, helm_ctx** out);

/* Releases every buffer of the context.  NULL is accepted. */
int helm_destroy(helm_ctx* c);

/* Solves H p_r = q_r for n_rhs right-hand sides by FGMRES(restart) with the
 * RS-CGC cycle as right preconditioner, x0 = 0, until the relative residual is
 * below tol (Sec. 5: 1e-6) or maxit preconditioner applications.  q, p: c128,
 * n_rhs * nodes(1) each, device or host pointers (host buffers are staged
 * through device memory inside the call).  stats: host array of n_rhs entries
 * or NULL.  Synchronises the stream.  Returns HELM_NOT_CONVERGED if any right-
 * hand side missed tol (p still holds the last iterate). */
int helm_solve(helm_ctx* c, const void* q, void* p, int n_rhs, double tol, int maxit,
               helm_stats* stats);

/* Gradient of L = 1/2 sum_r ||P_rec p_r - d_r||^2 with respect to kappa^2, by
 * the adjoint-state method (the paper has no adjoint; standard derivation for the
 * operator of Sec. 3.1).  H is complex-symmetric, so mu_r = conj(lambda_r)
 * solves H mu_r = conj(resid_r) with the same preconditioned solver, and with the
 * mass weights w_o of the stencil (coefficient mean on every mass coupling)
 *   dL/dkappa^2_j = omega^2 sum_r Re((1 - i gamma_j) sum_o w_o (mu_j p_{j+o} + mu_{j+o} p_j) / 2),
 * i.e. omega^2 sum_r Re((1 - i gamma_j) mu_{r,j} p_{r,j}) for the 5/7-point stencil.
 * p: c128 forward fields (n_rhs * nodes); resid: c128 P_rec^T (P_rec p - d) on the
 * full grid (zero off the receivers), or in general dL/dp in the convention
 * dL = Re(sum conj(resid) dp); grad: real FP64 [nodes], ACCUMULATED into (the caller
 * zeroes it); adj: optional c128 output of the adjoint fields mu (n_rhs * nodes), or
 * NULL.  lambda = conj(mu) is the gradient with respect to the source q.  All device
 * pointers.  stats as for helm_solve (the adjoint solves).  Synchronises the stream. */
int helm_adjoint_grad(helm_ctx* c, const void* p, const void* resid, int n_rhs, double tol,
                      int maxit, double* grad, void* adj, helm_stats* stats);

/* ---- Component entry points (one step of the method each; device pointers) ---- */

/* y = H_l x on level l (1, 2 or 3) for n_rhs vectors; dtype selects c128 or
 * c64 arithmetic (level 3 is c128 only).  Level 1 is the fine operator of
 * Sec. 3.1 with the absorbing layer; levels 2-3 the assembled stencils. */
int helm_apply(helm_ctx* c, int level, int dtype, const void* x, void* y, int n_rhs);

/* One smoothing sweep on level l (1 or 2) with the smoother of the options:
 * damped Jacobi x <- x + w D^-1 (b - H x), or a red-black sweep (colour
 * (i+j+k) even first, each colour updated simultaneously).  x in/out. */
int helm_smooth(helm_ctx* c, int level, int dtype, const void* b, void* x, int n_rhs);

/* r = b - H_l x on level l. */
int helm_residual(helm_ctx* c, int level, int dtype, const void* b, const void* x, void* r,
                  int n_rhs);

/* rc = R_l rf: restriction from level l to l+1 (l = 1 or 2) with the
 * transfer of the options (full weighting 1/4[1 2 1] per axis, or the cubic
 * 1/16[1 4 6 4 1] of Eq. intergrid), out-of-grid fine nodes dropped. */
int helm_restrict(helm_ctx* c, int level, int dtype, const void* rf, void* rc, int n_rhs);

/* xf += P_l ec: prolongation from level l+1 to l, P = 2^d R^T (the paper prints
 * 2^-d R^T; the coarse-grid correction is invariant to this scaling). */
int helm_prolong_add(helm_ctx* c, int level, int dtype, const void* ec, void* xf, int n_rhs);

/* Copies the assembled stencil of level l (2 or 3) to host memory `out`
 * (real FP64 pairs, layout [ncoef][nodes(l)][2], ncoef = (2r+1)^d, offset
 * index (dx+r) + (2r+1)((dy+r) + (2r+1)(dz+r))) and returns the radius r in
 * *radius.  out may be NULL to query r only.  Synchronises the stream. */
int helm_get_stencil(helm_ctx* c, int level, double* out, int* radius);

/* e = (H_4h^alpha)^-1 b on level 3 by the direct factorisation (c128), followed by
 * helm_opts.coarse_refine steps of iterative refinement. */
int helm_coarse_solve(helm_ctx* c, const void* b, void* e, int n_rhs);

/* e = (H_4h^alpha)^-1 b like helm_coarse_solve (without the refinement steps of
 * helm_opts.coarse_refine), but the call allocates nothing.
 * The paper has no counterpart: this entry point exists for callers that cannot
 * call cudaMalloc, such as a host framework that reserves all device memory
 * up front and forbids further allocations, or a latency-sensitive loop that
 * cannot afford the device-wide synchronisation an allocation may cause.
 * (helm_coarse_solve allocates its scratch on its first call, or when n_rhs
 * grows.)  The scratch vectors live in one static device array of 2^20
 * complex FP64 entries (16 MiB), which every GPU that loads the library holds
 * until the process exits.  A solve needs, per right-hand side, the update
 * vectors of all nested-dissection fronts, two vectors over the coarsest nodes
 * and the solve's partial sums, plus completion counters (two per front, one per
 * output split across jobs); larger requests return HELM_EINVAL and do nothing.  The first call on a device looks up the array's
 * device address with that device current; later calls reuse it.  The device the
 * context was set up on must be current: a call made with another device current
 * returns HELM_EINVAL and does nothing.  All calls
 * share the array: calls that may overlap on the GPU (two streams, two
 * contexts, two threads) race and corrupt each other's results, so serialise
 * them.  Nothing in the array needs to start at zero: every entry a call reads
 * is written earlier in the same call.  b, e: c128 device pointers. */
int helm_coarse_solve_noalloc(helm_ctx* c, const void* b, void* e, int n_rhs);

/* Failure detection of the coarsest solve (test support; the paper has no counterpart).
 * Every wait of the coarsest-solve kernel is bounded: a job that waits longer than a
 * limit (SM clock cycles, default 4e9, about 2 s at the maximum clock) for a front it
 * depends on records an error, the kernel's blocks skip their remaining arithmetic and
 * return, and the call reports HELM_ECUDA with "did not complete in time" in
 * helm_last_error.  The error stays recorded in the context: every later call that runs
 * the coarsest solve reports it again (set up a new context to continue).  The GPU and
 * the CUDA context stay usable.
 * helm_coarse_wait_check exercises that path without a fault: it sets the context's
 * dependency-wait limit to wait_cycles (>= 1) and makes job `job` of the solve's job list
 * (-1: the last job that has a dependency) wait for a completion count no solve reaches,
 * so that the context's next coarsest solve runs out of time after wait_cycles.  The
 * context is only fit for that check afterwards.  HELM_EINVAL for a bad limit or job.
 * Synchronises the stream. */
int helm_coarse_wait_check(helm_ctx* c, long long wait_cycles, int job);

/* Plan of the coarsest-level direct solve, computed on the host only (no GPU and no
 * context needed), as helm_setup builds it for a level-3 grid of n_nodes[0..dim-1]
 * nodes and a stencil of radius `radius`: the nested-dissection tree (leaf boxes of at
 * most leaf_max nodes; helm_setup uses 64), the front matrices, and the job list of the
 * persistent solve kernel for `grid` resident blocks.  symmetric = 1 for a
 * complex-symmetric operator (full-weighting or cubic transfers on both levels).
 * The plan is checked against every extent the solve kernel indexes and for the job
 * order its schedule needs; HELM_EINVAL (message in helm_last_error) if a check fails.
 * stats (8 entries, caller-owned host memory): fronts, tree levels, jobs, factor
 * entries, backward-sweep entries, partial-sum blocks, split outputs, largest boundary.
 * Sec. 2 and 3.1 fix only that the coarsest level is solved exactly; the paper has no
 * counterpart of the plan itself. */
int helm_coarse_plan(int dim, const int n_nodes[3], int radius, int leaf_max, int symmetric, int grid,
                     long long stats[8]);

/* z = M^-1 v: one application of the 3-level cycle from a zero initial guess,
 * v and z in c128 (the mixed precision mode computes levels 1-2 in c64). */
int helm_cycle(helm_ctx* c, const void* v, void* z, int n_rhs);

/* Number of kernel launches this context has issued so far (all entry points). */
long long helm_launch_count(const helm_ctx* c);

/* Facts about a set-up context (for byte / flop accounting). */
typedef enum {
  HELM_INFO_NODES1 = 0,              /* nodes of level 1 (fine) */
  HELM_INFO_NODES2 = 1,              /* nodes of level 2 */
  HELM_INFO_NODES3 = 2,              /* nodes of level 3 (coarsest) */
  HELM_INFO_RADIUS2 = 3,             /* stencil radius of the level-2 operator */
  HELM_INFO_RADIUS3 = 4,             /* stencil radius of the level-3 operator */
  HELM_INFO_COARSE_ENTRIES = 5,      /* complex entries of the coarsest factors (M and G^T), each read once per solve */
  HELM_INFO_COARSE_FRONTS = 6,       /* fronts of the nested-dissection tree */
  HELM_INFO_COARSE_LEVELS = 7,       /* levels of the nested-dissection tree */
  HELM_INFO_COARSE_BWD_ENTRIES = 8,  /* complex entries the backward sweep reads per solve */
  HELM_INFO_DOUBLE_FLOAT = 9,        /* 1 if the coarsest factors and Krylov basis are double-float */
  HELM_INFO_GRAPHS = 10,             /* CUDA graphs instantiated (helm_opts.graphs); -1 after a failed capture */
  HELM_INFO_CYCLE_KERNELS = 11       /* kernels of the fused cycle's fine passes (helm_set_cycle_kernels) */
} helm_info_key;

/* *value = the quantity selected by key. */
int helm_info(const helm_ctx* c, int key, long long* value);

/* Right-hand-side blocking of helm_solve / helm_adjoint_grad (many sources through one
 * cycle; the paper solves one source at a time).  The context holds FGMRES state for at
 * most max_rhs right-hand sides per block (helm_opts.max_rhs).
 *
 * helm_set_block: solve in blocks of `block` (1 <= block <= max_rhs).
 *
 * helm_autotune_block: time one FGMRES restart cycle (helm_opts.restart iterations, or
 * probe_iters if > 0) of blocks of 1, 2, 4, ... up to min(max_rhs, n_rhs) right-hand
 * sides taken from q (device, c128, [n_rhs][nodes]), pick the size with the least time
 * per right-hand side and iteration, and set it as the block size.  *best receives it,
 * ms_per_rhs_iter (optional, caller-owned host array of at least 7 entries) the measured
 * cost of each candidate in order.  Allocates scratch for the candidate solutions. */
int helm_set_block(helm_ctx* c, int block);
int helm_autotune_block(helm_ctx* c, const void* q, int n_rhs, int probe_iters, int* best,
                        double* ms_per_rhs_iter);

/* Kernels of the two fine passes of the fused 2D cycle (helm_opts.fuse_cycle; the mixed-
 * precision V(1,1) Jacobi cycle): 0 = shared-memory tiles (16 x 16 level-2 nodes down,
 * 32 x 16 fine nodes up); 1, 2, 3 = one warp per vertical strip of 58-60 fine columns
 * walking segments of 8, 16 or 32 coarse rows with a register window of three fine rows
 * (default 2).  Every kind computes the same operators and sums in the same order.
 *
 * helm_set_cycle_kernels: use kernel kind `kind`.
 *
 * helm_autotune_cycle: time the two fine passes of every kind on n_rhs right-hand sides
 * (the context's workspaces, zero inputs), keep the fastest, return it in *best and the
 * times (ms per down + up pair, optional caller-owned host array of 4 entries) in ms.
 * HELM_EINVAL if the context's cycle has no fused passes.  Synchronises the stream. */
int helm_set_cycle_kernels(helm_ctx* c, int kind);
int helm_autotune_cycle(helm_ctx* c, int n_rhs, int* best, double* ms);

/* ---- Launch timer (tracing) ---- */

/* Kernel classes of the launch timer. */
typedef enum {
  HELM_K_FINE = 0,          /* level-1 cycle kernels: smoothing / residual on the fine grid */
  HELM_K_STENCIL = 1,       /* level-2/3 assembled-stencil smoothing / residual */
  HELM_K_TRANSFER = 2,      /* restriction, prolongation, precision conversion */
  HELM_K_COARSE = 3,        /* coarsest-level direct solve (forward + backward sweeps) */
  HELM_K_ARNOLDI_MATVEC = 4,/* w = H z fused with the first Gram-Schmidt pass */
  HELM_K_ARNOLDI_UPDATE = 5,/* w <- w - V h fused with the re-orthogonalisation pass */
  HELM_K_ARNOLDI_NORM = 6,  /* v_{j+1} = (w - V h) / ||.|| */
  HELM_K_KRYLOV_OTHER = 7,  /* solution update, true residual, norms, Givens */
  HELM_K_SETUP = 8,         /* Galerkin assembly and coarsest factorisation */
  HELM_K_COUNT = 9
} helm_kernel_class;

/* Starts timing (CUDA event pairs on the context stream) every launch of the
 * classes whose bit (1 << class) is set in mask, after clearing the totals;
 * mask = 0 stops timing.  Timing adds two event records per timed launch. */
int helm_timer_enable(helm_ctx* c, unsigned mask);

/* Waits for the timed launches and returns the summed device time (ms) and the
 * number of timed launches of class cls.  Synchronises the stream. */
int helm_timer_read(helm_ctx* c, int cls, double* total_ms, long long* launches);

const char* helm_strerror(int status);
const char* helm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* HELM_H */
