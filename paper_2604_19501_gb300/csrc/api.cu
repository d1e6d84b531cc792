// C ABI of the RS-CGC Helmholtz solver (declared in include/helm.h): context set-up,
// the 3-level cycle (Algorithm TwoGrid applied recursively, Sec. 2) and the FGMRES
// driver (Sec. 5).
#include <cmath>
#include <functional>
#include <map>
#include <set>
#include <tuple>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "../../include/helm.h"
#include "adjoint.cuh"
#include "coarse.cuh"
#include "galerkin.cuh"
#include "cycle2d.cuh"
#include "gridops.cuh"
#include "krylov.cuh"
#include "timer.cuh"

namespace helm {

thread_local long long* g_launch_counter = nullptr;
static thread_local std::string t_last_error;
std::string& last_error_ref() { return t_last_error; }
void set_error(const std::string& s) { t_last_error = s; }

}  // namespace helm

using namespace helm;

struct helm_ctx {
  helm_opts o{};
  cudaStream_t s = nullptr;
  GridDims g[3];
  FineOp fine{};
  double* d_gam = nullptr;
  float* d_gam32 = nullptr;
  FineOp fine_cyc{};                           // the cycle's fine operator (with the CSLP shift)
  RcBox rcbox{{1, 1, 1}, {0, 0, 0}};           // real-coefficient box of fine (empty until set up)
  double* d_gam_cyc = nullptr;                 // shifted absorbing tables (CSLP only)
  float* d_gam32_cyc = nullptr;
  double* kap64 = nullptr;
  float* kap32 = nullptr;
  double* h_gam = nullptr;                     // host copy of the per-axis profiles
  int r2 = 1, r3 = 1, nc2 = 9, nc3 = 9;
  double2* A2_64 = nullptr;
  double2* A2_dinv64 = nullptr;
  float2* A2_32 = nullptr;
  float2* A2_dinv32 = nullptr;
  double* Mk2 = nullptr;
  double2* A3_64 = nullptr;
  double2* A3_dinv64 = nullptr;
  Transfer tR1{}, tP1{}, tR2{}, tP2{};
  CoarseSolver cs;
  // cycle workspaces (element size of c128 so either precision fits)
  int rhs_cap = 0;
  void *l1a = nullptr, *l1b = nullptr, *l1r = nullptr;
  void *l2b = nullptr, *l2a = nullptr, *l2c = nullptr, *l2r = nullptr;
  double2 *l3b = nullptr, *l3e = nullptr;
  double2 *l3r = nullptr, *l3d = nullptr;      // coarsest-solve refinement: residual and correction
  // Krylov workspaces (one right-hand side at a time)
  double2 *V = nullptr, *w = nullptr, *r = nullptr;
  void* Z = nullptr;
  std::vector<KrylovState> ks;                // one FGMRES state per right-hand side of a block
  double* d_scal = nullptr;                    // [block][KS_COUNT] scalars of the states
  double* h_scal = nullptr;                    // pinned copy of d_scal
  double2* d_kpart = nullptr;                  // reduction scratch shared by the states
  unsigned* d_kcounter = nullptr;
  int block = 1;                               // right-hand sides per FGMRES block
  // staging for host buffers
  double2* stage = nullptr;
  long long stage_cap = 0;
  // CUDA graphs of FGMRES iterations, by (iteration, block size, active right-hand sides)
  struct GraphEntry {
    cudaGraphExec_t exec;
    long long launches;                          // kernels in the graph (for the launch count)
    std::vector<LaunchTimer::Pending> timed;     // launch-timer event pairs recorded by the graph
  };
  std::map<std::tuple<int, int, unsigned long long>, GraphEntry> graphs;
  std::set<std::tuple<int, int, unsigned long long>> graph_seen;
  std::tuple<int, int, unsigned> graph_caps{-1, -1, 0u};   // workspace capacities and timer mask at capture
  const std::vector<LaunchTimer::Pending>* graph_timed = nullptr;   // pairs of the graph last launched
  bool graphs_broken = false;
  cudaStream_t cap_stream = nullptr;         // capture stream (the context's stream may be the legacy one)
  long long launches = 0;
  int* d_bad = nullptr;
  LaunchTimer timer;
  int fine_kind = HELM_FINE_ROWS16;            // kernels of the fused fine passes (FineKind)
  float4* cdf = nullptr;                       // mixed precision: fine coefficients as double-float
  float4* xd = nullptr;                        // mixed precision: the solution as double-float [B][n]
};

namespace {

struct LaunchScope {
  long long* prev;
  LaunchTimer* prev_timer;
  explicit LaunchScope(helm_ctx* c) : prev(g_launch_counter), prev_timer(g_timer) {
    g_launch_counter = c ? &c->launches : nullptr;
    g_timer = c ? &c->timer : nullptr;
  }
  ~LaunchScope() {
    g_launch_counter = prev;
    g_timer = prev_timer;
  }
};

int fail(int code, const std::string& msg) {
  set_error(msg);
  return code;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

Transfer make_transfer(int kind) {
  Transfer t{};
  if (kind == 0) {
    t.radius = 1;
    t.w[0] = 0.25; t.w[1] = 0.5; t.w[2] = 0.25;
  } else {
    t.radius = 2;
    t.w[0] = 1.0 / 16; t.w[1] = 4.0 / 16; t.w[2] = 6.0 / 16; t.w[3] = 4.0 / 16; t.w[4] = 1.0 / 16;
  }
  return t;
}

GridDims dims_of(int dim, const int n[3], int level) {
  GridDims g{};
  g.dim = dim;
  const int f = 1 << level;
  for (int a = 0; a < 3; ++a) g.N[a] = a < dim ? n[a] / f + 1 : 1;
  g.size = (long long)g.N[0] * g.N[1] * g.N[2];
  finish_dims(g);
  return g;
}

size_t esize(Prec p) { return p == P32 ? sizeof(float2) : sizeof(double2); }

template <typename T>
int dmalloc(T** p, size_t bytes) {
  if (cudaMalloc((void**)p, std::max<size_t>(bytes, 16)) != cudaSuccess) {
    cudaGetLastError();
    set_error("cudaMalloc of " + std::to_string(bytes) + " bytes failed");
    return HELM_ENOMEM;
  }
  return 0;
}

void free_workspaces(helm_ctx* c) {
  for (void* p : {c->l1a, c->l1b, c->l1r, c->l2b, c->l2a, c->l2c, c->l2r}) cudaFree(p);
  cudaFree(c->l3b);
  cudaFree(c->l3e);
  cudaFree(c->l3r);
  cudaFree(c->l3d);
  c->l1a = c->l1b = c->l1r = c->l2b = c->l2a = c->l2c = c->l2r = nullptr;
  c->l3b = c->l3e = c->l3r = c->l3d = nullptr;
  c->rhs_cap = 0;
}

int ensure_workspaces(helm_ctx* c, int nrhs) {
  if (nrhs <= c->rhs_cap) return 0;
  free_workspaces(c);
  const size_t e = sizeof(double2);
  const size_t n1 = (size_t)c->g[0].size * nrhs, n2 = (size_t)c->g[1].size * nrhs, n3 = (size_t)c->g[2].size * nrhs;
  if (int st = dmalloc(&c->l1a, n1 * e)) return st;
  if (int st = dmalloc(&c->l1b, n1 * e)) return st;
  if (int st = dmalloc(&c->l1r, n1 * e)) return st;
  if (int st = dmalloc(&c->l2b, n2 * e)) return st;
  if (int st = dmalloc(&c->l2a, n2 * e)) return st;
  if (int st = dmalloc(&c->l2c, n2 * e)) return st;
  if (int st = dmalloc(&c->l2r, n2 * e)) return st;
  if (int st = dmalloc(&c->l3b, n3 * e)) return st;
  if (int st = dmalloc(&c->l3e, n3 * e)) return st;
  if (c->o.coarse_refine > 0) {
    if (int st = dmalloc(&c->l3r, n3 * e)) return st;
    if (int st = dmalloc(&c->l3d, n3 * e)) return st;
  }
  c->rhs_cap = nrhs;
  return 0;
}

Prec cycle_prec(const helm_ctx* c) { return c->o.precision == HELM_MIXED ? P32 : P64; }

// ---------------------------------------------------------------- row operations per level
int row_op(helm_ctx* c, int level, Prec arith, int mode, Prec xs, Prec bs, Prec ys, const void* x,
           const void* b, void* y, int nrhs, double w, int colour) {
  if (level == 0)
    return launch_fine_row(c->fine_cyc, mode, arith, xs, bs, ys, arith == P64 ? (const void*)c->kap64 : (const void*)c->kap32,
                           x, b, y, nrhs, w, colour, c->s);
  if (level == 1)
    return launch_stencil_row(c->g[1], c->r2, arith, arith == P64 ? (const void*)c->A2_64 : (const void*)c->A2_32,
                              arith == P64 ? (const void*)c->A2_dinv64 : (const void*)c->A2_dinv32, mode, xs,
                              bs, ys, x, b, y, nrhs, w, colour, c->s);
  if (arith != P64) return fail(HELM_EINVAL, "level 3 is c128 only");
  return launch_stencil_row(c->g[2], c->r3, P64, c->A3_64, c->A3_dinv64, mode, xs, bs, ys, x, b, y, nrhs, w,
                            colour, c->s);
}

// `nu` smoothing sweeps on level `level` (0-based) with right-hand side b (storage bs);
// the iterate lives in *x, *t is the second buffer of the ping-pong pair.
int smooth(helm_ctx* c, int level, Prec P, const void* b, Prec bs, void** x, void** t, int nu,
           bool from_zero, int nrhs) {
  const double wj = c->o.jacobi_w[level];
  const long long n = c->g[level].size * nrhs;
  if (nu == 0 && from_zero) HELM_CUDA_TRY(cudaMemsetAsync(*x, 0, n * esize(P), c->s));
  for (int sweep = 0; sweep < nu; ++sweep) {
    const bool zero = from_zero && sweep == 0;
    if (c->o.smoother == HELM_SMOOTHER_JACOBI) {
      const int mode = zero ? MODE_JACOBI0 : MODE_JACOBI;
      if (int st = row_op(c, level, P, mode, P, bs, P, *x, b, *t, nrhs, wj, 0)) return st;
      std::swap(*x, *t);
    } else {
      if (zero) HELM_CUDA_TRY(cudaMemsetAsync(*x, 0, n * esize(P), c->s));
      for (int colour = 0; colour < 2; ++colour) {
        if (int st = row_op(c, level, P, MODE_RB, P, bs, P, *x, b, *t, nrhs, c->o.rb_w, colour)) return st;
        std::swap(*x, *t);
      }
    }
  }
  return 0;
}

// The coarsest solve of the cycle and of helm_coarse_solve: the direct factorisation, then
// o.coarse_refine steps of iterative refinement e <- e + A3^-1 (b - A3 e) with the
// residual formed in FP64 from the assembled level-3 stencil.  The workspaces must hold
// nrhs right-hand sides (ensure_workspaces) and must not be b or e.
int coarse_apply(helm_ctx* c, const double2* b, double2* e, int nrhs) {
  if (int st = coarse_solve(c->cs, b, e, nrhs, c->s)) return st;
  for (int k = 0; k < c->o.coarse_refine; ++k) {
    if (int st = row_op(c, 2, P64, MODE_RESID, P64, P64, P64, e, b, c->l3r, nrhs, 0.0, 0)) return st;
    if (int st = coarse_solve(c->cs, c->l3r, c->l3d, nrhs, c->s)) return st;
    if (int st = launch_add_c128(c->l3d, e, c->g[2].size * nrhs, c->s)) return st;
  }
  return 0;
}

// One visit of level 2 (index 1): smoothing, residual, restriction, exact coarsest solve,
// prolongation and correction, smoothing.  x2 in/out through *x.
int visit_level2(helm_ctx* c, Prec P, void** x, void** t, bool first, int nrhs) {
  if (int st = smooth(c, 1, P, c->l2b, P, x, t, c->o.nu1, first, nrhs)) return st;
  if (int st = row_op(c, 1, P, MODE_RESID, P, P, P, *x, c->l2b, c->l2r, nrhs, 0.0, 0)) return st;
  const long long n3 = c->g[2].size * nrhs;
  if (P == P64) {
    if (int st = launch_restrict(c->g[1], c->g[2], c->tR2, P64, c->l2r, c->l3b, nrhs, c->s)) return st;
    if (int st = coarse_apply(c, c->l3b, c->l3e, nrhs)) return st;
    if (int st = launch_prolong_add(c->g[1], c->g[2], c->tP2, P64, c->l3e, *x, nrhs, c->s)) return st;
  } else {
    // restrict in c64 into the upper half of l3e, widen to c128, solve, narrow back
    float2* b32 = (float2*)c->l3e;
    if (int st = launch_restrict(c->g[1], c->g[2], c->tR2, P32, c->l2r, b32, nrhs, c->s)) return st;
    if (int st = launch_convert(P32, P64, b32, c->l3b, n3, c->s)) return st;
    if (int st = coarse_apply(c, c->l3b, c->l3e, nrhs)) return st;
    float2* e32 = (float2*)c->l3b;
    if (int st = launch_convert(P64, P32, c->l3e, e32, n3, c->s)) return st;
    if (int st = launch_prolong_add(c->g[1], c->g[2], c->tP2, P32, e32, *x, nrhs, c->s)) return st;
  }
  return smooth(c, 1, P, c->l2b, P, x, t, c->o.nu2, false, nrhs);
}

// The fused 2D cycle applies: mixed precision (double-float input, c64 output), V(1,1)
// with damped Jacobi.
bool fused_cycle(const helm_ctx* c, Prec vs, Prec zs) {
  const helm_opts& o = c->o;
  return o.fuse_cycle && o.dim == 2 && o.precision == HELM_MIXED && vs == P_DF && zs == P32 &&
         o.cycle == HELM_CYCLE_V && o.smoother == HELM_SMOOTHER_JACOBI && o.nu1 == 1 && o.nu2 == 1 &&
         (c->r2 == 1 || c->r2 == 2);
}

Cycle2D make_cycle2d(const helm_ctx* c) {
  Cycle2D cy;
  cy.fine = c->fine_cyc;
  cy.kap = c->kap32;
  cy.g2 = c->g[1];
  cy.g3 = c->g[2];
  cy.r2 = c->r2;
  cy.coef2 = c->A2_32;
  cy.dinv2 = c->A2_dinv32;
  cy.rw1 = c->tR1.radius;
  cy.rw2 = c->tR2.radius;
  cy.pw2 = c->tP2.radius;
  cy.w1 = (float)c->o.jacobi_w[0];
  cy.w2 = (float)c->o.jacobi_w[1];
  cy.fine_kind = c->fine_kind;
  return cy;
}

int run_cycle_fused(helm_ctx* c, const void* v, void* z, int nrhs) {
  const Cycle2D cy = make_cycle2d(c);
  const float4* vd = static_cast<const float4*>(v);
  float2* r2 = static_cast<float2*>(c->l2b);
  float2* s2 = static_cast<float2*>(c->l2r);
  float2* y2 = static_cast<float2*>(c->l2a);
  if (int st = cycle2d_fine_down(cy, vd, r2, nrhs, c->s)) return st;
  if (int st = cycle2d_l2_resid(cy, r2, s2, nrhs, c->s)) return st;
  if (int st = cycle2d_l2_restrict(cy, s2, c->l3b, nrhs, c->s)) return st;
  if (int st = coarse_apply(c, c->l3b, c->l3e, nrhs)) return st;
  if (int st = cycle2d_l2_up(cy, r2, c->l3e, y2, nrhs, c->s)) return st;
  return cycle2d_fine_up(cy, vd, y2, static_cast<float2*>(z), nrhs, c->s);
}

// z = M^-1 v from a zero initial guess.  v has storage vs, z storage zs.
int run_cycle(helm_ctx* c, const void* v, Prec vs, void* z, Prec zs, int nrhs) {
  if (int st = ensure_workspaces(c, nrhs)) return st;
  if (fused_cycle(c, vs, zs)) return run_cycle_fused(c, v, z, nrhs);
  const Prec P = cycle_prec(c);
  void* x = c->l1a;
  void* t = c->l1b;
  if (int st = smooth(c, 0, P, v, vs, &x, &t, c->o.nu1, true, nrhs)) return st;
  if (int st = row_op(c, 0, P, MODE_RESID, P, vs, P, x, v, c->l1r, nrhs, 0.0, 0)) return st;
  if (int st = launch_restrict(c->g[0], c->g[1], c->tR1, P, c->l1r, c->l2b, nrhs, c->s)) return st;
  void* x2 = c->l2a;
  void* t2 = c->l2c;
  const int visits = c->o.cycle == HELM_CYCLE_W ? 2 : 1;
  for (int v2 = 0; v2 < visits; ++v2)
    if (int st = visit_level2(c, P, &x2, &t2, v2 == 0, nrhs)) return st;
  if (int st = launch_prolong_add(c->g[0], c->g[1], c->tP1, P, x2, x, nrhs, c->s)) return st;
  if (int st = smooth(c, 0, P, v, vs, &x, &t, c->o.nu2, false, nrhs)) return st;
  const long long n1 = c->g[0].size * nrhs;
  if (zs == P && x == z) return 0;
  return launch_convert(P, zs, x, z, n1, c->s);
}

int sync_scal(helm_ctx* c, int B) {
  HELM_CUDA_TRY(cudaMemcpyAsync(c->h_scal, c->d_scal, sizeof(double) * KS_COUNT * B, cudaMemcpyDeviceToHost, c->s));
  HELM_CUDA_TRY(cudaStreamSynchronize(c->s));
  return 0;
}

void drop_graphs(helm_ctx* c) {
  for (auto& g : c->graphs) {
    cudaGraphExecDestroy(g.second.exec);
    for (auto& p : g.second.timed) {
      c->timer.pool.push_back(p.a);
      c->timer.pool.push_back(p.b);
    }
  }
  c->graphs.clear();
  c->graph_seen.clear();
  c->graph_timed = nullptr;
}

// After the stream has completed a replayed graph: add its launch-timer pairs.
void collect_graph_timing(helm_ctx* c) {
  if (!c->graph_timed) return;
  for (const auto& p : *c->graph_timed) {
    float ms = 0.f;
    if (!(c->timer.mask >> p.cls & 1u)) continue;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      c->timer.total_ms[p.cls] += ms;
      c->timer.count[p.cls] += 1;
    } else {
      cudaGetLastError();   // an unreadable pair is skipped, not left as the next launch's error
    }
  }
  c->graph_timed = nullptr;
}

// Issues one FGMRES iteration's work (issue()), as plain launches or as a CUDA graph:
// a key is run plainly on first use (which also makes every allocation it needs), captured
// and replayed from its second use on.  Graphs are dropped when workspaces were
// reallocated or the launch timer's classes changed since their capture; the timer's event
// pairs recorded by a graph are read back after every replay (collect_graph_timing).  A
// failed capture leaves the context on plain launches.
int run_iteration(helm_ctx* c, const std::tuple<int, int, unsigned long long>& key, const std::function<int()>& issue) {
  if (!c->o.graphs || c->graphs_broken) return issue();
  const std::tuple<int, int, unsigned> caps{c->rhs_cap, c->cs.rhs_cap, c->timer.mask};
  if (caps != c->graph_caps) {
    drop_graphs(c);
    c->graph_caps = caps;
  }
  auto it = c->graphs.find(key);
  if (it != c->graphs.end()) {
    HELM_CUDA_TRY(cudaGraphLaunch(it->second.exec, c->s));
    c->launches += it->second.launches;
    c->graph_timed = &it->second.timed;
    return 0;
  }
  if (!c->graph_seen.count(key)) {
    c->graph_seen.insert(key);
    return issue();
  }
  const long long before = c->launches;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ex = nullptr;
  // The work is recorded on a private stream (the legacy default stream cannot be
  // captured) and the graph launched on the context's stream, which keeps its order.
  bool ok = c->cap_stream || cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) == cudaSuccess;
  const cudaStream_t user = c->s;
  if (ok) ok = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  const size_t p0 = c->timer.pending.size();
  std::vector<LaunchTimer::Pending> timed;
  if (ok) {
    c->s = c->cap_stream;
    const int st = issue();
    c->s = user;
    ok = cudaStreamEndCapture(c->cap_stream, &g) == cudaSuccess && st == 0 && g != nullptr &&
         cudaGraphInstantiate(&ex, g, 0) == cudaSuccess;
  }
  // timer pairs issued during the capture belong to the graph, not to the plain timeline
  if (c->timer.pending.size() > p0) {
    timed.assign(c->timer.pending.begin() + p0, c->timer.pending.end());
    c->timer.pending.resize(p0);
  }
  if (g) cudaGraphDestroy(g);
  if (!ok) {
    // the work was only recorded, not run: run it plainly and stay on plain launches
    cudaGetLastError();
    for (auto& p : timed) {
      c->timer.pool.push_back(p.a);
      c->timer.pool.push_back(p.b);
    }
    c->graphs_broken = true;
    drop_graphs(c);
    c->launches = before;
    return issue();
  }
  auto& entry = c->graphs[key];
  entry = helm_ctx::GraphEntry{ex, c->launches - before, std::move(timed)};
  HELM_CUDA_TRY(cudaGraphLaunch(ex, c->s));
  c->graph_timed = &entry.timed;
  return 0;
}

// FGMRES(m) for a block of B right-hand sides (device pointers, B * nodes each).  The
// cycle and the coarsest solve run once per iteration for the whole block (operators
// read once per block); each right-hand side keeps its own Arnoldi basis, Givens
// rotations and convergence test, and leaves the block's Arnoldi steps once it has
// converged.  Per right-hand side the arithmetic is that of a single solve.
// Layouts: V [m+1][B][n], Z [m][B][n], w and r [B][n].
// Gram-Schmidt passes of the mixed-precision Arnoldi step when helm_opts.arnoldi_passes is 0
constexpr int kDefaultArnoldiPasses = 2;

int fgmres_block(helm_ctx* c, const double2* q, double2* p, int B, double tol, int maxit, helm_stats* out) {
  const long long n = c->g[0].size;
  const int m = c->o.restart;
  const Prec zp = cycle_prec(c);
  const size_t zes = esize(zp);
  // mixed precision: the basis V and w are double-float (float4), arithmetic on FP32 pipes
  const bool df = zp == P32;
  const long long vstride = (long long)B * n;
  auto Vp = [&](int i, int r) { return c->V + ((size_t)i * B + r) * n; };
  auto Vd = [&](int i, int r) { return reinterpret_cast<float4*>(c->V) + ((size_t)i * B + r) * n; };
  auto Zp = [&](int j, int r) { return (char*)c->Z + ((size_t)j * B + r) * n * zes; };
  auto S = [&](int r) { return c->h_scal + (size_t)r * KS_COUNT; };
  HELM_CUDA_TRY(cudaMemsetAsync(p, 0, (size_t)B * n * sizeof(double2), c->s));
  for (int r = 0; r < B; ++r)
    if (int st = k_norm(c->ks[r], n, q + (size_t)r * n, c->r + (size_t)r * n, c->s)) return st;
  if (int st = sync_scal(c, B)) return st;
  std::vector<double> bnorm(B), beta(B), est(B);
  std::vector<int> its(B, 0), k(B, 0);
  std::vector<char> done(B, 0), part(B, 0), act(B, 0);
  for (int r = 0; r < B; ++r) {
    bnorm[r] = S(r)[KS_BNORM];
    beta[r] = S(r)[KS_BETA];
    if (!std::isfinite(bnorm[r])) return fail(HELM_EINVAL, "right-hand side is not finite");
    est[r] = bnorm[r] > 0 ? beta[r] / bnorm[r] : 0.0;
    if (bnorm[r] == 0.0) done[r] = 1;
  }
  while (true) {
    int npart = 0;
    for (int r = 0; r < B; ++r) {
      part[r] = !done[r] && beta[r] / bnorm[r] >= tol && its[r] < maxit;
      act[r] = part[r];
      k[r] = 0;
      npart += part[r];
    }
    if (npart == 0) break;
    for (int r = 0; r < B; ++r) {
      if (!part[r]) continue;
      if (df) {
        if (int st = k_start_cycle_df(c->ks[r], n, c->r + (size_t)r * n, Vd(0, r), c->s)) return st;
      } else if (int st = k_start_cycle(c->ks[r], n, c->r + (size_t)r * n, Vp(0, r), c->s)) {
        return st;
      }
    }
    for (int j = 0; j < m; ++j) {
      // the iteration's device work: cycle for the block, Arnoldi steps, scalars to the host
      auto issue = [&]() -> int {
        if (df) {
          if (int st = run_cycle(c, Vd(j, 0), P_DF, Zp(j, 0), zp, B)) return st;
        } else if (int st = run_cycle(c, Vp(j, 0), P64, Zp(j, 0), zp, B)) {
          return st;
        }
        for (int r = 0; r < B; ++r) {
          if (!act[r]) continue;
          if (df) {
            if (int st = k_arnoldi_df(c->ks[r], c->fine, c->rcbox, c->cdf, (const float2*)Zp(j, r),
                                      reinterpret_cast<float4*>(c->w) + (size_t)r * n, Vd(0, r), vstride, j,
                                      c->o.arnoldi_passes ? c->o.arnoldi_passes : kDefaultArnoldiPasses, c->s))
              return st;
          } else if (int st = k_arnoldi(c->ks[r], c->fine, c->kap64, Zp(j, r), zp, c->w + (size_t)r * n, Vp(0, r),
                                        vstride, j, c->s)) {
            return st;
          }
        }
        HELM_CUDA_TRY(cudaMemcpyAsync(c->h_scal, c->d_scal, sizeof(double) * KS_COUNT * B, cudaMemcpyDeviceToHost, c->s));
        return 0;
      };
      unsigned long long mask = 0;
      for (int r = 0; r < B && r < 64; ++r) mask |= (unsigned long long)(act[r] != 0) << r;
      if (B > 64) {
        if (int st = issue()) return st;
      } else if (int st = run_iteration(c, std::make_tuple(j, B, mask), issue)) {
        return st;
      }
      HELM_CUDA_TRY(cudaStreamSynchronize(c->s));
      collect_graph_timing(c);
      int nact = 0;
      for (int r = 0; r < B; ++r) {
        if (!act[r]) continue;
        ++its[r];
        k[r] = j + 1;
        est[r] = S(r)[KS_EST];
        if (!std::isfinite(est[r])) return fail(HELM_ENUMERIC, "non-finite residual estimate");
        if (est[r] < tol || its[r] >= maxit || S(r)[KS_HN] == 0.0) act[r] = 0;
        nact += act[r];
      }
      if (nact == 0) break;
      for (int r = 0; r < B; ++r) {
        if (!act[r]) continue;
        if (df) {
          if (int st = k_normalize_df(c->ks[r], n, reinterpret_cast<float4*>(c->w) + (size_t)r * n, Vd(0, r), vstride, j,
                                      Vd(j + 1, r), c->s))
            return st;
        } else if (int st = k_normalize(c->ks[r], n, c->w + (size_t)r * n, Vp(0, r), vstride, j, Vp(j + 1, r), c->s)) {
          return st;
        }
      }
    }
    for (int r = 0; r < B; ++r) {
      if (!part[r]) continue;
      float4* xd = df ? c->xd + (size_t)r * n : nullptr;
      if (int st = k_update_solution(c->ks[r], n, p + (size_t)r * n, Zp(0, r), zp, vstride, k[r], xd, c->s))
        return st;
      // mixed precision: the true residual in double-float from the copy of x just written
      if (df) {
        if (int st = k_true_residual_df(c->ks[r], c->fine, c->rcbox, c->cdf, q + (size_t)r * n, xd, c->r + (size_t)r * n, c->s))
          return st;
      } else if (int st = k_true_residual(c->ks[r], c->fine, c->kap64, q + (size_t)r * n, p + (size_t)r * n,
                                          c->r + (size_t)r * n, c->s)) {
        return st;
      }
    }
    if (int st = sync_scal(c, B)) return st;
    for (int r = 0; r < B; ++r) {
      if (!part[r]) continue;
      beta[r] = S(r)[KS_BETA];
      if (!std::isfinite(beta[r])) return fail(HELM_ENUMERIC, "non-finite residual");
    }
  }
  for (int r = 0; r < B; ++r) {
    helm_stats res{0, 1, 0.0, 0.0};
    if (bnorm[r] > 0) {
      res.iterations = its[r];
      res.relres = beta[r] / bnorm[r];
      res.converged = res.relres < tol ? 1 : 0;
      res.est_relres = est[r];
    }
    if (out) out[r] = res;
  }
  return coarse_status(c->cs, c->s);
}

// RS-CGC as a solver (Sec. 5, the parenthesised iteration counts of Table 3): the
// stationary iteration p <- p + M^-1 (q - H p) from p = 0, M^-1 one cycle, until the true
// relative residual ||q - H p|| / ||q|| (FP64) is below tol or maxit cycles ran.  The cycle
// runs once per iteration for the whole block; a right-hand side that has converged keeps
// its iterate (its correction is not added) and its residual.  The correction is added
// and the residual formed in FP64 in both precision modes.  The iteration works on context
// buffers only, so that a captured iteration replays for any q and p: the iterate x in
// w [B][n], a copy of q in V slot 1, the residual r [B][n]; the cycle reads its double-
// float input from V slot 0 (mixed precision) and writes Z [B][n].
int stationary_block(helm_ctx* c, const double2* q, double2* p, int B, double tol, int maxit, helm_stats* out) {
  const long long n = c->g[0].size;
  const Prec zp = cycle_prec(c);
  const bool df = zp == P32;
  const size_t zes = esize(zp);
  const size_t bytes = (size_t)B * n * sizeof(double2);
  double2* x = c->w;
  double2* qc = c->V + (size_t)B * n;
  auto S = [&](int r) { return c->h_scal + (size_t)r * KS_COUNT; };
  HELM_CUDA_TRY(cudaMemsetAsync(x, 0, bytes, c->s));
  for (int r = 0; r < B; ++r)
    if (int st = k_norm(c->ks[r], n, q + (size_t)r * n, qc + (size_t)r * n, c->s)) return st;
  HELM_CUDA_TRY(cudaMemcpyAsync(c->r, qc, bytes, cudaMemcpyDeviceToDevice, c->s));
  if (int st = sync_scal(c, B)) return st;
  std::vector<double> bnorm(B), beta(B);
  std::vector<int> its(B, 0);
  std::vector<char> act(B, 0);
  for (int r = 0; r < B; ++r) {
    bnorm[r] = S(r)[KS_BNORM];
    beta[r] = S(r)[KS_BETA];
    if (!std::isfinite(bnorm[r])) return fail(HELM_EINVAL, "right-hand side is not finite");
  }
  while (true) {
    int nact = 0;
    unsigned long long mask = 0;
    for (int r = 0; r < B; ++r) {
      act[r] = bnorm[r] > 0 && beta[r] / bnorm[r] >= tol && its[r] < maxit;
      nact += act[r];
      if (r < 64) mask |= (unsigned long long)(act[r] != 0) << r;
    }
    if (nact == 0) break;
    // the iteration's device work: cycle for the block, corrections and residuals of the
    // active right-hand sides, residual norms to the host
    auto issue = [&]() -> int {
      if (df) {
        float4* vd = reinterpret_cast<float4*>(c->V);
        if (int st = launch_convert(P64, P_DF, c->r, vd, (long long)B * n, c->s)) return st;
        if (int st = run_cycle(c, vd, P_DF, c->Z, zp, B)) return st;
      } else if (int st = run_cycle(c, c->r, P64, c->Z, zp, B)) {
        return st;
      }
      for (int r = 0; r < B; ++r) {
        if (!act[r]) continue;
        double2* xr = x + (size_t)r * n;
        float4* xd = df ? c->xd + (size_t)r * n : nullptr;
        if (int st = k_add_correction(n, xr, (const char*)c->Z + (size_t)r * n * zes, zp, xd, c->s)) return st;
        if (df) {
          if (int st = k_true_residual_df(c->ks[r], c->fine, c->rcbox, c->cdf, qc + (size_t)r * n, xd, c->r + (size_t)r * n, c->s))
            return st;
        } else if (int st = k_true_residual(c->ks[r], c->fine, c->kap64, qc + (size_t)r * n, xr, c->r + (size_t)r * n,
                                            c->s)) {
          return st;
        }
      }
      HELM_CUDA_TRY(cudaMemcpyAsync(c->h_scal, c->d_scal, sizeof(double) * KS_COUNT * B, cudaMemcpyDeviceToHost, c->s));
      return 0;
    };
    if (B > 64) {
      if (int st = issue()) return st;
    } else if (int st = run_iteration(c, std::make_tuple(-1, B, mask), issue)) {
      return st;
    }
    HELM_CUDA_TRY(cudaStreamSynchronize(c->s));
    collect_graph_timing(c);
    for (int r = 0; r < B; ++r) {
      if (!act[r]) continue;
      ++its[r];
      beta[r] = S(r)[KS_BETA];
      if (!std::isfinite(beta[r])) return fail(HELM_ENUMERIC, "non-finite residual");
    }
  }
  for (int r = 0; r < B; ++r) {
    helm_stats res{0, 1, 0.0, 0.0};
    if (bnorm[r] > 0) {
      res.iterations = its[r];
      res.relres = beta[r] / bnorm[r];
      res.converged = res.relres < tol ? 1 : 0;
      res.est_relres = res.relres;
    }
    if (out) out[r] = res;
  }
  HELM_CUDA_TRY(cudaMemcpyAsync(p, x, bytes, cudaMemcpyDeviceToDevice, c->s));
  return coarse_status(c->cs, c->s);
}

// One block of right-hand sides by the context's solver (helm_opts.solver).
int solve_block(helm_ctx* c, const double2* q, double2* p, int B, double tol, int maxit, helm_stats* out) {
  if (c->o.solver == HELM_SOLVER_CYCLE) return stationary_block(c, q, p, B, tol, maxit, out);
  return fgmres_block(c, q, p, B, tol, maxit, out);
}

int check_level(const helm_ctx* c, int level, int lo, int hi) {
  if (level < lo || level > hi) return fail(HELM_EINVAL, "level out of range");
  return 0;
}

Prec dtype_prec(int dtype) { return dtype == HELM_C64 ? P32 : P64; }

}  // namespace

extern "C" {

int helm_default_opts(helm_opts* o) {
  if (!o) return fail(HELM_EINVAL, "null options");
  std::memset(o, 0, sizeof(*o));
  o->dim = 2;
  o->h = 1.0;
  o->abc_gamma_max = 1.0;
  o->alpha2 = 1.0;
  o->alpha3 = 1.0;
  o->stencil = HELM_STENCIL_2ND;
  o->intergrid = HELM_INTERGRID_FW;
  o->cycle = HELM_CYCLE_V;
  o->nu1 = 1;
  o->nu2 = 1;
  o->smoother = HELM_SMOOTHER_JACOBI;
  o->jacobi_w[0] = 0.8;
  o->jacobi_w[1] = 0.8;
  o->rb_w = 1.0;
  o->precision = HELM_FP64;
  o->restart = 10;
  o->max_rhs = 1;
  o->stream = nullptr;
  o->fuse_cycle = 1;
  o->graphs = 0;
  o->cslp_beta = 0.0;
  o->solver = HELM_SOLVER_FGMRES;
  o->coarse_blocks = 0;
  o->coarse_refine = 0;
  o->coarse_block_min = 0;
  o->arnoldi_passes = 0;
  return HELM_OK;
}

int helm_setup(const helm_opts* o, const double* kappa2, helm_ctx** out) {
  if (!o || !kappa2 || !out) return fail(HELM_EINVAL, "null argument");
  *out = nullptr;
  if (o->dim != 2 && o->dim != 3) return fail(HELM_EINVAL, "dim must be 2 or 3");
  for (int a = 0; a < o->dim; ++a)
    if (o->n[a] < 4 || o->n[a] % 4) return fail(HELM_EINVAL, "cells per axis must be a positive multiple of 4");
  if (!(o->h > 0) || !std::isfinite(o->h) || !(o->omega >= 0) || !std::isfinite(o->omega))
    return fail(HELM_EINVAL, "h must be > 0 and omega >= 0, both finite");
  for (int f = 0; f < 2 * o->dim; ++f)
    if (o->abc_width[f] < 0 || o->abc_width[f] > o->n[f / 2]) return fail(HELM_EINVAL, "bad absorbing-layer width");
  if (!std::isfinite(o->alpha2) || !std::isfinite(o->alpha3) || !std::isfinite(o->abc_gamma_max) ||
      !std::isfinite(o->cslp_beta) || o->cslp_beta < 0.0)
    return fail(HELM_EINVAL, "non-finite shift or layer amplitude");
  if (o->solver != HELM_SOLVER_FGMRES && o->solver != HELM_SOLVER_CYCLE) return fail(HELM_EINVAL, "bad solver");
  if (o->coarse_blocks < 0) return fail(HELM_EINVAL, "coarse_blocks must be >= 0");
  if (o->coarse_refine < 0 || o->coarse_refine > 8) return fail(HELM_EINVAL, "coarse_refine must be in [0, 8]");
  if (o->coarse_block_min < 0) return fail(HELM_EINVAL, "coarse_block_min must be >= 0");
  if (o->arnoldi_passes < 0 || o->arnoldi_passes > 2) return fail(HELM_EINVAL, "arnoldi_passes must be 0, 1 or 2");
  if (o->stencil != HELM_STENCIL_2ND && o->stencil != HELM_STENCIL_4TH) return fail(HELM_EINVAL, "bad stencil");
  if (o->intergrid < HELM_INTERGRID_FW || o->intergrid > HELM_INTERGRID_LEVDEP)
    return fail(HELM_EINVAL, "bad intergrid transfer");
  if (o->dim == 3 && o->intergrid == HELM_INTERGRID_CUBIC)
    return fail(HELM_EINVAL, "3D cubic transfers (343-point coarsest stencil) are not built; use lev-dep");
  if (o->cycle != HELM_CYCLE_V && o->cycle != HELM_CYCLE_W) return fail(HELM_EINVAL, "bad cycle");
  if (o->smoother != HELM_SMOOTHER_JACOBI && o->smoother != HELM_SMOOTHER_REDBLACK)
    return fail(HELM_EINVAL, "bad smoother");
  if (o->nu1 < 0 || o->nu2 < 0 || o->nu1 + o->nu2 > 16) return fail(HELM_EINVAL, "bad sweep counts");
  if (o->precision != HELM_FP64 && o->precision != HELM_MIXED) return fail(HELM_EINVAL, "bad precision");
  if (o->restart < 1 || o->restart > 40) return fail(HELM_EINVAL, "restart must be in [1, 40]");
  if (o->max_rhs < 1) return fail(HELM_EINVAL, "max_rhs must be >= 1");
  {
    long long nodes = 1;
    for (int a = 0; a < o->dim; ++a) nodes *= (o->n[a] + 1);
    if (nodes >= (1LL << 31)) return fail(HELM_EINVAL, "more than 2^31 - 1 nodes per right-hand side");
  }

  helm_ctx* c = new helm_ctx();
  c->o = *o;
  if (c->o.dim == 2) c->o.n[2] = 0;
  c->s = (cudaStream_t)o->stream;
  LaunchScope scope(c);
  auto bail = [&](int st) { helm_destroy(c); return st; };
  for (int l = 0; l < 3; ++l) c->g[l] = dims_of(o->dim, c->o.n, l);
  const long long n1 = c->g[0].size;

  // medium: validated on the host, stored as FP64 and FP32
  std::vector<double> k64(n1);
  cudaError_t ce = is_device_ptr(kappa2)
                       ? cudaMemcpy(k64.data(), kappa2, n1 * sizeof(double), cudaMemcpyDeviceToHost)
                       : cudaMemcpy(k64.data(), kappa2, n1 * sizeof(double), cudaMemcpyHostToHost);
  if (ce != cudaSuccess) return bail(fail(HELM_ECUDA, std::string("reading kappa2: ") + cudaGetErrorString(ce)));
  std::vector<float> k32(n1);
  for (long long i = 0; i < n1; ++i) {
    if (!std::isfinite(k64[i]) || k64[i] < 0) return bail(fail(HELM_EINVAL, "kappa2 must be finite and >= 0"));
    k32[i] = (float)k64[i];
  }
  if (int st = dmalloc(&c->kap64, n1 * sizeof(double))) return bail(st);
  if (int st = dmalloc(&c->kap32, n1 * sizeof(float))) return bail(st);
  if (cudaMemcpy(c->kap64, k64.data(), n1 * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c->kap32, k32.data(), n1 * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
    return bail(fail(HELM_ECUDA, "uploading kappa2"));

  // absorbing profile per axis: gamma_max * ((lo - i)/lo)^2 or ((i - (n - hi))/hi)^2
  const int tot = c->g[0].N[0] + c->g[0].N[1] + c->g[0].N[2];
  std::vector<double> gam(tot, 0.0);
  int off = 0;
  for (int a = 0; a < 3; ++a) {
    const int nc = c->g[0].N[a] - 1;
    if (a < o->dim) {
      const int lo = o->abc_width[2 * a], hi = o->abc_width[2 * a + 1];
      for (int i = 0; i <= nc; ++i) {
        double t = 0.0;
        if (lo > 0 && i < lo) t += ((double)(lo - i) / lo) * ((double)(lo - i) / lo);
        if (hi > 0 && i > nc - hi) t += ((double)(i - (nc - hi)) / hi) * ((double)(i - (nc - hi)) / hi);
        gam[off + i] = o->abc_gamma_max * t;
      }
    }
    off += c->g[0].N[a];
  }
  if (int st = dmalloc(&c->d_gam, tot * sizeof(double))) return bail(st);
  if (cudaMemcpy(c->d_gam, gam.data(), tot * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
    return bail(fail(HELM_ECUDA, "uploading absorbing profile"));
  c->h_gam = new double[tot];
  std::memcpy(c->h_gam, gam.data(), tot * sizeof(double));
  c->fine.g = c->g[0];
  c->fine.order = o->stencil == HELM_STENCIL_4TH ? 1 : 0;
  c->fine.inv_h2 = 1.0 / (o->h * o->h);
  c->fine.omega2 = o->omega * o->omega;
  c->fine.gam[0] = c->d_gam;
  c->fine.gam[1] = c->d_gam + c->g[0].N[0];
  c->fine.gam[2] = c->d_gam + c->g[0].N[0] + c->g[0].N[1];
  for (int a = 0, off2 = 0; a < o->dim; off2 += c->g[0].N[a], ++a) {
    // the real-coefficient box of the double-float operator: indices with gamma zero at
    // themselves and their neighbours; left empty unless they form one contiguous range
    const int na = c->g[0].N[a];
    auto zero = [&](int i) { return i < 0 || i >= na || gam[off2 + i] == 0.0; };
    int lo = -1, hi = -2;
    for (int i = 0; i < na; ++i)
      if (zero(i - 1) && zero(i) && zero(i + 1)) {
        if (lo < 0) lo = i;
        hi = i;
      }
    bool contiguous = lo >= 0;
    for (int i = lo; contiguous && i <= hi; ++i) contiguous = zero(i - 1) && zero(i) && zero(i + 1);
    c->rcbox.lo[a] = contiguous ? lo : 1;
    c->rcbox.hi[a] = contiguous ? hi : 0;
  }
  {
    std::vector<float> g32(gam.begin(), gam.end());
    if (int st = dmalloc(&c->d_gam32, tot * sizeof(float))) return bail(st);
    if (cudaMemcpy(c->d_gam32, g32.data(), tot * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
      return bail(fail(HELM_ECUDA, "uploading absorbing profile"));
    c->fine.gam32[0] = c->d_gam32;
    c->fine.gam32[1] = c->d_gam32 + c->g[0].N[0];
    c->fine.gam32[2] = c->d_gam32 + c->g[0].N[0] + c->g[0].N[1];
  }
  // the cycle's operator: with the CSLP shift the x-axis table carries gamma + beta, so
  // that gamma_x + gamma_y (+ gamma_z) + beta enters every coefficient
  c->fine_cyc = c->fine;
  if (o->cslp_beta != 0.0) {
    std::vector<double> gs(gam);
    for (int i = 0; i < c->g[0].N[0]; ++i) gs[i] += o->cslp_beta;
    std::vector<float> gs32(gs.begin(), gs.end());
    if (int st = dmalloc(&c->d_gam_cyc, tot * sizeof(double))) return bail(st);
    if (int st = dmalloc(&c->d_gam32_cyc, tot * sizeof(float))) return bail(st);
    if (cudaMemcpy(c->d_gam_cyc, gs.data(), tot * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c->d_gam32_cyc, gs32.data(), tot * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
      return bail(fail(HELM_ECUDA, "uploading the shifted absorbing profile"));
    for (int a = 0, off2 = 0; a < 3; off2 += c->g[0].N[a], ++a) {
      c->fine_cyc.gam[a] = c->d_gam_cyc + off2;
      c->fine_cyc.gam32[a] = c->d_gam32_cyc + off2;
    }
  }

  // transfers: full weighting / linear everywhere (FW); the cubic stencil of Eq.
  // intergrid everywhere (cubic); cubic except the restriction to level 3 (Eq. levdep)
  const int cubic1 = o->intergrid != HELM_INTERGRID_FW;
  c->tR1 = c->tP1 = make_transfer(cubic1);
  c->tR2 = make_transfer(o->intergrid == HELM_INTERGRID_CUBIC);
  c->tP2 = make_transfer(cubic1);
  const int r2 = (c->tR1.radius + 1 + c->tP1.radius) / 2;
  const int r3 = (c->tR2.radius + r2 + c->tP2.radius) / 2;
  auto ncoef = [&](int r) { const int w = 2 * r + 1; return o->dim == 3 ? w * w * w : w * w; };

  // level 2: H_2h = R1 H_h P1 and the real mass part R1 omega^2 kappa^2 M P1
  const long long n2 = c->g[1].size, n3 = c->g[2].size;
  c->nc2 = ncoef(r2);
  double2* H20 = nullptr;
  if (int st = dmalloc(&H20, c->nc2 * n2 * sizeof(double2))) return bail(st);
  if (int st = dmalloc(&c->Mk2, c->nc2 * n2 * sizeof(double))) { cudaFree(H20); return bail(st); }
  int st = assemble_level2(c->fine_cyc, c->kap64, c->g[1], c->tR1.radius, c->tP1.radius, H20, c->Mk2, &c->r2, c->s);
  if (st) { cudaFree(H20); return bail(HELM_ECUDA); }
  // level-2 operator of the cycle: H_2h + (1 - alpha2^2) R1 K P1
  if ((st = dmalloc(&c->A2_64, c->nc2 * n2 * sizeof(double2)))) { cudaFree(H20); return bail(st); }
  if ((st = apply_shift(c->nc2 * n2, H20, c->Mk2, 1.0 - o->alpha2 * o->alpha2, c->A2_64, c->s))) {
    cudaFree(H20); return bail(HELM_ECUDA);
  }
  // level 3: R2 (H_2h + (1 - alpha3^2) R1 K P1) P2 (Eq. CoarseRealShifted)
  c->nc3 = ncoef(r3);
  if ((st = dmalloc(&c->A3_64, c->nc3 * n3 * sizeof(double2)))) { cudaFree(H20); return bail(st); }
  st = assemble_level3(c->g[1], c->r2, H20, c->Mk2, 1.0 - o->alpha3 * o->alpha3, c->g[2], c->tR2.radius,
                       c->tP2.radius, c->A3_64, &c->r3, c->s);
  cudaStreamSynchronize(c->s);
  cudaFree(H20);
  if (st) return bail(HELM_ECUDA);
  if ((st = dmalloc(&c->A2_dinv64, n2 * sizeof(double2))) || (st = dmalloc(&c->A2_32, c->nc2 * n2 * sizeof(float2))) ||
      (st = dmalloc(&c->A2_dinv32, n2 * sizeof(float2))) || (st = dmalloc(&c->A3_dinv64, n3 * sizeof(double2))) ||
      (st = dmalloc(&c->d_bad, sizeof(int))))
    return bail(st);
  if (cudaMemsetAsync(c->d_bad, 0, sizeof(int), c->s) != cudaSuccess) return bail(fail(HELM_ECUDA, "memset"));
  if (finalize_stencil(n2, c->nc2, c->nc2 / 2, c->A2_64, c->A2_dinv64, c->A2_32, c->A2_dinv32, c->d_bad, c->s) ||
      finalize_stencil(n3, c->nc3, c->nc3 / 2, c->A3_64, c->A3_dinv64, nullptr, nullptr, c->d_bad, c->s))
    return bail(HELM_ECUDA);
  int bad = 0;
  if (cudaMemcpy(&bad, c->d_bad, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return bail(fail(HELM_ECUDA, "reading diagonal check"));
  if (bad) return bail(fail(HELM_ENUMERIC, "zero or non-finite coarse diagonal"));

  // coarsest factorisation
  // the coarsest operator is complex-symmetric when R and P / 2^d are transposes on both levels
  const bool symmetric = o->intergrid != HELM_INTERGRID_LEVDEP;
  // mixed precision: the coarsest factors in double-float arithmetic (FP32 pipes);
  // FP64 mode: native FP64
  const bool df = o->precision == HELM_MIXED;
  if ((st = coarse_setup(c->cs, c->g[2], c->r3, c->A3_64, 64, symmetric, df, c->s, o->coarse_blocks,
                         o->coarse_block_min > 0 ? o->coarse_block_min : kHugeFront))) return bail(st);

  // workspaces
  const int m = o->restart;
  if ((st = ensure_workspaces(c, o->max_rhs))) return bail(st);
  const int B = o->max_rhs;
  c->block = B;
  if ((st = dmalloc(&c->V, (size_t)(m + 1) * B * n1 * sizeof(double2))) ||
      (st = dmalloc(&c->Z, (size_t)m * B * n1 * esize(cycle_prec(c)))) ||
      (st = dmalloc(&c->w, (size_t)B * n1 * sizeof(double2))) || (st = dmalloc(&c->r, (size_t)B * n1 * sizeof(double2))))
    return bail(st);
  if ((st = dmalloc(&c->d_scal, sizeof(double) * KS_COUNT * B)) ||
      (st = dmalloc(&c->d_kpart, sizeof(double2) * krylov_part_entries(m))) ||
      (st = dmalloc(&c->d_kcounter, sizeof(unsigned))))
    return bail(st);
  if (cudaMemset(c->d_kcounter, 0, sizeof(unsigned)) != cudaSuccess) return bail(fail(HELM_ECUDA, "memset"));
  c->ks.resize(B);
  for (int r = 0; r < B; ++r)
    if ((st = krylov_alloc(c->ks[r], m, c->d_scal + (size_t)r * KS_COUNT, c->d_kpart, c->d_kcounter)))
      return bail(st);
  if (o->precision == HELM_MIXED) {
    if ((st = dmalloc(&c->cdf, n1 * sizeof(float4))) || (st = dmalloc(&c->xd, (size_t)B * n1 * sizeof(float4))))
      return bail(st);
    if ((st = k_coef_df(c->fine, c->kap64, c->cdf, c->s))) return bail(HELM_ECUDA);
  }
  if (cudaMallocHost(&c->h_scal, sizeof(double) * KS_COUNT * B) != cudaSuccess) return bail(fail(HELM_ENOMEM, "pinned alloc"));
  if (cudaStreamSynchronize(c->s) != cudaSuccess) return bail(fail(HELM_ECUDA, cudaGetErrorString(cudaGetLastError())));
  *out = c;
  return HELM_OK;
}

int helm_destroy(helm_ctx* c) {
  if (!c) return HELM_OK;
  if (c->s) cudaStreamSynchronize(c->s);
  else cudaDeviceSynchronize();
  drop_graphs(c);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  free_workspaces(c);
  coarse_free(c->cs);
  for (auto& k : c->ks) krylov_free(k);
  for (void* p : {(void*)c->d_gam, (void*)c->d_gam32, (void*)c->d_gam_cyc, (void*)c->d_gam32_cyc, (void*)c->kap64, (void*)c->kap32, (void*)c->A2_64, (void*)c->A2_dinv64,
                  (void*)c->A2_32, (void*)c->A2_dinv32, (void*)c->Mk2, (void*)c->A3_64, (void*)c->A3_dinv64,
                  (void*)c->V, (void*)c->w, (void*)c->r, c->Z, (void*)c->stage, (void*)c->d_bad,
                  (void*)c->cdf, (void*)c->xd, (void*)c->d_scal, (void*)c->d_kpart, (void*)c->d_kcounter})
    cudaFree(p);
  if (c->h_scal) cudaFreeHost(c->h_scal);
  delete[] c->h_gam;
  delete c;
  return HELM_OK;
}

int helm_solve(helm_ctx* c, const void* q, void* p, int n_rhs, double tol, int maxit, helm_stats* stats) {
  if (!c || !q || !p) return fail(HELM_EINVAL, "null argument");
  if (n_rhs < 1 || !(tol > 0) || maxit < 1) return fail(HELM_EINVAL, "bad n_rhs, tol or maxit");
  LaunchScope scope(c);
  const long long n = c->g[0].size;
  const bool qd = is_device_ptr(q), pd = is_device_ptr(p);
  const double2* dq = (const double2*)q;
  double2* dp = (double2*)p;
  const long long need = (long long)n_rhs * n * ((qd ? 0 : 1) + (pd ? 0 : 1));
  if (need > c->stage_cap) {
    cudaFree(c->stage);
    c->stage = nullptr;
    c->stage_cap = 0;
    if (int st = dmalloc(&c->stage, need * sizeof(double2))) return st;
    c->stage_cap = need;
  }
  double2* sp = c->stage;
  if (!qd) {
    HELM_CUDA_TRY(cudaMemcpyAsync(sp, q, n_rhs * n * sizeof(double2), cudaMemcpyHostToDevice, c->s));
    dq = sp;
    sp += n_rhs * n;
  }
  if (!pd) dp = sp;
  int worst = HELM_OK;
  std::vector<helm_stats> st_block(c->block);
  for (int r0 = 0; r0 < n_rhs; r0 += c->block) {
    const int B = std::min(c->block, n_rhs - r0);
    if (int st = solve_block(c, dq + (size_t)r0 * n, dp + (size_t)r0 * n, B, tol, maxit, st_block.data())) return st;
    for (int r = 0; r < B; ++r) {
      if (stats) stats[r0 + r] = st_block[r];
      if (!st_block[r].converged) worst = HELM_NOT_CONVERGED;
    }
  }
  if (!pd) {
    HELM_CUDA_TRY(cudaMemcpyAsync(p, dp, n_rhs * n * sizeof(double2), cudaMemcpyDeviceToHost, c->s));
  }
  HELM_CUDA_TRY(cudaStreamSynchronize(c->s));
  if (worst != HELM_OK) set_error("not converged within maxit");
  return worst;
}

int helm_adjoint_grad(helm_ctx* c, const void* p, const void* resid, int n_rhs, double tol, int maxit,
                      double* grad, void* adj, helm_stats* stats) {
  if (!c || !p || !resid || !grad) return fail(HELM_EINVAL, "null argument");
  if (n_rhs < 1 || !(tol > 0) || maxit < 1) return fail(HELM_EINVAL, "bad n_rhs, tol or maxit");
  if (!is_device_ptr(p) || !is_device_ptr(resid) || !is_device_ptr(grad) || (adj && !is_device_ptr(adj)))
    return fail(HELM_EINVAL, "helm_adjoint_grad takes device pointers");
  LaunchScope scope(c);
  const long long n = c->g[0].size;
  // a block of conj(residual) right-hand sides and their adjoint fields at a time
  const long long need = 2LL * c->block * n;
  if (need > c->stage_cap) {
    cudaFree(c->stage);
    c->stage = nullptr;
    c->stage_cap = 0;
    if (int st = dmalloc(&c->stage, need * sizeof(double2))) return st;
    c->stage_cap = need;
  }
  double2* rhs = c->stage;
  double2* mu = c->stage + (size_t)c->block * n;
  int worst = HELM_OK;
  std::vector<helm_stats> st_block(c->block);
  for (int r0 = 0; r0 < n_rhs; r0 += c->block) {
    const int B = std::min(c->block, n_rhs - r0);
    if (int st = launch_conj((long long)B * n, (const double2*)resid + (size_t)r0 * n, rhs, c->s)) return st;
    double2* m_out = adj ? (double2*)adj + (size_t)r0 * n : mu;
    if (int st = solve_block(c, rhs, m_out, B, tol, maxit, st_block.data())) return st;
    for (int r = 0; r < B; ++r) {
      if (stats) stats[r0 + r] = st_block[r];
      if (!st_block[r].converged) worst = HELM_NOT_CONVERGED;
      // right-hand sides in order: the gradient sums over them deterministically
      if (int st = launch_gradient(c->fine, (const double2*)p + (size_t)(r0 + r) * n, m_out + (size_t)r * n, grad, c->s))
        return st;
    }
  }
  HELM_CUDA_TRY(cudaStreamSynchronize(c->s));
  if (worst != HELM_OK) set_error("adjoint solve not converged within maxit");
  return worst;
}

int helm_apply(helm_ctx* c, int level, int dtype, const void* x, void* y, int n_rhs) {
  if (!c || !x || !y || n_rhs < 1) return fail(HELM_EINVAL, "bad argument");
  if (int st = check_level(c, level, 1, 3)) return st;
  LaunchScope scope(c);
  const Prec P = dtype_prec(dtype);
  if (int st = row_op(c, level - 1, P, MODE_APPLY, P, P, P, x, x, y, n_rhs, 0.0, 0)) return st;
  return HELM_OK;
}

int helm_residual(helm_ctx* c, int level, int dtype, const void* b, const void* x, void* r, int n_rhs) {
  if (!c || !b || !x || !r || n_rhs < 1) return fail(HELM_EINVAL, "bad argument");
  if (int st = check_level(c, level, 1, 3)) return st;
  LaunchScope scope(c);
  const Prec P = dtype_prec(dtype);
  if (int st = row_op(c, level - 1, P, MODE_RESID, P, P, P, x, b, r, n_rhs, 0.0, 0)) return st;
  return HELM_OK;
}

int helm_smooth(helm_ctx* c, int level, int dtype, const void* b, void* x, int n_rhs) {
  if (!c || !b || !x || n_rhs < 1) return fail(HELM_EINVAL, "bad argument");
  if (int st = check_level(c, level, 1, 2)) return st;
  LaunchScope scope(c);
  if (int st = ensure_workspaces(c, n_rhs)) return st;
  const Prec P = dtype_prec(dtype);
  void* tmp = level == 1 ? c->l1r : c->l2r;
  void* xx = x;
  void* tt = tmp;
  if (int st = smooth(c, level - 1, P, b, P, &xx, &tt, 1, false, n_rhs)) return st;
  if (xx != x)
    HELM_CUDA_TRY(cudaMemcpyAsync(x, xx, c->g[level - 1].size * n_rhs * esize(P), cudaMemcpyDeviceToDevice, c->s));
  return HELM_OK;
}

int helm_restrict(helm_ctx* c, int level, int dtype, const void* rf, void* rc, int n_rhs) {
  if (!c || !rf || !rc || n_rhs < 1) return fail(HELM_EINVAL, "bad argument");
  if (int st = check_level(c, level, 1, 2)) return st;
  LaunchScope scope(c);
  const Transfer& t = level == 1 ? c->tR1 : c->tR2;
  if (int st = launch_restrict(c->g[level - 1], c->g[level], t, dtype_prec(dtype), rf, rc, n_rhs, c->s)) return st;
  return HELM_OK;
}

int helm_prolong_add(helm_ctx* c, int level, int dtype, const void* ec, void* xf, int n_rhs) {
  if (!c || !ec || !xf || n_rhs < 1) return fail(HELM_EINVAL, "bad argument");
  if (int st = check_level(c, level, 1, 2)) return st;
  LaunchScope scope(c);
  const Transfer& t = level == 1 ? c->tP1 : c->tP2;
  if (int st = launch_prolong_add(c->g[level - 1], c->g[level], t, dtype_prec(dtype), ec, xf, n_rhs, c->s))
    return st;
  return HELM_OK;
}

int helm_get_stencil(helm_ctx* c, int level, double* out, int* radius) {
  if (!c) return fail(HELM_EINVAL, "null context");
  if (int st = check_level(c, level, 2, 3)) return st;
  if (radius) *radius = level == 2 ? c->r2 : c->r3;
  if (!out) return HELM_OK;
  const long long n = c->g[level - 1].size * (level == 2 ? c->nc2 : c->nc3);
  HELM_CUDA_TRY(cudaStreamSynchronize(c->s));
  HELM_CUDA_TRY(cudaMemcpy(out, level == 2 ? c->A2_64 : c->A3_64, n * sizeof(double2), cudaMemcpyDeviceToHost));
  return HELM_OK;
}

int helm_coarse_solve(helm_ctx* c, const void* b, void* e, int n_rhs) {
  if (!c || !b || !e || n_rhs < 1) return fail(HELM_EINVAL, "bad argument");
  LaunchScope scope(c);
  if (c->o.coarse_refine > 0)
    if (int st = ensure_workspaces(c, n_rhs)) return st;
  if (int st = coarse_apply(c, (const double2*)b, (double2*)e, n_rhs)) return st;
  if (int st = coarse_status(c->cs, c->s)) return st;
  return HELM_OK;
}

int helm_coarse_solve_noalloc(helm_ctx* c, const void* b, void* e, int n_rhs) {
  if (!c || !b || !e || n_rhs < 1) return fail(HELM_EINVAL, "bad argument");
  LaunchScope scope(c);
  if (int st = coarse_solve_noalloc(c->cs, (const double2*)b, (double2*)e, n_rhs, c->s)) return st;
  if (int st = coarse_status(c->cs, c->s)) return st;
  return HELM_OK;
}

int helm_coarse_wait_check(helm_ctx* c, long long wait_cycles, int job) {
  if (!c) return fail(HELM_EINVAL, "null context");
  return coarse_plant_unreachable_wait(c->cs, wait_cycles, job, c->s);
}

int helm_cycle(helm_ctx* c, const void* v, void* z, int n_rhs) {
  if (!c || !v || !z || n_rhs < 1) return fail(HELM_EINVAL, "bad argument");
  LaunchScope scope(c);
  if (fused_cycle(c, P_DF, P32)) {
    // the fused mixed-precision cycle reads the double-float form of v and writes c64
    if (int st = ensure_workspaces(c, n_rhs)) return st;
    const long long n = c->g[0].size * n_rhs;
    if (int st = launch_convert(P64, P_DF, v, c->l1r, n, c->s)) return st;
    if (int st = run_cycle(c, c->l1r, P_DF, c->l1a, P32, n_rhs)) return st;
    if (int st = launch_convert(P32, P64, c->l1a, z, n, c->s)) return st;
  } else if (int st = run_cycle(c, v, P64, z, P64, n_rhs)) {
    return st;
  }
  if (int st = coarse_status(c->cs, c->s)) return st;
  return HELM_OK;
}

int helm_coarse_plan(int dim, const int n_nodes[3], int radius, int leaf_max, int symmetric, int grid,
                     long long stats[8]) {
  if (!n_nodes || !stats) return fail(HELM_EINVAL, "null argument");
  if ((dim != 2 && dim != 3) || radius < 1 || radius > 3 || leaf_max < 1 || grid < 1)
    return fail(HELM_EINVAL, "bad dim, radius, leaf_max or grid");
  GridDims g{};
  g.dim = dim;
  long long size = 1;
  for (int d = 0; d < 3; ++d) {
    g.N[d] = d < dim ? n_nodes[d] : 1;
    if (g.N[d] < 1) return fail(HELM_EINVAL, "bad node count");
    size *= g.N[d];
  }
  if (size >= (1LL << 31)) return fail(HELM_EINVAL, "grid too large");
  g.size = size;
  finish_dims(g);
  if (int st = coarse_plan_stats(g, radius, leaf_max, symmetric != 0, grid, stats)) return st;
  return HELM_OK;
}

long long helm_launch_count(const helm_ctx* c) { return c ? c->launches : 0; }

int helm_set_block(helm_ctx* c, int block) {
  if (!c) return fail(HELM_EINVAL, "null context");
  if (block < 1 || block > (int)c->ks.size()) return fail(HELM_EINVAL, "block must be in [1, max_rhs]");
  c->block = block;
  return HELM_OK;
}

int helm_autotune_block(helm_ctx* c, const void* q, int n_rhs, int probe_iters, int* best, double* ms_per_rhs_iter) {
  if (!c || !q || !best) return fail(HELM_EINVAL, "null argument");
  if (n_rhs < 1) return fail(HELM_EINVAL, "n_rhs must be >= 1");
  if (!is_device_ptr(q)) return fail(HELM_EINVAL, "helm_autotune_block takes a device pointer");
  LaunchScope scope(c);
  const int iters = probe_iters > 0 ? probe_iters : c->o.restart;
  const int cap = std::min((int)c->ks.size(), n_rhs);
  const long long n = c->g[0].size;
  if ((long long)cap * n > c->stage_cap) {
    cudaFree(c->stage);
    c->stage = nullptr;
    c->stage_cap = 0;
    if (int st = dmalloc(&c->stage, (long long)cap * n * sizeof(double2))) return st;
    c->stage_cap = (long long)cap * n;
  }
  std::vector<int> cands;
  for (int b = 1; b < cap; b *= 2) cands.push_back(b);
  cands.push_back(cap);
  cudaEvent_t e0, e1;
  HELM_CUDA_TRY(cudaEventCreate(&e0));
  HELM_CUDA_TRY(cudaEventCreate(&e1));
  std::vector<helm_stats> st(cap);
  double best_cost = 0.0;
  int best_b = 1;
  int status = HELM_OK;
  const int saved = c->block;
  for (size_t i = 0; i < cands.size(); ++i) {
    const int b = cands[i];
    c->block = b;
    // a first run allocates what a block of this size needs; the second is timed.  A
    // tolerance of zero keeps every right-hand side iterating for exactly `iters` steps.
    for (int rep = 0; rep < 2 && status == HELM_OK; ++rep) {
      if (rep == 1) cudaEventRecord(e0, c->s);
      status = solve_block(c, (const double2*)q, c->stage, b, 0.0, iters, st.data());
      if (rep == 1) cudaEventRecord(e1, c->s);
    }
    if (status != HELM_OK) break;
    float ms = 0.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      status = fail(HELM_ECUDA, "autotune timing failed");
      break;
    }
    const double cost = ms / ((double)b * iters);
    if (ms_per_rhs_iter && i < 7) ms_per_rhs_iter[i] = cost;
    if (i == 0 || cost < best_cost) {
      best_cost = cost;
      best_b = b;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (status != HELM_OK) {
    c->block = saved;
    return status;
  }
  c->block = best_b;
  *best = best_b;
  return HELM_OK;
}

int helm_set_cycle_kernels(helm_ctx* c, int kind) {
  if (!c) return fail(HELM_EINVAL, "null context");
  if (kind < HELM_FINE_TILES || kind > HELM_FINE_ROWS32) return fail(HELM_EINVAL, "unknown fine-pass kernel kind");
  c->fine_kind = kind;
  return HELM_OK;
}

int helm_autotune_cycle(helm_ctx* c, int n_rhs, int* best, double* ms) {
  if (!c || !best) return fail(HELM_EINVAL, "null argument");
  if (n_rhs < 1) return fail(HELM_EINVAL, "n_rhs must be >= 1");
  if (!fused_cycle(c, P_DF, P32)) return fail(HELM_EINVAL, "the context's cycle has no fused fine passes");
  LaunchScope scope(c);
  if (int st = ensure_workspaces(c, n_rhs)) return st;
  const long long n1 = c->g[0].size * n_rhs, n2 = c->g[1].size * n_rhs;
  // inputs: v = 0 (double-float) and y2 = 0; the passes' cost does not depend on the values
  HELM_CUDA_TRY(cudaMemsetAsync(c->l1r, 0, n1 * sizeof(float4), c->s));
  HELM_CUDA_TRY(cudaMemsetAsync(c->l2a, 0, n2 * sizeof(float2), c->s));
  Cycle2D cy = make_cycle2d(c);
  cudaEvent_t e0, e1;
  HELM_CUDA_TRY(cudaEventCreate(&e0));
  HELM_CUDA_TRY(cudaEventCreate(&e1));
  const float4* v = static_cast<const float4*>(c->l1r);
  int status = HELM_OK;
  double best_ms = 0.0;
  int best_k = c->fine_kind;
  for (int k = HELM_FINE_TILES; k <= HELM_FINE_ROWS32 && status == HELM_OK; ++k) {
    cy.fine_kind = k;
    constexpr int kReps = 5;
    for (int rep = -1; rep < kReps && status == HELM_OK; ++rep) {   // one untimed pass first
      if (rep == 0) cudaEventRecord(e0, c->s);
      status = cycle2d_fine_down(cy, v, static_cast<float2*>(c->l2b), n_rhs, c->s);
      if (status == HELM_OK)
        status = cycle2d_fine_up(cy, v, static_cast<const float2*>(c->l2a), static_cast<float2*>(c->l1a), n_rhs, c->s);
    }
    if (status != HELM_OK) break;
    cudaEventRecord(e1, c->s);
    float t = 0.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) {
      status = fail(HELM_ECUDA, "autotune timing failed");
      break;
    }
    const double per = t / kReps;
    if (ms) ms[k] = per;
    if (k == HELM_FINE_TILES || per < best_ms) {
      best_ms = per;
      best_k = k;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (status != HELM_OK) return status;
  c->fine_kind = best_k;
  *best = best_k;
  return HELM_OK;
}

int helm_info(const helm_ctx* c, int key, long long* value) {
  if (!c || !value) return fail(HELM_EINVAL, "null argument");
  switch (key) {
    case HELM_INFO_NODES1: *value = c->g[0].size; break;
    case HELM_INFO_NODES2: *value = c->g[1].size; break;
    case HELM_INFO_NODES3: *value = c->g[2].size; break;
    case HELM_INFO_RADIUS2: *value = c->r2; break;
    case HELM_INFO_RADIUS3: *value = c->r3; break;
    case HELM_INFO_COARSE_ENTRIES: *value = c->cs.factor_entries; break;
    case HELM_INFO_COARSE_FRONTS: *value = c->cs.nfronts; break;
    case HELM_INFO_COARSE_LEVELS: *value = c->cs.nlevels; break;
    case HELM_INFO_COARSE_BWD_ENTRIES: *value = c->cs.bwd_entries; break;
    case HELM_INFO_DOUBLE_FLOAT: *value = c->cs.df ? 1 : 0; break;
    case HELM_INFO_GRAPHS: *value = c->graphs_broken ? -1 : (long long)c->graphs.size(); break;
    case HELM_INFO_CYCLE_KERNELS: *value = c->fine_kind; break;
    default: return fail(HELM_EINVAL, "unknown info key");
  }
  return HELM_OK;
}

int helm_timer_enable(helm_ctx* c, unsigned mask) {
  if (!c) return fail(HELM_EINVAL, "null context");
  c->timer.reset();
  c->timer.mask = mask;
  return HELM_OK;
}

int helm_timer_read(helm_ctx* c, int cls, double* total_ms, long long* launches) {
  if (!c || cls < 0 || cls >= HELM_K_COUNT) return fail(HELM_EINVAL, "bad timer class");
  c->timer.resolve();
  if (total_ms) *total_ms = c->timer.total_ms[cls];
  if (launches) *launches = c->timer.count[cls];
  return HELM_OK;
}

const char* helm_strerror(int status) {
  switch (status) {
    case HELM_OK: return "ok";
    case HELM_EINVAL: return "invalid argument";
    case HELM_ENOMEM: return "out of device memory";
    case HELM_NOT_CONVERGED: return "not converged";
    case HELM_ECUDA: return "CUDA error";
    case HELM_ENUMERIC: return "numerical breakdown";
    default: return "unknown status";
  }
}

const char* helm_last_error(void) { return t_last_error.c_str(); }

}  // extern "C"
