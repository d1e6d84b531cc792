// Solve phase of the coarsest-level direct solver (Sec. 2: exact coarse solve) as one
// persistent kernel per right-hand-side block.
//
// Forward, leaves to root, every front turns its assembled right-hand side r_F into
// w_S = F_SS^-1 r_S and the update vector r_B - F_BS F_SS^-1 r_S passed to its parent
// (column sums over the rows of M).  Backward, root to leaves,
// x_S = w_S - (F_SS^-1 F_SB) x_B (column sums over the rows of G^T).
//
// Scheduling.  The job list holds every forward job (by tree height, leaves first) and
// then every backward job (root first); block g of the G resident blocks takes jobs g,
// g + G, g + 2G, ...  A forward job waits for its front's children to complete, a
// backward job for its parent (the root: for its own forward); every such dependency has
// a smaller job index, so with all blocks resident (cooperative launch) the job with the
// smallest unfinished index can always run and the schedule cannot deadlock.  Waits are
// bounded in time: a block that gives up records an error and skips its remaining work.
//
// Data movement.  Factor rows are constant during the solve, so a producer warp in every
// block keeps a ring of shared-memory stages filled ahead of the computation with bulk
// asynchronous copies (cp.async.bulk, completion counted on an mbarrier per stage), across
// job boundaries and while the consumer warps wait for dependencies; the consumers release
// each stage per warp on a second mbarrier.  The right-hand sides and
// children's update vectors, written by other blocks in the same launch, are read through
// L2 after an acquire on the completion counter.
//
// Reproducibility.  Every sum is taken in an order fixed by the job list: a job's rows
// split into a fixed number of interleaved parts per column, combined in part order, and
// job partial sums in chunk order.  None of it depends on the number of right-hand sides
// solved together, nor on how many resident blocks run the list (a context may run it on
// a share of the device, helm_opts.coarse_blocks).
#include <cstddef>
#include <type_traits>
#include "coarse.cuh"
#include "df64.cuh"

namespace helm {

namespace {

constexpr int kSplitMax = 16;                              // forward row parts per column
// Limit on a wait for a factor copy, in cycles of the waiting multiprocessor's clock
// (clock64 is monotonic per multiprocessor): about 2 s at the maximum SM clock, longer
// below it.  Dependency waits take their limit from the launch (CoarseSolver::wait_cycles,
// the same by default).
constexpr long long kWaitCycles = kDefaultWaitCycles;
constexpr int kStageBytes = kStageEntries * 16;
// Resident blocks per multiprocessor the kernel is shaped for: enough jobs in flight that
// one job's fixed latencies (dependency wait, gathers, write-back) overlap the others'
// streaming.  Single right-hand sides run four blocks, groups (with four times the
// per-job scratch) three; the rings keep 192 KiB or 144 KiB of factor rows in flight
// per multiprocessor.
template <int RG>
__host__ __device__ constexpr int blocks_per_sm_target() { return RG == 1 ? 4 : 3; }
template <int RG>
__host__ __device__ constexpr int ring_stages() { return 3; }
// per-job scratch: row values [kJobRows][RG] (reused for the row-part sums
// [kSweepThreads][RG] once the job's stages are consumed) and forward r_B [kTile][RG]
template <int RG>
__host__ __device__ constexpr int local_bytes() {
  return ((kJobRows > kSweepThreads ? kJobRows : kSweepThreads) + kTile) * RG * 16;
}
// after the local scratch: two job records, the ring's mbarriers, two flags and the
// output columns' nodes of the current and the next job
template <int RG>
__host__ __device__ constexpr int tail_bytes() {
  return 2 * (int)sizeof(SweepMeta) + 2 * ring_stages<RG>() * 8 + 16 + 2 * kTile * 4;
}
template <int RG>
__host__ __device__ constexpr int smem_bytes() {
  return ring_stages<RG>() * kStageBytes + local_bytes<RG>() + (tail_bytes<RG>() + 127) / 128 * 128;
}
static_assert(offsetof(SweepMeta, ld) == 21 * 4 && offsetof(SweepMeta, src) == 22 * 4, "record words read by the producer");
static_assert((smem_bytes<1>() + 1024) * blocks_per_sm_target<1>() <= 233472 &&
                  (smem_bytes<kRhsGroup>() + 1024) * blocks_per_sm_target<kRhsGroup>() <= 233472,
              "the targeted blocks per multiprocessor fit in shared memory");
static_assert(kTile <= kPartBlock, "partial block");
static_assert(kTile <= kSweepThreads, "one thread per output column at least");
static_assert(kSweepThreads >= 64, "thread 32 (warp 1) publishes completions");

struct SweepArgs {
  const SweepMeta* meta;
  int njobs;
  const int* S;
  const int* B;
  const int2* ctb;
  const double2* factors;
  const double2* b;
  double2* uv;
  double2* w;
  double2* x;
  float4* xd;
  double2* part;
  unsigned* counters;   // forward completions, backward completions, chunk slots
  int* err;
  int nrhs;
  long long nodes;
  long long uv_total;
  long long wait_cycles;   // limit on a dependency wait (SM clock cycles)
};

// ---- element operations on 16-byte complex values: double2 (FP64) or float4 (double-float)
__device__ __forceinline__ void mac(double2& acc, double2 m, double2 r) { acc = cmac(acc, m, r); }
__device__ __forceinline__ void mac(float4& acc, float4 m, float4 r) { df_cmac(acc, m, r); }
__device__ __forceinline__ void addto(double2& a, double2 b) {
  a.x += b.x;
  a.y += b.y;
}
__device__ __forceinline__ void addto(float4& a, float4 b) { df_acc_add(a, b); }
__device__ __forceinline__ void zero(double2& a) { a = make_double2(0.0, 0.0); }
__device__ __forceinline__ void zero(float4& a) { a = make_float4(0.f, 0.f, 0.f, 0.f); }
// Double-float values and accumulators share the float4 layout (re_hi, im_hi, re_lo,
// im_lo); the solve's scratch vectors (update vectors, w) hold double-float values in the
// 16-byte slots of the FP64 layout.  Conversions from and to c128 use bit operations
// (f2d, split_d): GB300 runs FP64 conversions and additions at the FP64 rate.
__device__ __forceinline__ void from_c128(double2& a, double2 v) { a = v; }
__device__ __forceinline__ void from_c128(float4& a, double2 v) {
  const dd re = split_d(v.x), im = split_d(v.y);
  a = make_float4(re.hi, im.hi, re.lo, im.lo);
}
__device__ __forceinline__ double2 to_c128(double2 a) { return a; }
__device__ __forceinline__ double2 to_c128(float4 a) { return make_double2(f2d(a.x) + f2d(a.z), f2d(a.y) + f2d(a.w)); }
__device__ __forceinline__ double2 norm(double2 a) { return a; }
__device__ __forceinline__ float4 norm(float4 a) {
  const dd re = dd_norm(a.x, a.z), im = dd_norm(a.y, a.w);
  return make_float4(re.hi, im.hi, re.lo, im.lo);
}
__device__ __forceinline__ double2 neg(double2 a) { return make_double2(-a.x, -a.y); }
__device__ __forceinline__ float4 neg(float4 a) { return make_float4(-a.x, -a.y, -a.z, -a.w); }
__device__ __forceinline__ double2 ldcg(const double2* p) { return __ldcg(p); }
__device__ __forceinline__ float4 ldcg(const float4* p) { return __ldcg(p); }

// ---- synchronisation primitives
__device__ __forceinline__ bool expired(long long t0, long long limit = kWaitCycles) { return clock64() - t0 > limit; }
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_relaxed(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Completion counts.  A block publishes its writes by a barrier over its consumer threads
// followed by one release increment; a waiter's acquire load followed by the same barrier
// makes them visible to all its consumer threads.
__device__ __forceinline__ void red_release(unsigned* p) {
  asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(p) : "memory");
}
__device__ __forceinline__ unsigned atom_add_acq_rel(unsigned* p) {
  unsigned old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(old) : "l"(p) : "memory");
  return old;
}

// *p >= target within `limit` cycles; false on a timeout (recorded) or when another
// block has already recorded an error.
__device__ bool wait_count(const unsigned* p, unsigned target, int* err, long long limit) {
  if (ld_acquire(p) >= target) return true;
  const long long t0 = clock64();
  while (true) {
    __nanosleep(64);
    if (ld_acquire(p) >= target) return true;
    if (ld_relaxed(err)) return false;
    if (expired(t0, limit)) {
      atomicCAS(err, 0, kErrSweepWait);
      return false;
    }
  }
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// The stage's copies have landed within the time limit.
__device__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  if (mbar_try(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try(bar, parity))
    if (expired(t0)) return false;
  return true;
}
__device__ __forceinline__ void bulk_copy(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

// ---- the block's sequence of stage fills: its jobs with factor rows, every pass over
// the right-hand-side groups, every stage of the job.  The cursor keeps the current job's
// copy source so that a fill reads no job data from memory.
__device__ __forceinline__ int job_stages(int rows, int srows) { return srows ? (rows + srows - 1) / srows : 0; }
struct Cursor {
  int j, pass, k, nst;
  int rows, cols, srows;
  long long ld;
  const double2* src;   // factor row r0 of the job, column c0
};
// The producer warp's next job with factor rows: lane l reads word l of the record.
__device__ void cursor_load(Cursor& c, const SweepArgs& a, int lane) {
  for (; c.j < a.njobs; c.j += gridDim.x) {
    const int w = reinterpret_cast<const int*>(a.meta + c.j)[lane];
    auto f = [&](int i) { return __shfl_sync(0xffffffffu, w, i); };
    const int r0 = f(1), r1 = f(2), c0 = f(3), c1 = f(4), srows = f(5);
    c.nst = job_stages(r1 - r0, srows);
    if (!c.nst) continue;
    c.rows = r1 - r0;
    c.cols = c1 - c0;
    c.srows = srows;
    c.ld = f(21);
    const long long src = (long long)(unsigned)f(22) | ((long long)f(23) << 32);
    c.src = a.factors + src;
    return;
  }
}
__device__ void cursor_next(Cursor& c, const SweepArgs& a, int npass, int lane) {
  if (++c.k < c.nst) return;
  c.k = 0;
  if (++c.pass < npass) return;
  c.pass = 0;
  c.j += gridDim.x;
  cursor_load(c, a, lane);
}
// Warp 0: copy the factor rows of the cursor's stage into shared memory at dst.
__device__ void issue_stage(const Cursor& c, uint32_t dst, uint32_t bar, int lane) {
  const int s0 = c.k * c.srows, n = min(c.srows, c.rows - s0);
  const double2* src = c.src + (long long)s0 * c.ld;
  const uint32_t row_bytes = (uint32_t)c.cols * 16u;
  if (lane == 0) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect(bar, row_bytes * (uint32_t)n);
  }
  __syncwarp();
  if (c.ld == c.cols) {
    if (lane == 0) bulk_copy(dst, src, row_bytes * (uint32_t)n, bar);
  } else {
    for (int q = lane; q < n; q += 32) bulk_copy(dst + (uint32_t)q * row_bytes, src + (long long)q * c.ld, row_bytes, bar);
  }
}

constexpr int kBlockThreads = kSweepThreads + 32;   // consumers + one producer warp

__device__ __forceinline__ void consumer_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kSweepThreads) : "memory"); }
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Block layout: the first kSweepThreads / 32 warps consume (compute), the last warp
// produces (copies factor rows into the ring).  Stage i of the block's fill sequence uses slot i mod NST; full[slot] completes
// when its copies land, empty[slot] when all consumer warps are done with it.
template <bool DF, int RG>
__global__ void __launch_bounds__(kBlockThreads, blocks_per_sm_target<RG>()) sweep_kernel(const SweepArgs a) {
  using E = typename std::conditional<DF, float4, double2>::type;
  // gather items a consumer thread handles per pass: the job's rows x group, its columns x group
  constexpr int kRowItems = (kJobRows * RG + kSweepThreads - 1) / kSweepThreads;
  constexpr int kColItems = (kTile * RG + kSweepThreads - 1) / kSweepThreads;
  constexpr int NST = ring_stages<RG>();
  constexpr int kLocalBytes = local_bytes<RG>();
  constexpr int kMetaWarp = kSweepThreads / 32 - 1;   // the consumer warp that reads job records
  extern __shared__ __align__(128) unsigned char smem[];
  E* const stage = reinterpret_cast<E*>(smem);
  unsigned char* const local = smem + NST * kStageBytes;
  E* const vs = reinterpret_cast<E*>(local);   // row values [kJobRows][RG]
  E* const red = vs;                           // row-part sums [threads][RG], after the stages
  E* const rbs = vs + (kJobRows > kSweepThreads ? kJobRows : kSweepThreads) * RG;   // forward r_B [kTile][RG]
  E* const uvE = reinterpret_cast<E*>(a.uv);   // update vectors and w in the arithmetic's form
  E* const wE = reinterpret_cast<E*>(a.w);
  SweepMeta* const metas = reinterpret_cast<SweepMeta*>(local + kLocalBytes);   // [2]: current and next job
  uint64_t* const full = reinterpret_cast<uint64_t*>(metas + 2);
  uint64_t* const empty = full + NST;
  volatile int* const flag = reinterpret_cast<volatile int*>(empty + NST);
  volatile int* const abort_copy = flag + 1;
  int* const sidx2 = const_cast<int*>(flag) + 4;   // node of each output column [2][kTile]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int npass = (a.nrhs + RG - 1) / RG;

  if (tid == 0) {
    for (int q = 0; q < NST; ++q) {
      mbar_init(smem_u32(&full[q]), 1);
      mbar_init(smem_u32(&empty[q]), kSweepThreads / 32);
    }
    *abort_copy = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == kMetaWarp && (int)blockIdx.x < a.njobs)
    reinterpret_cast<int*>(metas)[lane] = reinterpret_cast<const int*>(a.meta + blockIdx.x)[lane];
  __syncthreads();

  if (warp == kSweepThreads / 32) {
    // ---- producer: walk the block's fill sequence, one slot ahead of the consumers' release
    Cursor pc;
    pc.j = blockIdx.x;
    pc.pass = pc.k = 0;
    cursor_load(pc, a, lane);
    long long i = 0;
    for (; pc.j < a.njobs; ++i) {
      const int q = (int)(i % NST);
      if (i >= NST && !mbar_wait(smem_u32(&empty[q]), (uint32_t)(((i / NST) & 1) ^ 1))) {
        if (lane == 0) atomicCAS(a.err, 0, kErrSweepCopy);
        *abort_copy = 1;
        break;
      }
      if (*abort_copy) break;
      issue_stage(pc, smem_u32(stage + q * kStageEntries), smem_u32(&full[q]), lane);
      cursor_next(pc, a, npass, lane);
    }
    // copies still in flight must land before the block may exit (bounded)
    for (long long q = i > NST ? i - NST : 0; q < i; ++q)
      if (!mbar_wait(smem_u32(&full[q % NST]), (uint32_t)((q / NST) & 1))) break;
    return;
  }

  // ---- consumers
  long long ci = 0;   // position in the fill sequence
  bool ok = true;     // uniform over the consumers: false once a dependency failed anywhere
  // backward output: x = w - (G x_B) at node gi, as c128 and (double-float) its copy xd
  auto write_x = [&](long long gi, E w, E o) {
    addto(w, neg(o));
    w = norm(w);
    a.x[gi] = to_c128(w);
    if constexpr (DF) a.xd[gi] = w;
  };
  auto consume = [&](auto&& body) {
    const int q = (int)(ci % NST);
    const uint32_t par = (uint32_t)((ci / NST) & 1);
    ++ci;
    if (*abort_copy) return;
    if (!mbar_wait(smem_u32(&full[q]), par)) {
      atomicCAS(a.err, 0, kErrSweepCopy);
      *abort_copy = 1;
      return;
    }
    if (ok) body(stage + q * kStageEntries);
    __syncwarp();
    if (lane == 0) mbar_arrive(smem_u32(&empty[q]));
  };

  // Gathers of one pass in three steps: indices (node and child-map entries, known
  // before the job runs), the right-hand side b at the row nodes (forward; also known
  // before), and what other blocks of this launch write (children's update vectors; the
  // ancestors' x_B and this front's w), read once the job's dependencies have completed.
  // The first two steps of a job's first pass run while the block finishes its previous
  // job.
  int sI[kColItems];            // node of output column item
  // Single right-hand sides stage the row gathers in registers across the dependency
  // wait; groups (kRowItems times more items) gather straight into shared memory after
  // it, which keeps their registers for the accumulators.
  constexpr bool kPre = RG == 1;
  constexpr int kPreItems = kPre ? kRowItems : 1;
  int pI[kPreItems];            // forward: node of row item; backward: node of boundary row item
  int2 pc2[kPreItems], qc2[kColItems];
  double2 pv[kPreItems];
  auto gather_idx = [&](const SweepMeta& m, int r0, int nr) {
    const bool fw = m.kind == 0;
    const int rows = m.r1 - m.r0, cols = m.c1 - m.c0;
    // loads go straight into pre-set registers (no select on a loaded value, which would
    // wait for the load here instead of where the value is used)
#pragma unroll
    for (int i = 0; i < kColItems; ++i) {
      const int q = tid + i * kSweepThreads;
      sI[i] = -1;
      if (q < cols && (!fw || m.c0 + q < m.nS)) sI[i] = a.S[m.S_off + m.c0 + q];
    }
    if constexpr (kPre) {
#pragma unroll
      for (int i = 0; i < kRowItems; ++i) {
        const int q = tid + i * kSweepThreads;
        if (q < rows * nr) {
          const int t = m.r0 + q / nr;
          if (fw) {
            pI[i] = a.S[m.S_off + t];
            pc2[i] = a.ctb[m.ctb_off + t];
          } else {
            pI[i] = a.B[m.B_off + t];
          }
        }
      }
    }
    if (fw)
#pragma unroll
      for (int i = 0; i < kColItems; ++i) {
        const int q = tid + i * kSweepThreads;
        qc2[i] = make_int2(-1, -1);
        if (q < cols * nr && m.c0 + q / nr >= m.nS) qc2[i] = a.ctb[m.ctb_off + m.c0 + q / nr];
      }
  };
  auto gather_b = [&](const SweepMeta& m, int r0, int nr) {
    if (!kPre || m.kind != 0) return;
    const int rows = m.r1 - m.r0;
#pragma unroll
    for (int i = 0; i < kRowItems; ++i) {
      const int q = tid + i * kSweepThreads;
      if (q < rows * nr) pv[i] = a.b[(r0 + q % nr) * a.nodes + pI[i]];
    }
  };

  bool pre_done = false;   // the current job's first-pass indices and b are already in registers
  int cur = 0;
  // job records travel two jobs ahead: word (lane l) of the next job's record is in a
  // register of the record warp when the current job starts, the one after it is loaded then
  int next_word = 0;
  if (warp == kMetaWarp && (int)(blockIdx.x + gridDim.x) < a.njobs)
    next_word = reinterpret_cast<const int*>(a.meta + blockIdx.x + gridDim.x)[lane];
  for (int j = blockIdx.x; j < a.njobs; j += gridDim.x, cur ^= 1) {
    const SweepMeta& m = metas[cur];
    int* const sidx = sidx2 + cur * kTile;
    const bool fwd = m.kind == 0;
    const int r0j = m.r0, c0j = m.c0, nS = m.nS;
    const int rows = m.r1 - r0j, cols = m.c1 - c0j;
    const int nst = job_stages(rows, m.srows);
    const int nchunks = m.nchunks;
    const int jn = j + gridDim.x;
    const int jnn = jn + gridDim.x;
    int next2_word = 0;
    if (warp == kMetaWarp && jnn < a.njobs) next2_word = reinterpret_cast<const int*>(a.meta + jnn)[lane];

    if (!pre_done) {
      gather_idx(m, 0, min(RG, a.nrhs));
      gather_b(m, 0, min(RG, a.nrhs));
    }
#pragma unroll
    for (int i = 0; i < kColItems; ++i)
      if (tid + i * kSweepThreads < cols) sidx[tid + i * kSweepThreads] = sI[i];
    // dependencies: acquire loads of the completion counters (tid 0), then the barrier
    if (tid == 0) {
      bool good = ok;
      if (good && m.nwait > 0) {
        good = !ld_relaxed(a.err);
        for (int q = 0; q < m.nwait && good; ++q)
          good = wait_count(a.counters + m.wait[q], (unsigned)m.target[q], a.err, a.wait_cycles);
      }
      *flag = good;
    }
    consumer_sync();
    ok = ok && *flag;
    consumer_sync();

    // out_c = sum over the job's rows q of A[q][c] v[q]: nsplit interleaved row parts per
    // column, added in part order
    const int nsplit = min(kSplitMax, kSweepThreads / cols);
    const int c = tid % cols, part = tid / cols;
    const bool act = part < nsplit;
    // one row part per column: every active thread ends with its column's whole sum, and the
    // reduction through shared memory (and its two barriers) is skipped
    const bool direct = nsplit == 1;
    E wv[RG];   // backward: w at this thread's output column
    for (int p = 0; p < npass; ++p) {
      const int r0 = p * RG, nr = min(RG, a.nrhs - r0);
      if (p > 0) {
        gather_idx(m, r0, nr);
        gather_b(m, r0, nr);
      }
      if (ok) {
        // values written by other blocks of this launch
        if constexpr (kPre) {
#pragma unroll
          for (int i = 0; i < kRowItems; ++i) {
            const int q = tid + i * kSweepThreads;
            if (q < rows * nr) {
              const int r = r0 + q % nr;
              E* dst = vs + (q / nr) * RG + q % nr;
              if (fwd) {
                E v;
                from_c128(v, pv[i]);
                if (pc2[i].x >= 0) addto(v, ldcg(uvE + r * a.uv_total + pc2[i].x));
                if (pc2[i].y >= 0) addto(v, ldcg(uvE + r * a.uv_total + pc2[i].y));
                *dst = norm(v);
              } else {
                const long long gi = r * a.nodes + pI[i];
                if (DF) *reinterpret_cast<float4*>(dst) = __ldcg(a.xd + gi);
                else *reinterpret_cast<double2*>(dst) = __ldcg(a.x + gi);
              }
            }
          }
        } else {
          for (int q = tid; q < rows * nr; q += kSweepThreads) {
            const int t = r0j + q / nr, r = r0 + q % nr;
            E* dst = vs + (q / nr) * RG + q % nr;
            if (fwd) {
              E v;
              from_c128(v, a.b[r * a.nodes + a.S[m.S_off + t]]);
              const int2 cc = a.ctb[m.ctb_off + t];
              if (cc.x >= 0) addto(v, ldcg(uvE + r * a.uv_total + cc.x));
              if (cc.y >= 0) addto(v, ldcg(uvE + r * a.uv_total + cc.y));
              *dst = norm(v);
            } else {
              const long long gi = r * a.nodes + a.B[m.B_off + t];
              if (DF) *reinterpret_cast<float4*>(dst) = __ldcg(a.xd + gi);
              else *reinterpret_cast<double2*>(dst) = __ldcg(a.x + gi);
            }
          }
        }
        if (fwd) {
#pragma unroll
          for (int i = 0; i < kColItems; ++i) {
            const int q = tid + i * kSweepThreads;
            if (q < cols * nr) {
              const int r = r0 + q % nr;
              E v;
              zero(v);
              if (qc2[i].x >= 0) addto(v, ldcg(uvE + r * a.uv_total + qc2[i].x));
              if (qc2[i].y >= 0) addto(v, ldcg(uvE + r * a.uv_total + qc2[i].y));
              rbs[(q / nr) * RG + q % nr] = v;
            }
          }
        } else if (nchunks == 1 && tid < cols) {
#pragma unroll
          for (int rr = 0; rr < RG; ++rr)
            if (rr < nr) wv[rr] = ldcg(wE + (r0 + rr) * a.nodes + sI[0]);
        }
      }
      const bool last = p == npass - 1;
      if (last && warp == kMetaWarp && jn < a.njobs) reinterpret_cast<int*>(metas + (cur ^ 1))[lane] = next_word;
      consumer_sync();   // row values in place; the next job's record too
      // the next job's indices, read while this one streams its factor rows (its b once
      // they have arrived); this job's index registers are no longer needed
      pre_done = last && jn < a.njobs;
      if (pre_done) gather_idx(metas[cur ^ 1], 0, min(RG, a.nrhs));
      E acc[RG];
#pragma unroll
      for (int rr = 0; rr < RG; ++rr) zero(acc[rr]);
      for (int k = 0; k < nst; ++k) {
        consume([&](const E* st) {
          if (!act) return;
          const int base = k * m.srows, n = min(m.srows, rows - base);
#pragma unroll 2
          for (int q = part; q < n; q += nsplit) {
            const E mv = st[q * cols + c];
            const E* rv = vs + (base + q) * RG;
#pragma unroll
            for (int rr = 0; rr < RG; ++rr)
              if (RG == 1 || rr < nr) mac(acc[rr], mv, rv[rr]);
          }
        });
      }
      // the next job's right-hand-side values at the row nodes just gathered (this job's
      // value registers were consumed before its stage loop)
      if (pre_done) gather_b(metas[cur ^ 1], 0, min(RG, a.nrhs));
      if (!direct) {
        consumer_sync();   // every thread is done with the row values red overwrites
        if (ok && act)
#pragma unroll
          for (int rr = 0; rr < RG; ++rr) red[tid * RG + rr] = acc[rr];
        consumer_sync();
      }
      if (ok && tid < cols) {
#pragma unroll
        for (int rr = 0; rr < RG; ++rr) {
          if (rr >= nr) break;
          E v = acc[rr];
          if (!direct) {
            v = red[tid * RG + rr];
            for (int pp = 1; pp < nsplit; ++pp) addto(v, red[(pp * cols + tid) * RG + rr]);
          }
          const int r = r0 + rr;
          if (nchunks == 1) {
            const E o = norm(v);
            const int t = c0j + tid;
            if (fwd && t >= nS) {
              E u = rbs[tid * RG + rr];
              addto(u, m.bsign > 0 ? o : neg(o));
              uvE[r * a.uv_total + m.uv_off + t - nS] = norm(u);
            } else if (fwd) {
              wE[r * a.nodes + sidx[tid]] = o;
            } else {
              write_x(r * a.nodes + sidx[tid], wv[rr], o);
            }
          } else {
            reinterpret_cast<E*>(a.part)[((long long)(m.pbase + m.chunk) * a.nrhs + r) * kPartBlock + tid] = v;
          }
        }
      }
      consumer_sync();
    }
    ok = ok && !*abort_copy;

    // ---- output unit: the last of its jobs adds the partial sums in chunk order
    bool finalized = nchunks == 1;
    if (!finalized) {
      if (tid == 0) *flag = ok && atom_add_acq_rel(a.counters + m.slot) == (unsigned)nchunks - 1;
      consumer_sync();
      finalized = *flag;
      consumer_sync();
      if (finalized) {
        const E* P = reinterpret_cast<const E*>(a.part);
        const long long step = (long long)a.nrhs * kPartBlock;
        for (int q = tid; q < cols * a.nrhs; q += kSweepThreads) {
          const int i = q % cols, r = q / cols;
          const E* src = P + ((long long)m.pbase * a.nrhs + r) * kPartBlock + i;
          E v;
          zero(v);
          int ch = 0;
          for (; ch + 8 <= nchunks; ch += 8) {
            E t8[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) t8[u] = ldcg(src + (ch + u) * step);
#pragma unroll
            for (int u = 0; u < 8; ++u) addto(v, t8[u]);
          }
          for (; ch < nchunks; ++ch) addto(v, ldcg(src + ch * step));
          const E o = norm(v);
          const int t = c0j + i;
          if (fwd && t >= nS) {
            // r_F at t: the children's update-vector entries mapped to t (t is a boundary position)
            E rb;
            zero(rb);
            const int2 cc = a.ctb[m.ctb_off + t];
            if (cc.x >= 0) addto(rb, ldcg(uvE + r * a.uv_total + cc.x));
            if (cc.y >= 0) addto(rb, ldcg(uvE + r * a.uv_total + cc.y));
            addto(rb, m.bsign > 0 ? o : neg(o));
            uvE[r * a.uv_total + m.uv_off + t - nS] = norm(rb);
          } else {
            const long long gi = r * a.nodes + sidx[i];
            if (fwd) wE[gi] = o;
            else write_x(gi, ldcg(wE + gi), o);
          }
        }
      }
      consumer_sync();   // the finalisation's outputs are written (a single job's were, at the pass's end)
    }
    // published by a thread of warp 1: its release waits for the outputs to be visible while
    // thread 0 already polls the next job's dependencies
    if (finalized && ok && tid == 32) red_release(a.counters + m.done);
    next_word = next2_word;
  }
}

template <bool DF, int RG>
cudaError_t launch_one(const SweepArgs& a, int grid, cudaStream_t s) {
  // every block of the grid must be resident (cooperative launch): the schedule's waits
  // rely on it; any such grid size is correct, the job sizes were planned for cs.grid
  static std::atomic<bool> attr{false};
  if (!attr) {
    const cudaError_t e = cudaFuncSetAttribute(sweep_kernel<DF, RG>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes<RG>());
    if (e != cudaSuccess) return e;
    attr = true;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kBlockThreads);
  cfg.dynamicSmemBytes = smem_bytes<RG>();
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, sweep_kernel<DF, RG>, a);
}

template <bool DF, int RG>
int blocks_per_sm() {
  if (cudaFuncSetAttribute(sweep_kernel<DF, RG>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes<RG>()) != cudaSuccess)
    return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sweep_kernel<DF, RG>, kBlockThreads, smem_bytes<RG>()) != cudaSuccess)
    return 0;
  return n;
}

}  // namespace

int sweep_grid_size(int* grid, int* grid_group) {
  int dev = 0, sms = 0;
  HELM_CUDA_TRY(cudaGetDevice(&dev));
  HELM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int per_sm = std::min(blocks_per_sm<true, 1>(), blocks_per_sm<false, 1>());
  const int per_sm_group = std::min(blocks_per_sm<true, kRhsGroup>(), blocks_per_sm<false, kRhsGroup>());
  if (per_sm < 1 || per_sm_group < 1) {
    set_error("coarsest solve kernel does not fit on a multiprocessor");
    return HELM_ECUDA;
  }
  *grid = per_sm * sms;
  *grid_group = per_sm_group * sms;
  return 0;
}

int sweep_launch(const CoarseSolver& cs, const double2* b, double2* e, int nrhs, double2* uv, double2* w,
                 double2* part, unsigned* counters, float4* xd, cudaStream_t s) {
  HELM_CUDA_TRY(cudaMemsetAsync(counters, 0, cs.n_counters * sizeof(unsigned), s));
  SweepArgs a;
  a.meta = cs.d_meta;
  a.njobs = cs.njobs;
  a.S = cs.d_S;
  a.B = cs.d_B;
  a.ctb = cs.d_ctb;
  a.factors = cs.d_factors;
  a.b = b;
  a.uv = uv;
  a.w = w;
  a.x = e;
  a.xd = xd;
  a.part = part;
  a.counters = counters;
  a.err = cs.d_err;
  a.nrhs = nrhs;
  a.nodes = cs.g.size;
  a.uv_total = cs.uv_total;
  a.wait_cycles = cs.wait_cycles;
  cudaError_t le;
  if (nrhs == 1) le = cs.df ? launch_one<true, 1>(a, cs.grid, s) : launch_one<false, 1>(a, cs.grid, s);
  else le = cs.df ? launch_one<true, kRhsGroup>(a, cs.grid_group, s) : launch_one<false, kRhsGroup>(a, cs.grid_group, s);
  if (le != cudaSuccess) {
    set_error(std::string("coarsest solve launch: ") + cudaGetErrorString(le));
    return HELM_ECUDA;
  }
  HELM_LAUNCH_CHECK();
  return 0;
}

}  // namespace helm
