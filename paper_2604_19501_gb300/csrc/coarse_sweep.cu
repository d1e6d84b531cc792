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
// solved together.
#include <type_traits>
#include "coarse.cuh"
#include "df64.cuh"

namespace helm {

namespace {

constexpr int kSplitMax = 16;                              // forward row parts per column
// Limit on any wait, in cycles of the waiting multiprocessor's clock (clock64 is
// monotonic per multiprocessor): about 2 s at the maximum SM clock, longer below it.
constexpr long long kWaitCycles = 4000000000LL;
constexpr int kStageBytes = kStageEntries * 16;
// The ring is deeper for single right-hand sides, whose per-job scratch is smaller.
template <int RG>
__host__ __device__ constexpr int ring_stages() { return RG == 1 ? 6 : 4; }
// per-job scratch: row values [kJobRows][RG] (reused for the row-part sums
// [kSweepThreads][RG] once the job's stages are consumed) and forward r_B [kTile][RG]
template <int RG>
__host__ __device__ constexpr int local_bytes() {
  return ((kJobRows > kSweepThreads ? kJobRows : kSweepThreads) + kTile) * RG * 16;
}
template <int RG>
__host__ __device__ constexpr int smem_bytes() { return ring_stages<RG>() * kStageBytes + local_bytes<RG>() + 2048; }
static_assert(smem_bytes<kRhsGroup>() * 2 + 2048 <= 233472, "two blocks per multiprocessor");
static_assert(kTile <= kPartBlock, "partial block");
static_assert(kTile <= kSweepThreads, "one thread per output column at least");

struct SweepArgs {
  const FrontDesc* desc;
  const SweepJob* jobs;
  int njobs;
  const int* S;
  const int* B;
  const int* kids;
  const int2* ctb;
  const double2* factors;
  const double2* b;
  double2* uv;
  double2* w;
  double2* x;
  float4* xd;
  double2* part;
  unsigned* fwd_done;
  unsigned* bwd_done;
  unsigned* slots;
  int* err;
  int nrhs;
  long long nodes;
  long long uv_total;
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
__device__ __forceinline__ void from_c128(double2& a, double2 v) { a = v; }
__device__ __forceinline__ void from_c128(float4& a, double2 v) { a = to_df(v); }
__device__ __forceinline__ double2 to_c128(double2 a) { return a; }
__device__ __forceinline__ double2 to_c128(float4 a) { return from_df(a); }
__device__ __forceinline__ double2 ldcg(const double2* p) { return __ldcg(p); }
__device__ __forceinline__ float4 ldcg(const float4* p) { return __ldcg(p); }

// ---- synchronisation primitives
__device__ __forceinline__ bool expired(long long t0) { return clock64() - t0 > kWaitCycles; }
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

// *p >= target within the time limit; false on a timeout (recorded) or when another
// block has already recorded an error.
__device__ bool wait_count(const unsigned* p, unsigned target, int* err) {
  if (ld_acquire(p) >= target) return true;
  const long long t0 = clock64();
  while (true) {
    __nanosleep(64);
    if (ld_acquire(p) >= target) return true;
    if (ld_relaxed(err)) return false;
    if (expired(t0)) {
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
__device__ __forceinline__ int job_stages(const SweepJob& J) {
  return J.srows ? (J.r1 - J.r0 + J.srows - 1) / J.srows : 0;
}
struct Cursor {
  int j, pass, k, nst;
  int rows, cols, srows;
  long long ld;
  const double2* src;   // factor row r0 of the job, column c0
};
__device__ void cursor_load(Cursor& c, const SweepArgs& a) {
  for (; c.j < a.njobs; c.j += gridDim.x) {
    const SweepJob J = a.jobs[c.j];
    c.nst = job_stages(J);
    if (!c.nst) continue;
    const FrontDesc& d = a.desc[J.front];
    c.rows = J.r1 - J.r0;
    c.cols = J.c1 - J.c0;
    c.srows = J.srows;
    c.ld = J.kind == 0 ? (long long)(d.nS + d.nB) : (long long)d.g_ld;
    c.src = a.factors + (J.kind == 0 ? d.M_off : d.G_off) + (long long)J.r0 * c.ld + J.c0;
    return;
  }
}
__device__ void cursor_next(Cursor& c, const SweepArgs& a, int npass) {
  if (++c.k < c.nst) return;
  c.k = 0;
  if (++c.pass < npass) return;
  c.pass = 0;
  c.j += gridDim.x;
  cursor_load(c, a);
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

// r_F at front position t: b at the eliminated nodes plus the children's update-vector
// entries mapped to t (at most one per child), added in child order.
__device__ __forceinline__ double2 front_rhs(const SweepArgs& a, const FrontDesc& d, int t, int r) {
  double2 v = t < d.nS ? a.b[r * a.nodes + a.S[d.S_off + t]] : make_double2(0.0, 0.0);
  const int2 c = a.ctb[d.ctb_off + t];
  if (c.x >= 0) addto(v, __ldcg(a.uv + r * a.uv_total + c.x));
  if (c.y >= 0) addto(v, __ldcg(a.uv + r * a.uv_total + c.y));
  return v;
}
constexpr int kBlockThreads = kSweepThreads + 32;   // consumers + one producer warp

__device__ __forceinline__ void consumer_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kSweepThreads) : "memory"); }
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Block layout: warps 0-7 consume (compute), warp 8 produces (copies factor rows into the
// ring).  Stage i of the block's fill sequence uses slot i mod NST; full[slot] completes
// when its copies land, empty[slot] when all consumer warps are done with it.
template <bool DF, int RG>
__global__ void __launch_bounds__(kBlockThreads, 2) sweep_kernel(const SweepArgs a) {
  using E = typename std::conditional<DF, float4, double2>::type;
  // gather items a consumer thread handles per pass: the job's rows x group, its columns x group
  constexpr int kRowItems = (kJobRows * RG + kSweepThreads - 1) / kSweepThreads;
  constexpr int kColItems = (kTile * RG + kSweepThreads - 1) / kSweepThreads;
  constexpr int NST = ring_stages<RG>();
  constexpr int kLocalBytes = local_bytes<RG>();
  extern __shared__ __align__(128) unsigned char smem[];
  E* const stage = reinterpret_cast<E*>(smem);
  unsigned char* const local = smem + NST * kStageBytes;
  E* const vs = reinterpret_cast<E*>(local);   // row values [kJobRows][RG]
  E* const red = vs;                           // row-part sums [threads][RG], after the stages
  double2* const rbs = reinterpret_cast<double2*>(vs + (kJobRows > kSweepThreads ? kJobRows : kSweepThreads) * RG);   // forward r_B [kTile][RG]
  uint64_t* const full = reinterpret_cast<uint64_t*>(local + kLocalBytes);
  uint64_t* const empty = full + NST;
  volatile int* const flag = reinterpret_cast<volatile int*>(empty + NST);
  volatile int* const abort_copy = flag + 1;
  int* const sidx = const_cast<int*>(flag) + 4;                         // node of each output column [kTile]
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
  __syncthreads();

  if (warp == kSweepThreads / 32) {
    // ---- producer: walk the block's fill sequence, one slot ahead of the consumers' release
    Cursor pc;
    pc.j = blockIdx.x;
    pc.pass = pc.k = 0;
    cursor_load(pc, a);
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
      cursor_next(pc, a, npass);
    }
    // copies still in flight must land before the block may exit (bounded)
    for (long long q = i > NST ? i - NST : 0; q < i; ++q)
      if (!mbar_wait(smem_u32(&full[q % NST]), (uint32_t)((q / NST) & 1))) break;
    return;
  }

  // ---- consumers
  long long ci = 0;   // position in the fill sequence
  bool ok = true;     // uniform over the consumers: false once a dependency failed anywhere
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

  for (int j = blockIdx.x; j < a.njobs; j += gridDim.x) {
    const SweepJob J = a.jobs[j];
    const FrontDesc d = a.desc[J.front];
    const bool fwd = J.kind == 0;
    const int nst = job_stages(J);
    const int rows = J.r1 - J.r0, cols = J.c1 - J.c0;

    // Gathers of one pass, split into what is known before the dependencies complete
    // (right-hand side b, node and child-map indices) and what other blocks of this
    // launch write (children's update vectors; the ancestors' x_B).
    double2 pv[kRowItems];
    int2 pc2[kRowItems], qc2[kColItems];
    auto gather_pre = [&](int r0, int nr) {
      for (int q = tid; q < cols; q += kSweepThreads) {
        const int t = J.c0 + q;
        sidx[q] = (!fwd || t < d.nS) ? a.S[d.S_off + t] : -1;
      }
#pragma unroll
      for (int i = 0; i < kRowItems; ++i) {
        const int q = tid + i * kSweepThreads;
        if (q < rows * nr) {
          const int t = J.r0 + q / nr, r = r0 + q % nr;
          if (fwd) {
            pv[i] = a.b[r * a.nodes + a.S[d.S_off + t]];
            pc2[i] = a.ctb[d.ctb_off + t];
          } else {
            pc2[i].x = a.B[d.B_off + t];
          }
        }
      }
      if (fwd)
#pragma unroll
        for (int i = 0; i < kColItems; ++i) {
          const int q = tid + i * kSweepThreads;
          if (q < cols * nr) {
            const int t = J.c0 + q / nr;
            qc2[i] = t >= d.nS ? a.ctb[d.ctb_off + t] : make_int2(-1, -1);
          }
        }
    };
    auto gather_post = [&](int r0, int nr) {
#pragma unroll
      for (int i = 0; i < kRowItems; ++i) {
        const int q = tid + i * kSweepThreads;
        if (q < rows * nr) {
          const int r = r0 + q % nr;
          E* dst = vs + (q / nr) * RG + q % nr;
          if (fwd) {
            double2 v = pv[i];
            if (pc2[i].x >= 0) addto(v, __ldcg(a.uv + r * a.uv_total + pc2[i].x));
            if (pc2[i].y >= 0) addto(v, __ldcg(a.uv + r * a.uv_total + pc2[i].y));
            from_c128(*dst, v);
          } else {
            const long long gi = r * a.nodes + pc2[i].x;
            if (DF) *reinterpret_cast<float4*>(dst) = __ldcg(a.xd + gi);
            else *reinterpret_cast<double2*>(dst) = __ldcg(a.x + gi);
          }
        }
      }
      if (fwd)
#pragma unroll
        for (int i = 0; i < kColItems; ++i) {
          const int q = tid + i * kSweepThreads;
          if (q < cols * nr) {
            const int r = r0 + q % nr;
            double2 v = make_double2(0.0, 0.0);
            if (qc2[i].x >= 0) addto(v, __ldcg(a.uv + r * a.uv_total + qc2[i].x));
            if (qc2[i].y >= 0) addto(v, __ldcg(a.uv + r * a.uv_total + qc2[i].y));
            rbs[(q / nr) * RG + q % nr] = v;
          }
        }
    };
    // result v of column c for right-hand side r: forward, w at node S[t] (t = c0 + c < nS)
    // or the update-vector entry r_B + bsign v; backward, x_S = w_S - v
    auto write_out = [&](int c, int r, double2 v, double2 rb) {
      const int t = J.c0 + c;
      if (fwd && t >= d.nS) {
        a.uv[r * a.uv_total + d.uv_off + t - d.nS] = make_double2(rb.x + d.bsign * v.x, rb.y + d.bsign * v.y);
        return;
      }
      const long long gi = r * a.nodes + sidx[c];
      if (fwd) {
        a.w[gi] = v;
      } else {
        const double2 wv = __ldcg(a.w + gi);
        const double2 xv = make_double2(wv.x - v.x, wv.y - v.y);
        a.x[gi] = xv;
        if (DF) a.xd[gi] = to_df(xv);
      }
    };

    gather_pre(0, min(RG, a.nrhs));
    // dependencies
    if (tid == 0) {
      bool good = ok && !ld_relaxed(a.err);
      if (good) {
        if (fwd) {
          for (int q = 0; q < d.nkids && good; ++q) {
            const int k = a.kids[d.kid_off + q];
            good = wait_count(a.fwd_done + k, (unsigned)a.desc[k].fwd_units, a.err);
          }
        } else if (d.parent < 0) {
          good = wait_count(a.fwd_done + J.front, (unsigned)d.fwd_units, a.err);
        } else {
          good = wait_count(a.bwd_done + d.parent, (unsigned)a.desc[d.parent].bwd_units, a.err);
        }
        __threadfence();
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
    for (int p = 0; p < npass; ++p) {
      const int r0 = p * RG, nr = min(RG, a.nrhs - r0);
      if (p > 0) gather_pre(r0, nr);
      if (ok) gather_post(r0, nr);
      consumer_sync();
      E acc[RG];
#pragma unroll
      for (int rr = 0; rr < RG; ++rr) zero(acc[rr]);
      for (int k = 0; k < nst; ++k) {
        consume([&](const E* st) {
          if (!act) return;
          const int base = k * J.srows, n = min(J.srows, rows - base);
#pragma unroll 2
          for (int q = part; q < n; q += nsplit) {
            const E m = st[q * cols + c];
            const E* rv = vs + (base + q) * RG;
#pragma unroll
            for (int rr = 0; rr < RG; ++rr)
              if (RG == 1 || rr < nr) mac(acc[rr], m, rv[rr]);
          }
        });
      }
      consumer_sync();   // every thread is done with the row values red overwrites
      if (ok && act)
#pragma unroll
        for (int rr = 0; rr < RG; ++rr) red[tid * RG + rr] = acc[rr];
      consumer_sync();
      if (ok && tid < cols) {
        for (int rr = 0; rr < nr; ++rr) {
          E v = red[tid * RG + rr];
          for (int pp = 1; pp < nsplit; ++pp) addto(v, red[(pp * cols + tid) * RG + rr]);
          const int r = r0 + rr;
          if (J.nchunks == 1)
            write_out(tid, r, to_c128(v), fwd ? rbs[tid * RG + rr] : make_double2(0.0, 0.0));
          else
            reinterpret_cast<E*>(a.part)[((long long)(J.pbase + J.chunk) * a.nrhs + r) * kPartBlock + tid] = v;
        }
      }
      consumer_sync();
    }
    ok = ok && !*abort_copy;

    // ---- output unit: the last of its jobs adds the partial sums in chunk order
    bool finalized = J.nchunks == 1;
    if (!finalized) {
      __threadfence();
      consumer_sync();
      if (tid == 0) *flag = ok && atomicAdd(a.slots + J.slot, 1u) == (unsigned)J.nchunks - 1;
      consumer_sync();
      finalized = *flag;
      consumer_sync();
      if (finalized) {
        __threadfence();
        const E* P = reinterpret_cast<const E*>(a.part);
        const long long step = (long long)a.nrhs * kPartBlock;
        for (int q = tid; q < cols * a.nrhs; q += kSweepThreads) {
          const int i = q % cols, r = q / cols;
          const E* src = P + ((long long)J.pbase * a.nrhs + r) * kPartBlock + i;
          E v;
          zero(v);
          int ch = 0;
          for (; ch + 8 <= J.nchunks; ch += 8) {
            E t[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) t[u] = ldcg(src + (ch + u) * step);
#pragma unroll
            for (int u = 0; u < 8; ++u) addto(v, t[u]);
          }
          for (; ch < J.nchunks; ++ch) addto(v, ldcg(src + ch * step));
          const int t = J.c0 + i;
          write_out(i, r, to_c128(v), fwd && t >= d.nS ? front_rhs(a, d, t, r) : make_double2(0.0, 0.0));
        }
      }
    }
    if (finalized && ok) {
      __threadfence();
      consumer_sync();
      if (tid == 0) atomicAdd((fwd ? a.fwd_done : a.bwd_done) + J.front, 1u);
    }
    consumer_sync();
  }
}

template <bool DF, int RG>
cudaError_t launch_one(const SweepArgs& a, int grid, cudaStream_t s) {
  static bool attr = false;
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

int sweep_grid_size(int* grid) {
  int dev = 0, sms = 0;
  HELM_CUDA_TRY(cudaGetDevice(&dev));
  HELM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int per_sm = std::min(std::min(blocks_per_sm<true, 1>(), blocks_per_sm<true, kRhsGroup>()),
                              std::min(blocks_per_sm<false, 1>(), blocks_per_sm<false, kRhsGroup>()));
  if (per_sm < 1) {
    set_error("coarsest solve kernel does not fit on a multiprocessor");
    return HELM_ECUDA;
  }
  *grid = per_sm * sms;
  return 0;
}

int sweep_launch(const CoarseSolver& cs, const double2* b, double2* e, int nrhs, double2* uv, double2* w,
                 double2* part, unsigned* counters, float4* xd, cudaStream_t s) {
  HELM_CUDA_TRY(cudaMemsetAsync(counters, 0, cs.n_counters * sizeof(unsigned), s));
  SweepArgs a;
  a.desc = cs.d_desc;
  a.jobs = cs.d_jobs;
  a.njobs = cs.njobs;
  a.S = cs.d_S;
  a.B = cs.d_B;
  a.kids = cs.d_kids;
  a.ctb = cs.d_ctb;
  a.factors = cs.d_factors;
  a.b = b;
  a.uv = uv;
  a.w = w;
  a.x = e;
  a.xd = xd;
  a.part = part;
  a.fwd_done = counters;
  a.bwd_done = counters + cs.nfronts;
  a.slots = counters + 2 * cs.nfronts;
  a.err = cs.d_err;
  a.nrhs = nrhs;
  a.nodes = cs.g.size;
  a.uv_total = cs.uv_total;
  cudaError_t le;
  if (nrhs == 1) le = cs.df ? launch_one<true, 1>(a, cs.grid, s) : launch_one<false, 1>(a, cs.grid, s);
  else le = cs.df ? launch_one<true, kRhsGroup>(a, cs.grid, s) : launch_one<false, kRhsGroup>(a, cs.grid, s);
  if (le != cudaSuccess) {
    set_error(std::string("coarsest solve launch: ") + cudaGetErrorString(le));
    return HELM_ECUDA;
  }
  HELM_LAUNCH_CHECK();
  return 0;
}

}  // namespace helm
