// Exact solve on the coarsest level (Sec. 2: the coarse-grid correction uses an exact
// solution on the coarsest grid; Sec. 3.1: three levels so that the coarsest is small
// enough to solve directly).  The paper leaves the method open; this is a nested-
// dissection multifrontal factorisation in complex FP64.
//
// Symbolic phase (host): the node box is bisected recursively along its longest axis by
// separator slabs r nodes thick (r = stencil radius), which decouple the two halves.
// Every tree node ("front") eliminates its separator S (a leaf: its whole box); its
// boundary B is the ring of nodes within distance r around its box, all of which lie in
// ancestor separators.
//
// Numeric phase (device, level by level from the leaves): the front matrix F over
// S u B is assembled from the stencil entries of the S rows/columns and the children's
// update matrices (extend-add), then Gauss-Jordan elimination with row pivoting inside S
// on the augmented matrix [F | I_S] yields
//   rows S: [ I | F_SS^-1 F_SB | F_SS^-1 ],   rows B: [ 0 | U | -F_BS F_SS^-1 ],
// U = F_BB - F_BS F_SS^-1 F_SB being the update passed to the parent.
//
// Stored per front: M = [F_SS^-1 | F_SS^-1 F_SB] (|S| x |F|) when the coarsest operator is
// complex-symmetric (full-weighting or cubic transfers on both levels), since then
// F_BS F_SS^-1 = (F_SS^-1 F_SB)^T; otherwise M = [F_SS^-1 | -F_BS F_SS^-1]^T.  Both cases
// also keep G^T = (F_SS^-1 F_SB)^T (|B| x |S|).  Small fronts are eliminated by one thread
// block each; large fronts by a pair of grid-wide kernels per pivot (pivot search + row
// swap/scale, elimination).
//
// Solve (coarse_sweep.cu): forward, leaves to root, every front turns its assembled
// right-hand side r_F into w_S = F_SS^-1 r_S and the update vector r_B - F_BS F_SS^-1 r_S
// for its parent, as column sums over M.  Backward, root to leaves,
// x_S = w_S - (F_SS^-1 F_SB) x_B, as column sums over G^T.  Both are split into row chunks
// whose partial sums the last job of a column tile adds in chunk order: the summation
// order is fixed, so results are reproducible bit for bit.
#include <algorithm>
#include <mutex>
#include <unordered_map>
#include "coarse.cuh"
#include "df64.cuh"
#include "timer.cuh"

namespace helm {

namespace {

struct HostFront {
  int height = 0;
  int parent = -1;
  std::vector<int> S, B, kids;
  int lo[3], hi[3];
};

struct Builder {
  int dim, N[3], r, leaf_max;
  std::vector<HostFront> fronts;

  int gidx(int x, int y, int z) const { return x + N[0] * (y + N[1] * z); }

  void box_nodes(const int lo[3], const int hi[3], std::vector<int>& out) const {
    for (int z = lo[2]; z < hi[2]; ++z)
      for (int y = lo[1]; y < hi[1]; ++y)
        for (int x = lo[0]; x < hi[0]; ++x) out.push_back(gidx(x, y, z));
  }

  void ring_nodes(const int lo[3], const int hi[3], std::vector<int>& out) const {
    int a[3], b[3];
    for (int d = 0; d < 3; ++d) {
      const int rr = d < dim ? r : 0;
      a[d] = std::max(0, lo[d] - rr);
      b[d] = std::min(N[d], hi[d] + rr);
    }
    for (int z = a[2]; z < b[2]; ++z)
      for (int y = a[1]; y < b[1]; ++y)
        for (int x = a[0]; x < b[0]; ++x) {
          const bool inside = x >= lo[0] && x < hi[0] && y >= lo[1] && y < hi[1] && z >= lo[2] && z < hi[2];
          if (!inside) out.push_back(gidx(x, y, z));
        }
  }

  int build(const int lo[3], const int hi[3], int parent) {
    const int id = (int)fronts.size();
    fronts.emplace_back();
    {
      HostFront& f = fronts[id];
      f.parent = parent;
      for (int d = 0; d < 3; ++d) { f.lo[d] = lo[d]; f.hi[d] = hi[d]; }
    }
    long long vol = 1;
    int axis = 0, ext = 0;
    for (int d = 0; d < dim; ++d) {
      vol *= (hi[d] - lo[d]);
      if (hi[d] - lo[d] > ext) { ext = hi[d] - lo[d]; axis = d; }
    }
    std::vector<int> S, B;
    ring_nodes(lo, hi, B);
    if (vol <= leaf_max || ext < r + 2) {
      box_nodes(lo, hi, S);
    } else {
      const int mid = lo[axis] + (ext - r) / 2;
      int llo[3], lhi[3], slo[3], shi[3], rlo[3], rhi[3];
      for (int d = 0; d < 3; ++d) {
        llo[d] = slo[d] = rlo[d] = lo[d];
        lhi[d] = shi[d] = rhi[d] = hi[d];
      }
      lhi[axis] = mid;
      slo[axis] = mid;
      shi[axis] = mid + r;
      rlo[axis] = mid + r;
      box_nodes(slo, shi, S);
      std::vector<int> kids;
      kids.push_back(build(llo, lhi, id));
      if (rhi[axis] > rlo[axis]) kids.push_back(build(rlo, rhi, id));
      int h = 0;
      for (int k : kids) h = std::max(h, fronts[k].height + 1);
      fronts[id].kids = kids;
      fronts[id].height = h;
    }
    fronts[id].S = std::move(S);
    fronts[id].B = std::move(B);
    return id;
  }
};

// ------------------------------------------------------------------ factorisation kernels
__global__ void fact_assemble_kernel(const FrontDesc* __restrict__ desc, const int* __restrict__ list,
                                     double2* __restrict__ aug, const int2* __restrict__ ents,
                                     const double2* __restrict__ coef, const double2* __restrict__ upool,
                                     const int* __restrict__ kids, const int* __restrict__ cmap) {
  const FrontDesc d = desc[list[blockIdx.x]];
  const int nF = d.nS + d.nB, ld = nF + d.nS;
  double2* A = aug + d.aug_off;
  const long long tot = (long long)nF * ld;
  for (long long t = threadIdx.x; t < tot; t += blockDim.x) {
    const int row = (int)(t / ld), col = (int)(t % ld);
    A[t] = make_double2((row < d.nS && col == nF + row) ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  // original entries: each destination appears once per front
  for (int e = threadIdx.x; e < d.ent_cnt; e += blockDim.x) {
    const int2 en = ents[d.ent_off + e];
    const double2 v = coef[en.y];
    A[en.x].x += v.x;
    A[en.x].y += v.y;
  }
  __syncthreads();
  // extend-add of the children's update matrices, one child at a time
  for (int c = 0; c < d.nkids; ++c) {
    const FrontDesc kd = desc[kids[d.kid_off + c]];
    const int* map = cmap + kd.cmap_off;
    const double2* U = upool + kd.U_off;
    const long long n2 = (long long)kd.nB * kd.nB;
    for (long long t = threadIdx.x; t < n2; t += blockDim.x) {
      const int a = (int)(t / kd.nB), b = (int)(t % kd.nB);
      const double2 v = U[t];
      double2& dst = A[(long long)map[a] * ld + map[b]];
      dst.x += v.x;
      dst.y += v.y;
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(512) fact_gj_kernel(const FrontDesc* __restrict__ desc,
                                                      const int* __restrict__ list,
                                                      double2* __restrict__ aug, int* __restrict__ err) {
  const FrontDesc d = desc[list[blockIdx.x]];
  const int nS = d.nS, nF = d.nS + d.nB, ld = nF + d.nS;
  double2* A = aug + d.aug_off;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  __shared__ double s_val[32];
  __shared__ int s_idx[32];
  __shared__ int s_piv;
  __shared__ double2 s_inv;
  for (int k = 0; k < nS; ++k) {
    // pivot: largest |a_ik| over the rows of S not yet eliminated (ties: lowest row)
    double best = -1.0;
    int bi = nS;
    for (int i = k + tid; i < nS; i += blockDim.x) {
      const double2 a = A[(long long)i * ld + k];
      const double v = a.x * a.x + a.y * a.y;
      if (v > best) { best = v; bi = i; }
    }
    for (int off = 16; off > 0; off >>= 1) {
      const double ov = __shfl_down_sync(0xffffffffu, best, off);
      const int oi = __shfl_down_sync(0xffffffffu, bi, off);
      if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    if (lane == 0) { s_val[warp] = best; s_idx[warp] = bi; }
    __syncthreads();
    if (tid == 0) {
      double bv = s_val[0];
      int bidx = s_idx[0];
      for (int w = 1; w < nwarp; ++w)
        if (s_val[w] > bv || (s_val[w] == bv && s_idx[w] < bidx)) { bv = s_val[w]; bidx = s_idx[w]; }
      if (!(bv > 0.0) || !isfinite(bv) || bidx >= nS) { atomicExch(err, 1); bidx = k; }
      s_piv = bidx;
    }
    __syncthreads();
    const int p = s_piv;
    if (p != k)
      for (int c = k + tid; c < ld; c += blockDim.x) {
        const double2 t = A[(long long)k * ld + c];
        A[(long long)k * ld + c] = A[(long long)p * ld + c];
        A[(long long)p * ld + c] = t;
      }
    __syncthreads();
    if (tid == 0) {
      const double2 a = A[(long long)k * ld + k];
      const double m = a.x * a.x + a.y * a.y;
      s_inv = make_double2(a.x / m, -a.y / m);
    }
    __syncthreads();
    const double2 inv = s_inv;
    for (int c = k + 1 + tid; c < ld; c += blockDim.x) {
      const double2 a = A[(long long)k * ld + c];
      A[(long long)k * ld + c] = make_double2(a.x * inv.x - a.y * inv.y, a.x * inv.y + a.y * inv.x);
    }
    __syncthreads();
    if (tid == 0) A[(long long)k * ld + k] = make_double2(1.0, 0.0);
    for (int i = warp; i < nF; i += nwarp) {
      if (i == k) continue;
      const double2 f = A[(long long)i * ld + k];
      if (f.x == 0.0 && f.y == 0.0) continue;
      double2* Ai = A + (long long)i * ld;
      const double2* Ak = A + (long long)k * ld;
      for (int c = k + 1 + lane; c < ld; c += 32) {
        const double2 b = Ak[c];
        double2 v = Ai[c];
        v.x -= f.x * b.x - f.y * b.y;
        v.y -= f.x * b.y + f.y * b.x;
        Ai[c] = v;
      }
      __syncwarp();
      if (lane == 0) Ai[k] = make_double2(0.0, 0.0);
    }
    __syncthreads();
  }
}


// ------------------------------------------------------------------ large-front elimination
// One pivot step k of Gauss-Jordan elimination on the augmented fronts of a level, split
// over many blocks.  Kernel 1: every block finds the same pivot row p (largest |a_ik|,
// rows k..nS-1, lowest index on ties), block 0 records p and the old a_kk, and every
// block swaps rows k and p and scales the new row k over its slice of columns k+1..ld-1
// (column k is left alone so that all blocks read the same pivot value).  Kernel 2: every
// other row i subtracts f_i times row k (f_p = old a_kk) and its column-k entry becomes 0.
__global__ void __launch_bounds__(256) gj_pivot_kernel(const FrontDesc* __restrict__ desc,
                                                       const int* __restrict__ list, double2* __restrict__ aug,
                                                       int k, int* __restrict__ piv, double2* __restrict__ akk,
                                                       int* __restrict__ err) {
  const int fi = blockIdx.y;
  const FrontDesc d = desc[list[fi]];
  const int nS = d.nS, nF = d.nS + d.nB, ld = nF + d.nS;
  if (k >= nS) return;
  double2* A = aug + d.aug_off;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  __shared__ double s_val[32];
  __shared__ int s_idx[32];
  __shared__ int s_p;
  double best = -1.0;
  int bi = nS;
  for (int i = k + tid; i < nS; i += blockDim.x) {
    const double2 a = A[(long long)i * ld + k];
    const double v = a.x * a.x + a.y * a.y;
    if (v > best) { best = v; bi = i; }
  }
  for (int off = 16; off > 0; off >>= 1) {
    const double ov = __shfl_down_sync(0xffffffffu, best, off);
    const int oi = __shfl_down_sync(0xffffffffu, bi, off);
    if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
  }
  if (lane == 0) { s_val[warp] = best; s_idx[warp] = bi; }
  __syncthreads();
  if (tid == 0) {
    double bv = s_val[0];
    int bidx = s_idx[0];
    for (int w = 1; w < nwarp; ++w)
      if (s_val[w] > bv || (s_val[w] == bv && s_idx[w] < bidx)) { bv = s_val[w]; bidx = s_idx[w]; }
    if (!(bv > 0.0) || !isfinite(bv) || bidx >= nS) {
      if (blockIdx.x == 0) atomicExch(err, 1);
      bidx = k;
    }
    s_p = bidx;
    if (blockIdx.x == 0) {
      piv[fi] = bidx;
      akk[fi] = A[(long long)k * ld + k];
    }
  }
  __syncthreads();
  const int p = s_p;
  const double2 a = A[(long long)p * ld + k];
  const double m = a.x * a.x + a.y * a.y;
  const double2 inv = make_double2(a.x / m, -a.y / m);
  const int span = (ld - k - 1 + gridDim.x - 1) / gridDim.x;
  const int c0 = k + 1 + blockIdx.x * span, c1 = min(ld, c0 + span);
  for (int c = c0 + tid; c < c1; c += blockDim.x) {
    const double2 vk = A[(long long)k * ld + c];
    const double2 vp = A[(long long)p * ld + c];
    A[(long long)k * ld + c] = make_double2(vp.x * inv.x - vp.y * inv.y, vp.x * inv.y + vp.y * inv.x);
    if (p != k) A[(long long)p * ld + c] = vk;
  }
}

__global__ void __launch_bounds__(256) gj_elim_kernel(const FrontDesc* __restrict__ desc,
                                                      const int* __restrict__ list, double2* __restrict__ aug,
                                                      int k, const int* __restrict__ piv,
                                                      const double2* __restrict__ akk) {
  const int fi = blockIdx.y;
  const FrontDesc d = desc[list[fi]];
  const int nS = d.nS, nF = d.nS + d.nB, ld = nF + d.nS;
  if (k >= nS) return;
  double2* A = aug + d.aug_off;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int p = piv[fi];
  const double2* Ak = A + (long long)k * ld;
  for (int i = blockIdx.x * nwarp + warp; i < nF; i += gridDim.x * nwarp) {
    double2* Ai = A + (long long)i * ld;
    if (i == k) {
      if (lane == 0) Ai[k] = make_double2(1.0, 0.0);
      continue;
    }
    const double2 f = (i == p) ? akk[fi] : Ai[k];
    if (f.x != 0.0 || f.y != 0.0) {
      for (int c = k + 1 + lane; c < ld; c += 32) {
        const double2 b = Ak[c];
        double2 v = Ai[c];
        v.x -= f.x * b.x - f.y * b.y;
        v.y -= f.x * b.y + f.y * b.x;
        Ai[c] = v;
      }
    }
    if (lane == 0) Ai[k] = make_double2(0.0, 0.0);
  }
}

// Copies the factors out of the eliminated augmented fronts.
// Factors are stored as complex FP64 (double2) or, with `df`, as double-float float4 of the
// same size.
__device__ __forceinline__ void store_factor(double2* base, long long i, double2 v, bool df) {
  if (df) reinterpret_cast<float4*>(base)[i] = to_df(v);
  else base[i] = v;
}

__global__ void fact_extract_kernel(const FrontDesc* __restrict__ desc, const int* __restrict__ list,
                                    const double2* __restrict__ aug, double2* __restrict__ factors,
                                    double2* __restrict__ upool, bool df) {
  const FrontDesc d = desc[list[blockIdx.x]];
  const int nS = d.nS, nB = d.nB, nF = nS + nB, ld = nF + nS;
  const double2* A = aug + d.aug_off;
  double2* M = factors + d.M_off;
  double2* U = upool + d.U_off;
  const long long nm = (long long)nS * nF;
  for (long long t = threadIdx.x; t < nm; t += blockDim.x) {
    const int row = (int)(t / nF), col = (int)(t % nF);
    if (d.bsign < 0)   // [F_SS^-1 | G]
      store_factor(M, t, A[(long long)row * ld + (col < nS ? nF + col : col)], df);
    else               // X^T, X = [F_SS^-1 ; -F_BS F_SS^-1]
      store_factor(M, t, A[(long long)col * ld + nF + row], df);
  }
  // G^T = (F_SS^-1 F_SB)^T, [nB][nS], read by the backward sweep as column sums
  double2* GT = factors + d.G_off;
  for (long long t = threadIdx.x; t < (long long)nS * nB; t += blockDim.x) {
    const int c = (int)(t / nS), row = (int)(t % nS);
    store_factor(GT, t, A[(long long)row * ld + nS + c], df);
  }
  for (long long t = threadIdx.x; t < (long long)nB * nB; t += blockDim.x) {
    const int row = (int)(t / nB), col = (int)(t % nB);
    U[t] = A[(long long)(nS + row) * ld + nS + col];
  }
}

// Host side of the set-up: the nested-dissection tree, the front descriptors and the solve
// job list (no device work).
struct CoarsePlan {
  std::vector<FrontDesc> desc;
  std::vector<int> Sall, Ball, kids, cmap;
  std::vector<int2> ents, ctb;
  std::vector<std::vector<int>> bigs, smalls;
  std::vector<SweepJob> jobs;
  std::vector<SweepMeta> meta;
  long long aug_max = 0, upool = 0;
};

template <typename T>
int upload(T** dst, const std::vector<T>& v) {
  if (v.empty()) { *dst = nullptr; return 0; }
  HELM_CUDA_TRY(cudaMalloc(dst, v.size() * sizeof(T)));
  HELM_CUDA_TRY(cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return 0;
}

constexpr int kJobsPerBlockLevel = 1;   // solve jobs per resident block and tree level aimed for
constexpr int kBigFront = 96;      // fronts with at least this many eliminated nodes use the grid-wide elimination

}  // namespace

// Host check of the solve plan against the extents the solve kernel indexes: every job's
// factor rows and columns inside the factor pool, at most one stage of shared memory per
// fill, partial blocks and slots inside their buffers, and every dependency of a job
// listed before it (the condition under which the persistent schedule cannot deadlock).
static int validate_plan(const CoarseSolver& cs, const CoarsePlan& P) {
  auto bad = [](const std::string& m) {
    set_error("coarsest solve plan: " + m);
    return HELM_EINVAL;
  };
  const auto& D = P.desc;
  std::vector<long long> first_fwd(cs.nfronts, -1), last_fwd(cs.nfronts, -1), first_bwd(cs.nfronts, -1),
      last_bwd(cs.nfronts, -1);
  std::vector<int> fwd_units_seen(cs.nfronts, 0), bwd_units_seen(cs.nfronts, 0);
  for (size_t j = 0; j < P.jobs.size(); ++j) {
    const SweepJob& J = P.jobs[j];
    if (J.front < 0 || J.front >= cs.nfronts) return bad("front index");
    const FrontDesc& d = D[J.front];
    const int rows = J.r1 - J.r0, cols = J.c1 - J.c0;
    if (J.nchunks < 1 || J.chunk < 0 || J.chunk >= J.nchunks) return bad("job chunks");
    if (J.nchunks > 1 && (J.slot < 0 || J.slot >= cs.n_slots || J.pbase < 0 || J.pbase + J.nchunks > cs.part_blocks))
      return bad("partial slot");
    if (J.kind != 0 && J.kind != 1) return bad("job kind");
    // forward: M [nS][nF]; backward: G^T [nB][nS]
    const int nrows = J.kind == 0 ? d.nS : d.nB, ncols = J.kind == 0 ? d.nS + d.nB : d.nS;
    const long long off = J.kind == 0 ? d.M_off : d.G_off;
    if (J.kind == 1 && d.g_ld != d.nS) return bad("backward stride");
    if (J.c0 < 0 || cols < 1 || J.c1 > ncols || cols > kTile || cols > kPartBlock) return bad("job columns");
    if (nrows == 0) {
      if (J.kind != 1 || J.r0 != 0 || J.r1 != 0 || J.srows != 0 || J.nchunks != 1) return bad("empty job");
    } else {
      if (J.r0 < 0 || rows < 1 || J.r1 > nrows || rows > kJobRows) return bad("job rows");
      if (J.srows < 1 || (long long)J.srows * cols > kStageEntries) return bad("job stage");
      if (off + (long long)(J.r1 - 1) * ncols + J.c1 > cs.factor_entries) return bad("factor extent");
    }
    auto& first = J.kind == 0 ? first_fwd : first_bwd;
    auto& last = J.kind == 0 ? last_fwd : last_bwd;
    auto& units = J.kind == 0 ? fwd_units_seen : bwd_units_seen;
    if (first[J.front] < 0) first[J.front] = (long long)j;
    last[J.front] = (long long)j;
    if (J.chunk == 0) ++units[J.front];
  }
  for (int f = 0; f < cs.nfronts; ++f) {
    const FrontDesc& d = D[f];
    if (first_fwd[f] < 0 || first_bwd[f] < 0) return bad("front without jobs");
    if (fwd_units_seen[f] != d.fwd_units || bwd_units_seen[f] != d.bwd_units) return bad("unit counts");
    for (int q = 0; q < d.nkids; ++q)
      if (last_fwd[P.kids[d.kid_off + q]] >= first_fwd[f]) return bad("forward dependency order");
    if (d.parent < 0) {
      if (last_fwd[f] >= first_bwd[f]) return bad("root dependency order");
    } else if (last_bwd[d.parent] >= first_bwd[f]) {
      return bad("backward dependency order");
    }
  }
  return 0;
}

int coarse_plan(CoarseSolver& cs, CoarsePlan& P, const GridDims& g, int r, int leaf_max, bool symmetric,
                int grid) {
  cs.g = g;
  cs.r = r;
  cs.grid = grid;
  auto& desc = P.desc;
  auto& Sall = P.Sall;
  auto& Ball = P.Ball;
  auto& kids = P.kids;
  auto& cmap = P.cmap;
  auto& ents = P.ents;
  auto& ctb = P.ctb;
  auto& bigs = P.bigs;
  auto& smalls = P.smalls;
  auto& jobs = P.jobs;
  Builder bld;
  bld.dim = g.dim;
  for (int d = 0; d < 3; ++d) bld.N[d] = g.N[d];
  bld.r = r;
  bld.leaf_max = leaf_max;
  int lo[3] = {0, 0, 0}, hi[3] = {g.N[0], g.N[1], g.N[2]};
  bld.build(lo, hi, -1);
  auto& F = bld.fronts;
  cs.nfronts = (int)F.size();
  int H = 0;
  for (auto& f : F) H = std::max(H, f.height);
  cs.nlevels = H + 1;
  cs.level_fronts.assign(cs.nlevels, {});
  for (int i = 0; i < cs.nfronts; ++i) cs.level_fronts[F[i].height].push_back(i);

  const int W = 2 * r + 1;
  desc.assign(cs.nfronts, FrontDesc{});
  long long xg = 0, uoff = 0, rfo = 0, uvo = 0;
  for (int i = 0; i < cs.nfronts; ++i) {
    HostFront& f = F[i];
    FrontDesc& d = desc[i];
    d.nS = (int)f.S.size();
    d.nB = (int)f.B.size();
    d.S_off = (int)Sall.size();
    d.B_off = (int)Ball.size();
    Sall.insert(Sall.end(), f.S.begin(), f.S.end());
    Ball.insert(Ball.end(), f.B.begin(), f.B.end());
    const int nF = d.nS + d.nB;
    d.bsign = symmetric ? -1 : 1;
    d.M_off = xg;
    xg += (long long)nF * d.nS;
    d.G_off = xg;       // G^T [nB][nS]
    d.g_ld = d.nS;
    xg += (long long)d.nS * d.nB;
    d.U_off = uoff;
    uoff += (long long)d.nB * d.nB;
    d.ctb_off = rfo;
    rfo += nF;
    d.uv_off = uvo;
    uvo += d.nB;
    d.kid_off = (int)kids.size();
    d.nkids = (int)f.kids.size();
    d.parent = f.parent;
    kids.insert(kids.end(), f.kids.begin(), f.kids.end());
  }
  // child maps and original entries need the position of a node inside a front
  for (int i = 0; i < cs.nfronts; ++i) {
    HostFront& f = F[i];
    FrontDesc& d = desc[i];
    std::unordered_map<int, int> pos;
    pos.reserve(2 * (f.S.size() + f.B.size()));
    for (int t = 0; t < d.nS; ++t) pos[f.S[t]] = t;
    for (int t = 0; t < d.nB; ++t) pos[f.B[t]] = d.nS + t;
    for (int k : f.kids) {
      desc[k].cmap_off = (int)cmap.size();
      for (int node : F[k].B) {
        auto it = pos.find(node);
        if (it == pos.end()) { set_error("nested dissection: child boundary outside parent front"); return HELM_EINVAL; }
        cmap.push_back(it->second);
      }
    }
    const int ld = d.nS + d.nB + d.nS;
    d.ent_off = (int)ents.size();
    for (int t = 0; t < d.nS; ++t) {
      const int node = f.S[t];
      const int x = node % g.N[0], y = (node / g.N[0]) % g.N[1], z = node / (g.N[0] * g.N[1]);
      for (int bz = (g.dim == 3 ? -r : 0); bz <= (g.dim == 3 ? r : 0); ++bz)
        for (int by = -r; by <= r; ++by)
          for (int bx = -r; bx <= r; ++bx) {
            const int X = x + bx, Y = y + by, Z = z + bz;
            if (X < 0 || X >= g.N[0] || Y < 0 || Y >= g.N[1] || Z < 0 || Z >= g.N[2]) continue;
            const int nb = X + g.N[0] * (Y + g.N[1] * Z);
            auto it = pos.find(nb);
            if (it == pos.end()) continue;   // eliminated in a descendant front
            const int o = (bx + r) + W * ((by + r) + W * (g.dim == 3 ? bz + r : 0));
            const int oneg = (-bx + r) + W * ((-by + r) + W * (g.dim == 3 ? -bz + r : 0));
            ents.push_back(make_int2(t * ld + it->second, (int)((long long)o * g.size + node)));
            if (it->second >= d.nS)
              ents.push_back(make_int2(it->second * ld + t, (int)((long long)oneg * g.size + nb)));
          }
    }
    d.ent_cnt = (int)ents.size() - d.ent_off;
  }
  cs.factor_entries = xg;
  cs.bwd_entries = 0;
  for (auto& d : desc) cs.bwd_entries += (long long)d.nS * d.nB;
  cs.max_nB = 0;
  for (auto& d : desc) cs.max_nB = std::max(cs.max_nB, d.nB);
  cs.uv_total = uvo;
  // for every front position, the update-vector entries of the children that map to it
  ctb.assign(rfo, make_int2(-1, -1));
  for (int i = 0; i < cs.nfronts; ++i) {
    const FrontDesc& d = desc[i];
    for (int c = 0; c < d.nkids; ++c) {
      const FrontDesc& kd = desc[kids[d.kid_off + c]];
      for (int a = 0; a < kd.nB; ++a) {
        int2& slot = ctb[d.ctb_off + cmap[kd.cmap_off + a]];
        const int src = (int)(kd.uv_off + a);
        if (c == 0) slot.x = src;
        else if (c == 1) slot.y = src;
        else { set_error("nested dissection: more than two children"); return HELM_EINVAL; }
      }
    }
  }
  // per-level augmented work offsets and fronts by elimination path
  long long aug_max = 0;
  bigs.assign(cs.nlevels, {});
  smalls.assign(cs.nlevels, {});
  for (int h = 0; h < cs.nlevels; ++h) {
    long long off = 0;
    for (int f : cs.level_fronts[h]) {
      desc[f].aug_off = off;
      const int nS = desc[f].nS, nF = nS + desc[f].nB;
      off += (long long)nF * (nF + nS);
      (nS >= kBigFront ? bigs[h] : smalls[h]).push_back(f);
    }
    aug_max = std::max(aug_max, off);
  }
  // solve jobs: forward by height from the leaves, then backward from the root.  Rows per
  // job are sized so that a level has about kJobsPerBlockLevel jobs per resident block,
  // and are a whole number of stages.
  const long long target = (long long)kJobsPerBlockLevel * cs.grid;
  auto job_rows = [&](long long level_rows, int srows) {
    const long long want = std::max<long long>(srows, (level_rows + target - 1) / target);
    const long long cap = (long long)(kJobRows / srows) * srows;
    return (int)std::min(cap, (want + srows - 1) / srows * srows);
  };
  jobs.clear();
  int slot = 0;
  long long pbase = 0;
  // column tiles of a front matrix with `nrows` rows and `ncols` columns, row chunks of
  // each; rows are split beyond kJobRows only where the level has too few tiles to keep
  // every resident block busy
  auto add_tiles = [&](int f, int kind, int nrows, int ncols, long long level_rows, bool split) {
    for (int c0 = 0; c0 < ncols; c0 += kTile) {
      const int cols = std::min(kTile, ncols - c0);
      if (nrows == 0) {   // the root's backward: x_S = w_S
        jobs.push_back(SweepJob{f, kind, 0, 0, c0, c0 + cols, 0, 1, 0, -1, 0});
        continue;
      }
      const int srows = std::min(kJobRows, std::max(1, kStageEntries / cols));
      const int jr = split ? job_rows(level_rows, srows) : (kJobRows / srows) * srows;
      const int nch = (nrows + jr - 1) / jr;
      for (int ch = 0; ch < nch; ++ch)
        jobs.push_back(SweepJob{f, kind, ch * jr, std::min(nrows, (ch + 1) * jr), c0, c0 + cols, srows, nch, ch,
                                nch > 1 ? slot : -1, nch > 1 ? (int)pbase : 0});
      if (nch > 1) {
        ++slot;
        pbase += nch;
      }
    }
  };
  for (int h = 0; h < cs.nlevels; ++h) {   // forward: M [nS][nF]
    long long level_rows = 0, tiles = 0;
    for (int f : cs.level_fronts[h]) {
      const int t = (desc[f].nS + desc[f].nB + kTile - 1) / kTile;
      level_rows += (long long)t * desc[f].nS;
      tiles += t;
    }
    for (int f : cs.level_fronts[h]) {
      desc[f].fwd_units = (desc[f].nS + desc[f].nB + kTile - 1) / kTile;
      add_tiles(f, 0, desc[f].nS, desc[f].nS + desc[f].nB, level_rows, tiles < 2LL * grid);
    }
  }
  for (int h = cs.nlevels - 1; h >= 0; --h) {   // backward: G^T [nB][nS]
    long long level_rows = 0, tiles = 0;
    for (int f : cs.level_fronts[h]) {
      const int t = (desc[f].nS + kTile - 1) / kTile;
      level_rows += (long long)t * desc[f].nB;
      tiles += t;
    }
    for (int f : cs.level_fronts[h]) {
      desc[f].bwd_units = (desc[f].nS + kTile - 1) / kTile;
      add_tiles(f, 1, desc[f].nB, desc[f].nS, level_rows, tiles < 2LL * grid);
    }
  }
  cs.njobs = (int)jobs.size();
  cs.n_slots = slot;
  cs.part_blocks = std::max<long long>(1, pbase);
  cs.n_counters = 2LL * cs.nfronts + slot;
  P.aug_max = aug_max;
  P.upool = uoff;
  if (int st = validate_plan(cs, P)) return st;
  // the kernel's job records; counters: forward completions [0, nfronts), backward
  // completions [nfronts, 2 nfronts), chunk slots after them
  P.meta.assign(jobs.size(), SweepMeta{});
  for (size_t j = 0; j < jobs.size(); ++j) {
    const SweepJob& J = jobs[j];
    const FrontDesc& d = desc[J.front];
    SweepMeta& m = P.meta[j];
    m.kind = J.kind;
    m.r0 = J.r0;
    m.r1 = J.r1;
    m.c0 = J.c0;
    m.c1 = J.c1;
    m.srows = J.srows;
    m.nchunks = J.nchunks;
    m.chunk = J.chunk;
    m.slot = J.nchunks > 1 ? 2 * cs.nfronts + J.slot : -1;
    m.pbase = J.pbase;
    m.nS = d.nS;
    m.nB = d.nB;
    m.S_off = d.S_off;
    m.B_off = d.B_off;
    m.bsign = d.bsign;
    m.front = J.front;
    m.ld = J.kind == 0 ? d.nS + d.nB : d.g_ld;
    m.src = (J.kind == 0 ? d.M_off : d.G_off) + (long long)J.r0 * m.ld + J.c0;
    m.ctb_off = d.ctb_off;
    m.uv_off = d.uv_off;
    m.done = J.kind == 0 ? J.front : cs.nfronts + J.front;
    if (J.kind == 0) {
      if (d.nkids > 2) {
        set_error("coarsest solve plan: a front with more than two children");
        return HELM_EINVAL;
      }
      m.nwait = d.nkids;
      for (int q = 0; q < d.nkids; ++q) {
        const int k = P.kids[d.kid_off + q];
        m.wait[q] = k;
        m.target[q] = desc[k].fwd_units;
      }
    } else if (d.parent < 0) {
      m.nwait = 1;
      m.wait[0] = J.front;
      m.target[0] = d.fwd_units;
    } else {
      m.nwait = 1;
      m.wait[0] = cs.nfronts + d.parent;
      m.target[0] = desc[d.parent].bwd_units;
    }
  }
  return 0;
}

int coarse_plan_stats(const GridDims& g, int r, int leaf_max, bool symmetric, int grid, long long stats[8]) {
  CoarseSolver cs;
  CoarsePlan P;
  if (int st = coarse_plan(cs, P, g, r, leaf_max, symmetric, grid)) return st;
  stats[0] = cs.nfronts;
  stats[1] = cs.nlevels;
  stats[2] = cs.njobs;
  stats[3] = cs.factor_entries;
  stats[4] = cs.bwd_entries;
  stats[5] = cs.part_blocks;
  stats[6] = cs.n_slots;
  stats[7] = cs.max_nB;
  return 0;
}

int coarse_setup(CoarseSolver& cs, const GridDims& g, int r, const double2* coef, int leaf_max,
                 bool symmetric, bool df, cudaStream_t s, int blocks, int huge_min) {
  HELM_CUDA_TRY(cudaGetDevice(&cs.device));
  int grid = 0, grid_group = 0;
  if (int st = sweep_grid_size(&grid, &grid_group)) return st;
  CoarsePlan P;
  if (int st = coarse_plan(cs, P, g, r, leaf_max, symmetric, grid)) return st;
  cs.grid_group = grid_group;
  // a share of the device, e.g. for solves running side by side: the job list stays the
  // one planned for the whole device (and with it every summation order), only fewer
  // blocks run it
  if (blocks > 0) {
    cs.grid = std::min(cs.grid, blocks);
    cs.grid_group = std::min(cs.grid_group, blocks);
  }
  cs.df = df;
  const auto& desc = P.desc;
  const auto& bigs = P.bigs;
  const auto& smalls = P.smalls;
  const long long aug_max = P.aug_max, uoff = P.upool;
  cs.d_level_list.resize(cs.nlevels);
  cs.big_list.resize(cs.nlevels);
  cs.small_list.resize(cs.nlevels);
  if (upload(&cs.d_desc, desc) || upload(&cs.d_S, P.Sall) || upload(&cs.d_B, P.Ball) ||
      upload(&cs.d_kids, P.kids) || upload(&cs.d_cmap, P.cmap) || upload(&cs.d_ctb, P.ctb))
    return HELM_ECUDA;
  int2* d_ents = nullptr;
  if (upload(&d_ents, P.ents)) return HELM_ECUDA;
  if (upload(&cs.d_meta, P.meta)) return HELM_ECUDA;
  for (int h = 0; h < cs.nlevels; ++h) {
    if (upload(&cs.d_level_list[h], cs.level_fronts[h]) || upload(&cs.big_list[h], bigs[h]) ||
        upload(&cs.small_list[h], smalls[h]))
      return HELM_ECUDA;
  }
  HELM_CUDA_TRY(cudaMalloc(&cs.d_factors, std::max<long long>(1, cs.factor_entries) * sizeof(double2)));
  HELM_CUDA_TRY(cudaMalloc(&cs.d_err, sizeof(int)));
  HELM_CUDA_TRY(cudaMemsetAsync(cs.d_err, 0, sizeof(int), s));
  double2 *d_aug = nullptr, *d_upool = nullptr, *d_akk = nullptr;
  int* d_piv = nullptr;
  size_t maxbig = 1;
  for (auto& v : bigs) maxbig = std::max(maxbig, v.size());
  HELM_CUDA_TRY(cudaMalloc(&d_aug, std::max<long long>(1, aug_max) * sizeof(double2)));
  HELM_CUDA_TRY(cudaMalloc(&d_upool, std::max<long long>(1, uoff) * sizeof(double2)));
  HELM_CUDA_TRY(cudaMalloc(&d_piv, maxbig * sizeof(int)));
  HELM_CUDA_TRY(cudaMalloc(&d_akk, maxbig * sizeof(double2)));
  // fronts with at least huge_min eliminated nodes: blocked elimination (coarse_blocked.cu)
  int max_huge_S = 0;
  long long max_huge_ld = 0;
  std::vector<std::vector<int>> normal(cs.nlevels), big_normal(cs.nlevels), huge(cs.nlevels);
  for (int h = 0; h < cs.nlevels; ++h) {
    for (int f : cs.level_fronts[h]) (desc[f].nS >= huge_min ? huge[h] : normal[h]).push_back(f);
    for (int f : bigs[h])
      if (desc[f].nS < huge_min) big_normal[h].push_back(f);
    for (int f : huge[h]) {
      max_huge_S = std::max(max_huge_S, desc[f].nS);
      max_huge_ld = std::max<long long>(max_huge_ld, 2LL * desc[f].nS + desc[f].nB);
    }
  }
  float2* d_w32 = nullptr;
  double2 *d_dinv = nullptr, *d_xbuf = nullptr;
  int* d_hpiv = nullptr;
  if (max_huge_S > 0) {
    HELM_CUDA_TRY(cudaMalloc(&d_w32, (size_t)max_huge_S * 64 * sizeof(float2)));
    HELM_CUDA_TRY(cudaMalloc(&d_dinv, (size_t)64 * 64 * sizeof(double2)));
    HELM_CUDA_TRY(cudaMalloc(&d_xbuf, (size_t)64 * max_huge_ld * sizeof(double2)));
    HELM_CUDA_TRY(cudaMalloc(&d_hpiv, 64 * sizeof(int)));
  }
  auto free_setup = [&]() {
    cudaFree(d_aug);
    cudaFree(d_upool);
    cudaFree(d_ents);
    cudaFree(d_piv);
    cudaFree(d_akk);
    cudaFree(d_w32);
    cudaFree(d_dinv);
    cudaFree(d_xbuf);
    cudaFree(d_hpiv);
  };
  {
    KernelTimer kt(HELM_K_SETUP, s);
    for (int h = 0; h < cs.nlevels; ++h) {
      int* d_normal = nullptr;
      int* d_bign = nullptr;
      if (upload(&d_normal, normal[h]) || upload(&d_bign, big_normal[h])) { free_setup(); return HELM_ECUDA; }
      auto fail_level = [&](int st) { cudaFree(d_normal); cudaFree(d_bign); free_setup(); return st; };
      if (!normal[h].empty()) {
        fact_assemble_kernel<<<(int)normal[h].size(), 256, 0, s>>>(cs.d_desc, d_normal, d_aug, d_ents, coef, d_upool,
                                                                   cs.d_kids, cs.d_cmap);
        if (cudaGetLastError() != cudaSuccess) return fail_level(HELM_ECUDA);
        count_launch();
      }
      for (int f : huge[h])
        if (int st = big_front_assemble(desc[f], desc, P.kids, d_aug, d_ents, coef, d_upool, cs.d_cmap, s))
          return fail_level(st);
      if (!smalls[h].empty()) {
        fact_gj_kernel<<<(int)smalls[h].size(), 512, 0, s>>>(cs.d_desc, cs.small_list[h], d_aug, cs.d_err);
        if (cudaGetLastError() != cudaSuccess) return fail_level(HELM_ECUDA);
        count_launch();
      }
      if (!big_normal[h].empty()) {
        int maxS = 0, maxF = 0, maxLd = 0;
        for (int f : big_normal[h]) {
          maxS = std::max(maxS, desc[f].nS);
          maxF = std::max(maxF, desc[f].nS + desc[f].nB);
          maxLd = std::max(maxLd, 2 * desc[f].nS + desc[f].nB);
        }
        const dim3 gp((maxLd + 2047) / 2048, (unsigned)big_normal[h].size());
        const dim3 ge((maxF + 7) / 8, (unsigned)big_normal[h].size());
        for (int k = 0; k < maxS; ++k) {
          gj_pivot_kernel<<<gp, 256, 0, s>>>(cs.d_desc, d_bign, d_aug, k, d_piv, d_akk, cs.d_err);
          gj_elim_kernel<<<ge, 256, 0, s>>>(cs.d_desc, d_bign, d_aug, k, d_piv, d_akk);
          if (cudaGetLastError() != cudaSuccess) return fail_level(HELM_ECUDA);
          count_launch();
          count_launch();
        }
      }
      for (int f : huge[h])
        if (int st = big_front_eliminate(desc[f], d_aug, d_w32, d_hpiv, d_dinv, d_xbuf, cs.d_err, s)) return fail_level(st);
      if (!normal[h].empty()) {
        fact_extract_kernel<<<(int)normal[h].size(), 256, 0, s>>>(cs.d_desc, d_normal, d_aug, cs.d_factors, d_upool, df);
        if (cudaGetLastError() != cudaSuccess) return fail_level(HELM_ECUDA);
        count_launch();
      }
      for (int f : huge[h])
        if (int st = big_front_extract(desc[f], d_aug, cs.d_factors, d_upool, df, s)) return fail_level(st);
      // the level's device lists are read by kernels still queued: free them after the stream
      if (cudaStreamSynchronize(s) != cudaSuccess) return fail_level(HELM_ECUDA);
      cudaFree(d_normal);
      cudaFree(d_bign);
    }
  }
  HELM_CUDA_TRY(cudaStreamSynchronize(s));
  free_setup();
  int herr = 0;
  HELM_CUDA_TRY(cudaMemcpy(&herr, cs.d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (herr) { set_error("coarsest factorisation: zero or non-finite pivot"); return HELM_ENUMERIC; }
  return 0;
}

static int ensure_rhs(CoarseSolver& cs, int nrhs) {
  if (nrhs <= cs.rhs_cap) return 0;
  cudaFree(cs.d_uv);
  cudaFree(cs.d_w);
  cudaFree(cs.d_part);
  cudaFree(cs.d_counters);
  cudaFree(cs.d_xd);
  cs.d_uv = cs.d_w = cs.d_part = nullptr;
  cs.d_counters = nullptr;
  cs.d_xd = nullptr;
  cs.rhs_cap = 0;
  HELM_CUDA_TRY(cudaMalloc(&cs.d_xd, cs.g.size * nrhs * sizeof(float4)));
  HELM_CUDA_TRY(cudaMalloc(&cs.d_uv, std::max<long long>(1, cs.uv_total) * nrhs * sizeof(double2)));
  HELM_CUDA_TRY(cudaMalloc(&cs.d_w, cs.g.size * nrhs * sizeof(double2)));
  HELM_CUDA_TRY(cudaMalloc(&cs.d_part, cs.part_blocks * kPartBlock * nrhs * sizeof(double2)));
  HELM_CUDA_TRY(cudaMalloc(&cs.d_counters, std::max<long long>(1, cs.n_counters) * sizeof(unsigned)));
  cs.rhs_cap = nrhs;
  return 0;
}

int coarse_solve(CoarseSolver& cs, const double2* b, double2* e, int nrhs, cudaStream_t s) {
  if (int st = ensure_rhs(cs, nrhs)) return st;
  KernelTimer kt(HELM_K_COARSE, s);
  return sweep_launch(cs, b, e, nrhs, cs.d_uv, cs.d_w, cs.d_part, cs.d_counters, cs.d_xd, s);
}

int coarse_plant_unreachable_wait(CoarseSolver& cs, long long wait_cycles, int job, cudaStream_t s) {
  if (wait_cycles < 1) {
    set_error("wait limit must be at least one cycle");
    return HELM_EINVAL;
  }
  if (job < -1 || job >= cs.njobs) {
    set_error("job index out of range");
    return HELM_EINVAL;
  }
  HELM_CUDA_TRY(cudaStreamSynchronize(s));
  std::vector<SweepMeta> meta(cs.njobs);
  HELM_CUDA_TRY(cudaMemcpy(meta.data(), cs.d_meta, cs.njobs * sizeof(SweepMeta), cudaMemcpyDeviceToHost));
  if (job == -1)
    for (int j = cs.njobs - 1; j >= 0 && job < 0; --j)
      if (meta[j].nwait > 0) job = j;
  if (job < 0 || meta[job].nwait < 1) {
    set_error("the chosen job has no dependency to wait for");
    return HELM_EINVAL;
  }
  // a completion count no solve reaches: each counter counts output units of one front
  meta[job].target[0] = 0x40000000;
  HELM_CUDA_TRY(cudaMemcpy(cs.d_meta + job, &meta[job], sizeof(SweepMeta), cudaMemcpyHostToDevice));
  cs.wait_cycles = wait_cycles;
  return 0;
}

int coarse_status(const CoarseSolver& cs, cudaStream_t s) {
  if (!cs.d_err) return 0;
  HELM_CUDA_TRY(cudaStreamSynchronize(s));
  int herr = 0;
  HELM_CUDA_TRY(cudaMemcpy(&herr, cs.d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (herr == kErrSweepWait) { set_error("coarsest solve: a front dependency did not complete in time"); return HELM_ECUDA; }
  if (herr == kErrSweepCopy) { set_error("coarsest solve: a factor copy did not complete in time"); return HELM_ECUDA; }
  if (herr) { set_error("coarsest solver in error state"); return HELM_ECUDA; }
  return 0;
}

// ------------------------------------------------------------------ allocation-free variant
// Scratch of coarse_solve_noalloc: the front vectors, update vectors and the forward
// result of every right-hand side, carved from one file-scope device array instead of
// buffers the context allocates.  Every device that loads the library holds it until
// the process exits.
constexpr long long kNoAllocScratchEntries = 1LL << 20;   // 1 Mi complex FP64 = 16 MiB
static __device__ __align__(256) double2 g_noalloc_scratch[kNoAllocScratchEntries];

namespace {
std::mutex g_noalloc_mu;
constexpr int kMaxDevices = 64;
double2* g_noalloc_addr[kMaxDevices] = {};
}  // namespace

int coarse_solve_noalloc(const CoarseSolver& cs, const double2* b, double2* e, int nrhs, cudaStream_t s) {
  const long long per_rhs = cs.uv_total + cs.g.size + cs.part_blocks * kPartBlock + cs.g.size;
  const long long counter_entries = (cs.n_counters * (long long)sizeof(unsigned) + sizeof(double2) - 1) / sizeof(double2);
  if (nrhs < 1 || per_rhs * nrhs + counter_entries > kNoAllocScratchEntries) {
    set_error("allocation-free coarsest solve needs " + std::to_string(per_rhs * nrhs + counter_entries) +
              " complex scratch entries; the static array holds " + std::to_string(kNoAllocScratchEntries));
    return HELM_EINVAL;
  }
  // the array's address is per device: look it up on the context's device, and refuse a
  // call made with another device current (its stream and buffers live on the context's)
  int dev = 0;
  HELM_CUDA_TRY(cudaGetDevice(&dev));
  if (dev != cs.device) {
    set_error("allocation-free coarsest solve: device " + std::to_string(dev) + " is current, the context was set up on " +
              std::to_string(cs.device));
    return HELM_EINVAL;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("device ordinal out of range for the allocation-free scratch table");
    return HELM_EINVAL;
  }
  double2* base = nullptr;
  {
    // set-up once per device, with that device current: the host-side symbol is a
    // stand-in, its device address comes from the runtime
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
      void* p = nullptr;
      HELM_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
      g_noalloc_addr[dev] = static_cast<double2*>(p);
    }
    base = g_noalloc_addr[dev];
  }
  // The completion counters must start at zero and are cleared by sweep_launch; every
  // other scratch entry that is read is written earlier in the same call (update vectors
  // and partial sums by the jobs that produce them, w and its double-float copy for every
  // eliminated node).
  unsigned* counters = reinterpret_cast<unsigned*>(base);
  double2* uv = base + counter_entries;
  double2* w = uv + cs.uv_total * nrhs;
  double2* part = w + cs.g.size * nrhs;
  float4* xd = reinterpret_cast<float4*>(part + cs.part_blocks * kPartBlock * nrhs);   // float4 and double2 are both 16 bytes
  return sweep_launch(cs, b, e, nrhs, uv, w, part, counters, xd, s);
}

void coarse_free(CoarseSolver& cs) {
  cudaFree(cs.d_desc);
  cudaFree(cs.d_S);
  cudaFree(cs.d_B);
  cudaFree(cs.d_kids);
  cudaFree(cs.d_cmap);
  cudaFree(cs.d_factors);
  cudaFree(cs.d_err);
  for (auto p : cs.d_level_list) cudaFree(p);
  cudaFree(cs.d_meta);
  for (auto p : cs.big_list) cudaFree(p);
  for (auto p : cs.small_list) cudaFree(p);
  cudaFree(cs.d_part);
  cudaFree(cs.d_counters);
  cudaFree(cs.d_ctb);
  cudaFree(cs.d_uv);
  cudaFree(cs.d_w);
  cudaFree(cs.d_xd);
  cs = CoarseSolver();
}

}  // namespace helm
