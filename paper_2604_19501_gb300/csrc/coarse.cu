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
// F_BS F_SS^-1 = (F_SS^-1 F_SB)^T; otherwise M = [F_SS^-1 | -F_BS F_SS^-1]^T plus
// G = F_SS^-1 F_SB.  Small fronts are eliminated by one thread block each; large fronts by
// a pair of grid-wide kernels per pivot (pivot search + row swap/scale, elimination).
//
// Solve: forward, leaves to root, every front turns its assembled right-hand side r_F
// into w_S = F_SS^-1 r_S and the update vector r_B - F_BS F_SS^-1 r_S for its parent:
// column sums over M, split into row chunks whose partial sums the last block of a column
// tile adds in chunk order.  Backward, root to leaves, x_S = w_S - (F_SS^-1 F_SB) x_B
// (row dot products).  The summation order is fixed, so results are reproducible bit
// for bit.
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
  if (d.bsign > 0) {
    double2* G = factors + d.G_off;
    for (long long t = threadIdx.x; t < (long long)nS * nB; t += blockDim.x) {
      const int row = (int)(t / nB), col = (int)(t % nB);
      store_factor(G, t, A[(long long)row * ld + nS + col], df);
    }
  }
  for (long long t = threadIdx.x; t < (long long)nB * nB; t += blockDim.x) {
    const int row = (int)(t / nB), col = (int)(t % nB);
    U[t] = A[(long long)(nS + row) * ld + nS + col];
  }
}

// ------------------------------------------------------------------ solve kernels
// Right-hand side of front position t: b at the eliminated nodes plus the entries of the
// children's update vectors that map to t (at most one per child), added in child order.
__device__ __forceinline__ double2 front_rhs(const FrontDesc& d, const int* __restrict__ Sidx,
                                             const int2* __restrict__ ctb, const double2* __restrict__ b,
                                             const double2* __restrict__ uv, int t, int r, long long nodes,
                                             long long uv_total) {
  double2 v = t < d.nS ? b[r * nodes + Sidx[d.S_off + t]] : make_double2(0.0, 0.0);
  const int2 c = ctb[d.ctb_off + t];
  if (c.x >= 0) {
    const double2 u = uv[r * uv_total + c.x];
    v.x += u.x;
    v.y += u.y;
  }
  if (c.y >= 0) {
    const double2 u = uv[r * uv_total + c.y];
    v.x += u.x;
    v.y += u.y;
  }
  return v;
}

// out_t < nS: w at node S[t]; t >= nS: the update vector r_B + bsign * out.
__device__ __forceinline__ void fwd_write(const FrontDesc& d, const int* __restrict__ Sidx,
                                          const int2* __restrict__ ctb, const double2* __restrict__ b, int t,
                                          int r, double2 v, double2* __restrict__ uv, double2* __restrict__ w,
                                          long long nodes, long long uv_total) {
  if (t < d.nS) {
    w[r * nodes + Sidx[d.S_off + t]] = v;
  } else {
    const double2 rb = front_rhs(d, Sidx, ctb, b, uv, t, r, nodes, uv_total);
    uv[r * uv_total + d.uv_off + t - d.nS] = make_double2(rb.x + d.bsign * v.x, rb.y + d.bsign * v.y);
  }
}

// Forward sweep of one level: out_t = sum_{s in [s0, s1)} M[s][t] r_S[s] for one column tile;
// r_S is assembled on the fly from b and the children's update vectors.  Fronts split
// into several row chunks leave partial sums that the last block of the tile adds in
// chunk order.
template <bool DF, int RG>
__global__ void __launch_bounds__(kFwdCols) fwd_colsum_kernel(
    const FrontDesc* __restrict__ desc, const FwdJob* __restrict__ jobs, const int* __restrict__ Sidx,
    const int2* __restrict__ ctb, const double2* __restrict__ factors, const double2* __restrict__ b,
    double2* __restrict__ uv, double2* __restrict__ w, double2* __restrict__ part,
    unsigned* __restrict__ counters, int nrhs, long long nodes, long long uv_total) {
  pdl_trigger();
  // job lists, fronts and factors are written at set-up: read before the wait
  const FwdJob job = jobs[blockIdx.x];
  const FrontDesc d = desc[job.front];
  const int nF = d.nS + d.nB;
  const int tid = threadIdx.x;
  const int t = job.tile * kFwdCols + tid;
  const int s0 = job.s0, s1 = job.s1, nrow = s1 - s0;
  // right-hand-side values of the chunk for a group of kRhsGroup right-hand sides
  __shared__ double2 rs[kFwdMaxChunk][RG];
  __shared__ float4 rsd[kFwdMaxChunk][RG];
  __shared__ bool s_last;
  pdl_wait();
  for (int r0 = 0; r0 < nrhs; r0 += RG) {
    const int nr = min(RG, nrhs - r0);
    for (int q = tid; q < nrow * nr; q += blockDim.x) {
      const int row = q / nr, rr = q % nr;
      const double2 v = front_rhs(d, Sidx, ctb, b, uv, s0 + row, r0 + rr, nodes, uv_total);
      if (DF) rsd[row][rr] = to_df(v);
      else rs[row][rr] = v;
    }
    __syncthreads();
    // every factor entry is loaded once and applied to the whole group
    double2 acc[RG];
    float4 a4[RG];
#pragma unroll
    for (int rr = 0; rr < RG; ++rr) {
      acc[rr] = make_double2(0.0, 0.0);
      a4[rr] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (t < nF) {
      if (DF) {
        const float4* col = reinterpret_cast<const float4*>(factors + d.M_off) + (long long)s0 * nF + t;
#pragma unroll 8
        for (int s = 0; s < nrow; ++s) {
          const float4 m = __ldcs(col + (long long)s * nF);
#pragma unroll
          for (int rr = 0; rr < RG; ++rr)
            if (RG == 1 || rr < nr) df_cmac(a4[rr], m, rsd[s][rr]);
        }
      } else {
        const double2* col = factors + d.M_off + (long long)s0 * nF + t;
#pragma unroll 8
        for (int s = 0; s < nrow; ++s) {
          const double2 m = __ldcs(col + (long long)s * nF);
#pragma unroll
          for (int rr = 0; rr < RG; ++rr)
            if (RG == 1 || rr < nr) acc[rr] = cmac(acc[rr], m, rs[s][rr]);
        }
      }
    }
#pragma unroll
    for (int rr = 0; rr < RG; ++rr) {
      if (rr >= nr) break;
      const int r = r0 + rr;
      if (job.nchunks == 1) {
        if (t < nF) fwd_write(d, Sidx, ctb, b, t, r, DF ? from_df(a4[rr]) : acc[rr], uv, w, nodes, uv_total);
      } else {
        const long long pi = ((long long)(job.pbase + job.chunk) * nrhs + r) * kFwdCols + tid;
        if (DF) reinterpret_cast<float4*>(part)[pi] = a4[rr];
        else part[pi] = acc[rr];
      }
    }
    __syncthreads();
  }
  if (job.nchunks == 1) return;
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = (atomicAdd(&counters[job.slot], 1u) == (unsigned)job.nchunks - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  for (int r = 0; r < nrhs; ++r) {
    double2 acc = make_double2(0.0, 0.0);
    float4 a4 = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int q = 0; q < job.nchunks; ++q) {
      const long long pi = ((long long)(job.pbase + q) * nrhs + r) * kFwdCols + tid;
      if (DF) {
        df_acc_add(a4, __ldcg(reinterpret_cast<const float4*>(part) + pi));
      } else {
        const double2 v = __ldcg(part + pi);
        acc.x += v.x;
        acc.y += v.y;
      }
    }
    if (t < nF) fwd_write(d, Sidx, ctb, b, t, r, DF ? from_df(a4) : acc, uv, w, nodes, uv_total);
  }
  if (tid == 0) counters[job.slot] = 0u;
}

// One warp per row of G: x_S[row] = w_S[row] - G[row, :] . x_B; a block handles a range
// of rows of one front for a group of kRhsGroup right-hand sides.  x_B of the group is
// first staged in shared memory (as double-float with DF) when it fits, so the row loops
// stream G once for the whole group.  With DF the factors are double-float and the sweep
// also writes the double-float copy xd of x.
template <bool DF, int RG>
__global__ void __launch_bounds__(512) bwd_matvec_kernel(const FrontDesc* __restrict__ desc,
                                                         const int4* __restrict__ rows,
                                                         const int* __restrict__ Sidx,
                                                         const int* __restrict__ Bidx,
                                                         const double2* __restrict__ factors,
                                                         const double2* __restrict__ w,
                                                         double2* __restrict__ x, float4* __restrict__ xd,
                                                         int nrhs, long long nodes, int smem_cap) {
  extern __shared__ float4 xs[];
  pdl_trigger();
  const int4 job = rows[blockIdx.x];
  const FrontDesc d = desc[job.x];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int* B = Bidx + d.B_off;
  pdl_wait();
  for (int r0 = 0; r0 < nrhs; r0 += RG) {
    const int nr = min(RG, nrhs - r0);
    const bool staged = d.nB * nr <= smem_cap;
    if (staged) {
      for (int q = threadIdx.x; q < d.nB * nr; q += blockDim.x) {
        const int rr = q / d.nB, c = q % d.nB;
        const long long gi = (r0 + rr) * nodes + B[c];
        if (DF) xs[rr * d.nB + c] = xd[gi];
        else reinterpret_cast<double2*>(xs)[rr * d.nB + c] = x[gi];
      }
      __syncthreads();
    }
    for (int row = job.y + warp; row < job.z; row += nwarp) {
      const int node = Sidx[d.S_off + row];
      double2 acc[RG];
      float4 a4[RG];
#pragma unroll
      for (int rr = 0; rr < RG; ++rr) {
        acc[rr] = make_double2(0.0, 0.0);
        a4[rr] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      if (DF) {
        const float4* G = reinterpret_cast<const float4*>(factors + d.G_off) + (long long)row * d.g_ld;
#pragma unroll 4
        for (int c = lane; c < d.nB; c += 32) {
          const float4 g = __ldcs(G + c);
#pragma unroll
          for (int rr = 0; rr < RG; ++rr)
            if (RG == 1 || rr < nr) df_cmac(a4[rr], g, staged ? xs[rr * d.nB + c] : xd[(r0 + rr) * nodes + B[c]]);
        }
      } else {
        const double2* G = factors + d.G_off + (long long)row * d.g_ld;
        const double2* xs2 = reinterpret_cast<const double2*>(xs);
#pragma unroll 4
        for (int c = lane; c < d.nB; c += 32) {
          const double2 g = __ldcs(G + c);
#pragma unroll
          for (int rr = 0; rr < RG; ++rr)
            if (RG == 1 || rr < nr) acc[rr] = cmac(acc[rr], g, staged ? xs2[rr * d.nB + c] : x[(r0 + rr) * nodes + B[c]]);
        }
      }
#pragma unroll
      for (int rr = 0; rr < RG; ++rr) {
        if (rr >= nr) break;
        double2 v;
        if (DF) {
          const float4 sum = df_warp_sum(a4[rr]);
          v = from_df(sum);
        } else {
          v = acc[rr];
          for (int off = 16; off > 0; off >>= 1) {
            v.x += __shfl_down_sync(0xffffffffu, v.x, off);
            v.y += __shfl_down_sync(0xffffffffu, v.y, off);
          }
        }
        if (lane == 0) {
          const long long gi = (r0 + rr) * nodes + node;
          const double2 wv = w[gi];
          const double2 xv = make_double2(wv.x - v.x, wv.y - v.y);
          x[gi] = xv;
          if (DF) xd[gi] = to_df(xv);
        }
      }
    }
    if (staged) __syncthreads();
  }
}

template <typename T>
int upload(T** dst, const std::vector<T>& v) {
  if (v.empty()) { *dst = nullptr; return 0; }
  HELM_CUDA_TRY(cudaMalloc(dst, v.size() * sizeof(T)));
  HELM_CUDA_TRY(cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return 0;
}

constexpr int kRowsPerBlock = 16;  // warps per block in the backward sweep (minimum rows per block)
constexpr int kTargetBlocks = 1024;   // blocks per tree level the sweeps aim for
constexpr int kBwdSmemEntries = 6144;   // x_B entries staged in shared memory (96 KiB)
constexpr int kBigFront = 96;      // fronts with at least this many eliminated nodes use the grid-wide elimination

}  // namespace

int coarse_setup(CoarseSolver& cs, const GridDims& g, int r, const double2* coef, int leaf_max,
                 bool symmetric, bool df, cudaStream_t s) {
  cs.g = g;
  cs.r = r;
  cs.df = df;
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
  std::vector<FrontDesc> desc(cs.nfronts);
  std::vector<int> Sall, Ball, kids, cmap;
  std::vector<int2> ents;
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
    if (symmetric) {
      d.G_off = d.M_off + d.nS;
      d.g_ld = nF;
    } else {
      d.G_off = xg;
      d.g_ld = d.nB;
      xg += (long long)d.nS * d.nB;
    }
    d.U_off = uoff;
    uoff += (long long)d.nB * d.nB;
    d.ctb_off = rfo;
    rfo += nF;
    d.uv_off = uvo;
    uvo += d.nB;
    d.kid_off = (int)kids.size();
    d.nkids = (int)f.kids.size();
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
        if (it == pos.end()) { set_error("nested dissection: child boundary outside parent front"); return HELM_ECUDA; }
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
  std::vector<int2> ctb(rfo, make_int2(-1, -1));
  for (int i = 0; i < cs.nfronts; ++i) {
    const FrontDesc& d = desc[i];
    for (int c = 0; c < d.nkids; ++c) {
      const FrontDesc& kd = desc[kids[d.kid_off + c]];
      for (int a = 0; a < kd.nB; ++a) {
        int2& slot = ctb[d.ctb_off + cmap[kd.cmap_off + a]];
        const int src = (int)(kd.uv_off + a);
        if (c == 0) slot.x = src;
        else if (c == 1) slot.y = src;
        else { set_error("nested dissection: more than two children"); return HELM_ECUDA; }
      }
    }
  }
  // per-level augmented work offsets and solve job lists
  long long aug_max = 0;
  cs.d_level_list.resize(cs.nlevels);
  cs.d_fwd_jobs.resize(cs.nlevels);
  cs.d_bwd_rows.resize(cs.nlevels);
  cs.n_fwd_jobs.resize(cs.nlevels);
  cs.n_bwd_rows.resize(cs.nlevels);
  cs.big_list.resize(cs.nlevels);
  cs.small_list.resize(cs.nlevels);
  cs.part_entries = 1;
  cs.n_slots = 1;
  std::vector<std::vector<int>> bigs(cs.nlevels), smalls(cs.nlevels);
  std::vector<std::vector<FwdJob>> fjobs(cs.nlevels);
  std::vector<std::vector<int4>> brows(cs.nlevels);
  for (int h = 0; h < cs.nlevels; ++h) {
    long long off = 0;
    int slot = 0, pbase = 0;
    // row chunks and backward rows per block sized so that a level has about
    // kTargetBlocks blocks: small fronts are not split, large fronts are
    long long work = 0, rows_total = 0;
    for (int f : cs.level_fronts[h]) {
      work += (long long)((desc[f].nS + desc[f].nB + kFwdCols - 1) / kFwdCols) * desc[f].nS;
      rows_total += desc[f].nS;
    }
    int chunk_rows = (int)std::max<long long>(kFwdMinChunk, (work + kTargetBlocks - 1) / kTargetBlocks);
    chunk_rows = std::min(kFwdMaxChunk, (chunk_rows + kFwdMinChunk - 1) / kFwdMinChunk * kFwdMinChunk);
    const int bwd_rows = (int)std::max<long long>(kRowsPerBlock, (rows_total + kTargetBlocks - 1) / kTargetBlocks);
    for (int f : cs.level_fronts[h]) {
      desc[f].aug_off = off;
      const int nS = desc[f].nS, nF = nS + desc[f].nB;
      off += (long long)nF * (nF + nS);
      (nS >= kBigFront ? bigs[h] : smalls[h]).push_back(f);
      const int tiles = (nF + kFwdCols - 1) / kFwdCols;
      const int chunks = (nS + chunk_rows - 1) / chunk_rows;
      for (int tl = 0; tl < tiles; ++tl) {
        for (int ch = 0; ch < chunks; ++ch)
          fjobs[h].push_back(FwdJob{f, tl, ch * chunk_rows, std::min(nS, (ch + 1) * chunk_rows), chunks, ch,
                                    slot, pbase});
        if (chunks > 1) {
          pbase += chunks;
          ++slot;
        }
      }
      for (int r0 = 0; r0 < nS; r0 += bwd_rows) brows[h].push_back(make_int4(f, r0, std::min(nS, r0 + bwd_rows), 0));
    }
    aug_max = std::max(aug_max, off);
    cs.part_entries = std::max<long long>(cs.part_entries, (long long)pbase * kFwdCols);
    cs.n_slots = std::max(cs.n_slots, slot);
    cs.n_fwd_jobs[h] = (int)fjobs[h].size();
    cs.n_bwd_rows[h] = (int)brows[h].size();
  }
  if (upload(&cs.d_desc, desc) || upload(&cs.d_S, Sall) || upload(&cs.d_B, Ball) ||
      upload(&cs.d_kids, kids) || upload(&cs.d_cmap, cmap) || upload(&cs.d_ctb, ctb))
    return HELM_ECUDA;
  int2* d_ents = nullptr;
  if (upload(&d_ents, ents)) return HELM_ECUDA;
  for (int h = 0; h < cs.nlevels; ++h) {
    if (upload(&cs.d_level_list[h], cs.level_fronts[h]) || upload(&cs.d_fwd_jobs[h], fjobs[h]) ||
        upload(&cs.d_bwd_rows[h], brows[h]) || upload(&cs.big_list[h], bigs[h]) ||
        upload(&cs.small_list[h], smalls[h]))
      return HELM_ECUDA;
  }
  HELM_CUDA_TRY(cudaMalloc(&cs.d_factors, std::max<long long>(1, xg) * sizeof(double2)));
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
  {
    KernelTimer kt(HELM_K_SETUP, s);
    for (int h = 0; h < cs.nlevels; ++h) {
      const int nf = (int)cs.level_fronts[h].size();
      fact_assemble_kernel<<<nf, 256, 0, s>>>(cs.d_desc, cs.d_level_list[h], d_aug, d_ents, coef, d_upool,
                                              cs.d_kids, cs.d_cmap);
      HELM_LAUNCH_CHECK();
      if (!smalls[h].empty()) {
        fact_gj_kernel<<<(int)smalls[h].size(), 512, 0, s>>>(cs.d_desc, cs.small_list[h], d_aug, cs.d_err);
        HELM_LAUNCH_CHECK();
      }
      if (!bigs[h].empty()) {
        int maxS = 0, maxF = 0, maxLd = 0;
        for (int f : bigs[h]) {
          maxS = std::max(maxS, desc[f].nS);
          maxF = std::max(maxF, desc[f].nS + desc[f].nB);
          maxLd = std::max(maxLd, 2 * desc[f].nS + desc[f].nB);
        }
        const dim3 gp((maxLd + 2047) / 2048, (unsigned)bigs[h].size());
        const dim3 ge((maxF + 7) / 8, (unsigned)bigs[h].size());
        for (int k = 0; k < maxS; ++k) {
          gj_pivot_kernel<<<gp, 256, 0, s>>>(cs.d_desc, cs.big_list[h], d_aug, k, d_piv, d_akk, cs.d_err);
          HELM_LAUNCH_CHECK();
          gj_elim_kernel<<<ge, 256, 0, s>>>(cs.d_desc, cs.big_list[h], d_aug, k, d_piv, d_akk);
          HELM_LAUNCH_CHECK();
        }
      }
      fact_extract_kernel<<<nf, 256, 0, s>>>(cs.d_desc, cs.d_level_list[h], d_aug, cs.d_factors, d_upool, df);
      HELM_LAUNCH_CHECK();
    }
  }
  HELM_CUDA_TRY(cudaStreamSynchronize(s));
  cudaFree(d_aug);
  cudaFree(d_upool);
  cudaFree(d_ents);
  cudaFree(d_piv);
  cudaFree(d_akk);
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
  HELM_CUDA_TRY(cudaMalloc(&cs.d_xd, cs.g.size * nrhs * sizeof(float4)));
  HELM_CUDA_TRY(cudaMalloc(&cs.d_uv, std::max<long long>(1, cs.uv_total) * nrhs * sizeof(double2)));
  HELM_CUDA_TRY(cudaMalloc(&cs.d_w, cs.g.size * nrhs * sizeof(double2)));
  HELM_CUDA_TRY(cudaMalloc(&cs.d_part, cs.part_entries * nrhs * sizeof(double2)));
  HELM_CUDA_TRY(cudaMalloc(&cs.d_counters, cs.n_slots * sizeof(unsigned)));
  HELM_CUDA_TRY(cudaMemset(cs.d_counters, 0, cs.n_slots * sizeof(unsigned)));
  cs.rhs_cap = nrhs;
  return 0;
}

static int solve_sweeps(const CoarseSolver& cs, const double2* b, double2* e, int nrhs, double2* uv,
                        double2* w, double2* part, unsigned* counters, float4* xd, cudaStream_t s) {
  static bool attr_set = false;
  if (!attr_set) {
    const int bytes = kBwdSmemEntries * (int)sizeof(float4);
    cudaFuncSetAttribute(bwd_matvec_kernel<true, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    cudaFuncSetAttribute(bwd_matvec_kernel<false, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    cudaFuncSetAttribute(bwd_matvec_kernel<true, kRhsGroup>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    cudaFuncSetAttribute(bwd_matvec_kernel<false, kRhsGroup>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    attr_set = true;
  }
  for (int h = 0; h < cs.nlevels; ++h) {
    auto fk = nrhs == 1 ? (cs.df ? fwd_colsum_kernel<true, 1> : fwd_colsum_kernel<false, 1>)
                        : (cs.df ? fwd_colsum_kernel<true, kRhsGroup> : fwd_colsum_kernel<false, kRhsGroup>);
    const cudaError_t le = launch_pdl(fk,
                                      dim3(cs.n_fwd_jobs[h]), dim3(kFwdCols), 0, s, cs.d_desc, cs.d_fwd_jobs[h],
                                      cs.d_S, cs.d_ctb, cs.d_factors, b, uv, w, part, counters, nrhs, cs.g.size,
                                      cs.uv_total);
    if (le != cudaSuccess) { set_error(std::string("coarse forward launch: ") + cudaGetErrorString(le)); return HELM_ECUDA; }
    HELM_LAUNCH_CHECK();
  }
  for (int h = cs.nlevels - 1; h >= 0; --h) {
    const size_t sm = (size_t)std::min((long long)cs.max_nB * std::min(nrhs, kRhsGroup), (long long)kBwdSmemEntries) *
                      sizeof(float4);
    auto bk = nrhs == 1 ? (cs.df ? bwd_matvec_kernel<true, 1> : bwd_matvec_kernel<false, 1>)
                        : (cs.df ? bwd_matvec_kernel<true, kRhsGroup> : bwd_matvec_kernel<false, kRhsGroup>);
    const cudaError_t le = launch_pdl(bk,
                                      dim3(cs.n_bwd_rows[h]), dim3(32 * kRowsPerBlock), sm, s, cs.d_desc,
                                      cs.d_bwd_rows[h], cs.d_S, cs.d_B, cs.d_factors, w, e, xd, nrhs, cs.g.size,
                                      kBwdSmemEntries);
    if (le != cudaSuccess) { set_error(std::string("coarse backward launch: ") + cudaGetErrorString(le)); return HELM_ECUDA; }
    HELM_LAUNCH_CHECK();
  }
  return 0;
}

int coarse_solve(CoarseSolver& cs, const double2* b, double2* e, int nrhs, cudaStream_t s) {
  if (int st = ensure_rhs(cs, nrhs)) return st;
  KernelTimer kt(HELM_K_COARSE, s);
  return solve_sweeps(cs, b, e, nrhs, cs.d_uv, cs.d_w, cs.d_part, cs.d_counters, cs.d_xd, s);
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
  const long long per_rhs = cs.uv_total + cs.g.size + cs.part_entries + cs.g.size;
  const long long counter_entries = (cs.n_slots * (long long)sizeof(unsigned) + sizeof(double2) - 1) / sizeof(double2);
  if (nrhs < 1 || per_rhs * nrhs + counter_entries > kNoAllocScratchEntries) {
    set_error("allocation-free coarsest solve needs " + std::to_string(per_rhs * nrhs + counter_entries) +
              " complex scratch entries; the static array holds " + std::to_string(kNoAllocScratchEntries));
    return HELM_EINVAL;
  }
  int dev = 0;
  HELM_CUDA_TRY(cudaGetDevice(&dev));
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
  // The column-tile counters must start at zero and are cleared here; every other
  // scratch entry that is read is written earlier in the same call (update vectors and
  // partial sums by the kernels that produce them, w and its double-float copy for
  // every eliminated node).
  unsigned* counters = reinterpret_cast<unsigned*>(base);
  HELM_CUDA_TRY(cudaMemsetAsync(counters, 0, cs.n_slots * sizeof(unsigned), s));
  double2* uv = base + counter_entries;
  double2* w = uv + cs.uv_total * nrhs;
  double2* part = w + cs.g.size * nrhs;
  float4* xd = reinterpret_cast<float4*>(part + cs.part_entries * nrhs);   // float4 and double2 are both 16 bytes
  return solve_sweeps(cs, b, e, nrhs, uv, w, part, counters, xd, s);
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
  for (auto p : cs.d_fwd_jobs) cudaFree(p);
  for (auto p : cs.d_bwd_rows) cudaFree(p);
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
