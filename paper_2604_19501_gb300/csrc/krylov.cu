// Flexible GMRES machinery on the device (Sec. 5: FGMRES with the RS-CGC cycle as
// preconditioner, stopping at a relative residual of 1e-6), in complex FP64.
//
// One Arnoldi step j, after z_j = M^-1 v_j:
//   arnoldi_matvec   w = H z_j and the first classical Gram-Schmidt pass h1 = V^H w
//   arnoldi_update   w' = w - V h1 (not stored) and the second pass h2 = V^H w', ||w'||^2
//   arnoldi_small    H(:, j) = h1 + h2, ||w' - V h2||, Givens rotations, residual estimate
//   arnoldi_normalize v_{j+1} = (w - V (h1 + h2)) / ||w' - V h2||
// (classical Gram-Schmidt with one re-orthogonalisation, CGS2).  In the mixed precision
// the step can instead take one double-float pass (arnoldi_cgs_df_t: matvec, h = V^H w and
// ||w||^2 in one kernel; helm_opts.arnoldi_passes = 1).  Every reduction keeps
// per-thread partial sums in shared memory over a fixed grid, reduces each block once and
// lets the last block sum the block partials in block order, so the result does not
// depend on scheduling.
#include "krylov.cuh"
#include "fineop.cuh"
#include "timer.cuh"

namespace helm {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double2 warp_sum2(double2 v) {
  for (int off = 16; off > 0; off >>= 1) {
    v.x += __shfl_down_sync(0xffffffffu, v.x, off);
    v.y += __shfl_down_sync(0xffffffffu, v.y, off);
  }
  return v;
}

// sacc[i * blockDim + tid] holds per-thread partials of nval sums.  Reduces the block,
// then the last block to finish reduces all blocks into out[0..nval).
__device__ void reduce_finish(double2* sacc, int nval, double2* __restrict__ part,
                              unsigned* __restrict__ counter, double2* __restrict__ out) {
  __shared__ bool s_last;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  __syncthreads();
  for (int i = warp; i < nval; i += nwarp) {
    double2 v = make_double2(0.0, 0.0);
    for (int t = lane; t < (int)blockDim.x; t += 32) {
      const double2 a = sacc[i * blockDim.x + t];
      v.x += a.x;
      v.y += a.y;
    }
    v = warp_sum2(v);
    if (lane == 0) part[(long long)blockIdx.x * nval + i] = v;
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  for (int i = warp; i < nval; i += nwarp) {
    double2 v = make_double2(0.0, 0.0);
    for (int b = lane; b < (int)gridDim.x; b += 32) {
      const double2 a = __ldcg(part + (long long)b * nval + i);
      v.x += a.x;
      v.y += a.y;
    }
    v = warp_sum2(v);
    if (lane == 0) out[i] = v;
  }
  if (tid == 0) *counter = 0u;
}

// w = H z (FP64 arithmetic; z stored as c128 or c64), h1_i = v_i^H w (i < nv), ||w||^2.
template <typename TZ>
__global__ void __launch_bounds__(kThreads) arnoldi_matvec_kernel(
    FineOp op, const double* __restrict__ kap, const c2<TZ>* __restrict__ z, double2* __restrict__ w,
    const double2* __restrict__ V, long long vstride, int nv, double2* __restrict__ part,
    unsigned* __restrict__ counter, double2* __restrict__ out) {
  extern __shared__ double2 sacc[];
  const int tid = threadIdx.x;
  for (int i = 0; i <= nv; ++i) sacc[i * blockDim.x + tid] = make_double2(0.0, 0.0);
  const long long n = op.g.size;
  for (long long p = blockIdx.x * (long long)blockDim.x + tid; p < n; p += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    node_coords(op.g, p, i, j, k);
    const double2 d = fine_diag<double>(op, kap, p, i, j, k);
    const double2 wv = fine_apply_at<double, TZ>(op, d, z, p, p, i, j, k, kap);
    w[p] = wv;
    for (int q = 0; q < nv; ++q) {
      double2& a = sacc[q * blockDim.x + tid];
      a = cmacc(a, V[q * vstride + p], wv);
    }
    sacc[nv * blockDim.x + tid].x += wv.x * wv.x + wv.y * wv.y;
  }
  reduce_finish(sacc, nv + 1, part, counter, out);
}

// w' = w - sum_i h1_i v_i (kept in registers); h2_i = v_i^H w'; ||w'||^2.
__global__ void __launch_bounds__(kThreads) arnoldi_update_kernel(
    long long n, double2* __restrict__ w, const double2* __restrict__ V, long long vstride, int nv,
    const double2* __restrict__ h1, double2* __restrict__ part, unsigned* __restrict__ counter,
    double2* __restrict__ out) {
  extern __shared__ double2 sacc[];
  __shared__ double2 sh[64];
  const int tid = threadIdx.x;
  for (int i = 0; i <= nv; ++i) sacc[i * blockDim.x + tid] = make_double2(0.0, 0.0);
  for (int i = tid; i < nv; i += blockDim.x) sh[i] = h1[i];
  __syncthreads();
  for (long long p = blockIdx.x * (long long)blockDim.x + tid; p < n; p += (long long)gridDim.x * blockDim.x) {
    double2 wv = w[p];
    for (int q = 0; q < nv; ++q) {
      const double2 v = V[q * vstride + p];
      const double2 h = sh[q];
      wv.x -= h.x * v.x - h.y * v.y;
      wv.y -= h.x * v.y + h.y * v.x;
    }
    for (int q = 0; q < nv; ++q) {
      double2& a = sacc[q * blockDim.x + tid];
      a = cmacc(a, V[q * vstride + p], wv);
    }
    sacc[nv * blockDim.x + tid].x += wv.x * wv.x + wv.y * wv.y;
  }
  reduce_finish(sacc, nv + 1, part, counter, out);
}

// v_out = (w - sum_i h_i v_i) * st->inv_hn with h = h1 + h2 (stored in h2 by the small step)
__global__ void __launch_bounds__(kThreads) arnoldi_normalize_kernel(
    long long n, const double2* __restrict__ w, const double2* __restrict__ V, long long vstride, int nv,
    const double2* __restrict__ h2, const double* __restrict__ inv_hn, double2* __restrict__ vout) {
  __shared__ double2 sh[64];
  for (int i = threadIdx.x; i < nv; i += blockDim.x) sh[i] = h2[i];
  __syncthreads();
  const double s = *inv_hn;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    double2 wv = w[p];
    for (int q = 0; q < nv; ++q) {
      const double2 v = V[q * vstride + p];
      const double2 h = sh[q];
      wv.x -= h.x * v.x - h.y * v.y;
      wv.y -= h.x * v.y + h.y * v.x;
    }
    vout[p] = make_double2(wv.x * s, wv.y * s);
  }
}

// Hessenberg column j, Givens rotations and the residual estimate (one thread).
__device__ void arnoldi_small_body(const KrylovState& st, int j, int m) {
  double2* H = st.H;   // [(m+1) x m], column j at H[i * m + j]
  double hs2 = 0.0;
  for (int i = 0; i <= j; ++i) {
    const double2 a = st.h1[i], b = st.h2[i];
    const double2 hsum = make_double2(a.x + b.x, a.y + b.y);
    H[i * m + j] = hsum;
    st.h2[i] = hsum;   // the normalisation forms w - V (h1 + h2) from the unmodified w
    hs2 += b.x * b.x + b.y * b.y;
  }
  const double hn = sqrt(fmax(st.h2[j + 1].x - hs2, 0.0));
  for (int i = 0; i < j; ++i) {
    const double c = st.cs[i];
    const double2 s = st.sn[i];
    const double2 a = H[i * m + j], b = H[(i + 1) * m + j];
    // [a; b] <- [c a + s b; -conj(s) a + c b]
    H[i * m + j] = make_double2(c * a.x + s.x * b.x - s.y * b.y, c * a.y + s.x * b.y + s.y * b.x);
    H[(i + 1) * m + j] = make_double2(-(s.x * a.x + s.y * a.y) + c * b.x, -(s.x * a.y - s.y * a.x) + c * b.y);
  }
  const double2 a = H[j * m + j];
  const double aa = hypot(a.x, a.y);
  double c;
  double2 s, rr;
  if (aa == 0.0) {
    c = 0.0;
    s = make_double2(1.0, 0.0);
    rr = make_double2(hn, 0.0);
  } else {
    const double t = hypot(aa, hn);
    const double2 ph = make_double2(a.x / aa, a.y / aa);
    c = aa / t;
    s = make_double2(ph.x * hn / t, ph.y * hn / t);   // ph * conj(hn) / t, hn real
    rr = make_double2(ph.x * t, ph.y * t);
  }
  H[j * m + j] = rr;
  st.cs[j] = c;
  st.sn[j] = s;
  const double2 gj = st.g[j];
  // g_{j+1} = -conj(s) g_j ; g_j = c g_j
  st.g[j + 1] = make_double2(-(s.x * gj.x + s.y * gj.y), -(s.x * gj.y - s.y * gj.x));
  st.g[j] = make_double2(c * gj.x, c * gj.y);
  st.scal[KS_HN] = hn;
  st.scal[KS_INV_HN] = hn > 0.0 ? 1.0 / hn : 0.0;
  st.scal[KS_EST] = hypot(st.g[j + 1].x, st.g[j + 1].y) / st.scal[KS_BNORM];
}
__global__ void arnoldi_small_kernel(KrylovState st, int j, int m) {
  if (threadIdx.x == 0 && blockIdx.x == 0) arnoldi_small_body(st, j, m);
}

// y = R^-1 g on the k x k leading block of the rotated Hessenberg matrix (one thread).
__global__ void lsq_kernel(KrylovState st, int k, int m) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = k - 1; i >= 0; --i) {
    double2 acc = st.g[i];
    for (int l = i + 1; l < k; ++l) {
      const double2 h = st.H[i * m + l], y = st.y[l];
      acc.x -= h.x * y.x - h.y * y.y;
      acc.y -= h.x * y.y + h.y * y.x;
    }
    const double2 d = st.H[i * m + i];
    const double dd = d.x * d.x + d.y * d.y;
    st.y[i] = make_double2((acc.x * d.x + acc.y * d.y) / dd, (acc.y * d.x - acc.x * d.y) / dd);
  }
}

// x += z with the sum in FP64 (z c128 or c64): the correction step of the stationary
// cycle iteration, one right-hand side per call.
template <typename TZ>
__global__ void __launch_bounds__(kThreads) add_correction_kernel(long long n, double2* __restrict__ x,
                                                                  const c2<TZ>* __restrict__ z,
                                                                  float4* __restrict__ xd) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    double2 v = x[p];
    if constexpr (sizeof(TZ) == sizeof(float)) {
      // (double) z by bit operations (the same values), and x's double-float copy
      const float2 zf = z[p];
      v.x += f2d(zf.x);
      v.y += f2d(zf.y);
      x[p] = v;
      if (xd) xd[p] = cdd_store(cdd{split_d(v.x), split_d(v.y)});
    } else {
      const c2<double> d = cvt<double>(z[p]);
      v.x += d.x;
      v.y += d.y;
      x[p] = v;
    }
  }
}

// x += sum_i y_i z_i
template <typename TZ>
__global__ void __launch_bounds__(kThreads) solution_update_kernel(long long n, double2* __restrict__ x,
                                                                   const c2<TZ>* __restrict__ Z,
                                                                   long long zstride, int k,
                                                                   const double2* __restrict__ y) {
  __shared__ double2 sy[64];
  for (int i = threadIdx.x; i < k; i += blockDim.x) sy[i] = y[i];
  __syncthreads();
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    double2 acc = x[p];
    for (int q = 0; q < k; ++q) acc = cmac(acc, sy[q], cvt<double>(Z[q * zstride + p]));
    x[p] = acc;
  }
}

// x += Z y for a c64 basis Z: the correction sum_q y_q z_q is formed in double-float (z_q
// are exact floats, y_q rounded to about 48 bits) and added to x in FP64; xd receives the
// double-float copy of the new x that the double-float true residual reads.
__global__ void __launch_bounds__(kThreads) solution_update_df_kernel(long long n, double2* __restrict__ x,
                                                                      const float2* __restrict__ Z,
                                                                      long long zstride, int k,
                                                                      const double2* __restrict__ y,
                                                                      float4* __restrict__ xd) {
  __shared__ float4 sy[64];
  for (int i = threadIdx.x; i < k; i += blockDim.x) sy[i] = cdd_store(cdd_make(y[i]));
  __syncthreads();
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    racc re{0.f, 0.f}, im{0.f, 0.f};
    for (int q = 0; q < k; ++q) cacc_add_cz(re, im, cdd_load(sy[q]), Z[q * zstride + p], 1.f);
    const dd ar = racc_dd(re), ai = racc_dd(im);
    double2 xv = x[p];
    xv.x += f2d(ar.hi) + f2d(ar.lo);
    xv.y += f2d(ai.hi) + f2d(ai.lo);
    x[p] = xv;
    xd[p] = cdd_store(cdd{split_d(xv.x), split_d(xv.y)});
  }
}

// r = b - H x (FP64) and ||r||^2 (in out[0].x)
__global__ void __launch_bounds__(kThreads) true_residual_kernel(FineOp op, const double* __restrict__ kap,
                                                                 const double2* __restrict__ b,
                                                                 const double2* __restrict__ x,
                                                                 double2* __restrict__ r,
                                                                 double2* __restrict__ part,
                                                                 unsigned* __restrict__ counter,
                                                                 double2* __restrict__ out) {
  extern __shared__ double2 sacc[];
  const int tid = threadIdx.x;
  sacc[tid] = make_double2(0.0, 0.0);
  for (long long p = blockIdx.x * (long long)blockDim.x + tid; p < op.g.size;
       p += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    node_coords(op.g, p, i, j, k);
    const double2 d = fine_diag<double>(op, kap, p, i, j, k);
    const double2 ax = fine_apply_at<double, double>(op, d, x, p, p, i, j, k, kap);
    const double2 rv = make_double2(b[p].x - ax.x, b[p].y - ax.y);
    r[p] = rv;
    sacc[tid].x += rv.x * rv.x + rv.y * rv.y;
  }
  reduce_finish(sacc, 1, part, counter, out);
}

// ||b||^2 (out[0].x) and, if vout, vout = b (a copy used as the first residual)
__global__ void __launch_bounds__(kThreads) norm2_kernel(long long n, const double2* __restrict__ b,
                                                         double2* __restrict__ vout,
                                                         double2* __restrict__ part,
                                                         unsigned* __restrict__ counter,
                                                         double2* __restrict__ out) {
  extern __shared__ double2 sacc[];
  const int tid = threadIdx.x;
  sacc[tid] = make_double2(0.0, 0.0);
  for (long long p = blockIdx.x * (long long)blockDim.x + tid; p < n; p += (long long)gridDim.x * blockDim.x) {
    const double2 v = b[p];
    if (vout) vout[p] = v;
    sacc[tid].x += v.x * v.x + v.y * v.y;
  }
  reduce_finish(sacc, 1, part, counter, out);
}

// v = r * (1 / beta); resets g = (beta, 0, ...)
__global__ void __launch_bounds__(kThreads) start_cycle_kernel(long long n, const double2* __restrict__ r,
                                                               double2* __restrict__ v, KrylovState st,
                                                               int m) {
  const double beta = st.scal[KS_BETA];
  const double s = 1.0 / beta;
  if (blockIdx.x == 0)
    for (int i = threadIdx.x; i <= m; i += blockDim.x) st.g[i] = make_double2(i == 0 ? beta : 0.0, 0.0);
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    const double2 a = r[p];
    v[p] = make_double2(a.x * s, a.y * s);
  }
}

__global__ void set_scalar_kernel(double* dst, const double2* src_x, int do_sqrt) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *dst = do_sqrt ? sqrt(src_x->x) : src_x->x;
}


// ------------------------------------------------------------------ double-float variants
// Mixed-precision contexts keep the Krylov basis V and w as double-float (float4 per
// complex entry, the size of complex FP64) and run the Arnoldi streams on the FP32 pipes.
struct DfConsts {
  dd ih2, ih2_6, inv24;
  RcBox box;   // real-coefficient box of the operator (fine_apply_df_any)
};

// c = omega^2 kappa^2 (1 - i gamma) per node as double-float.
__global__ void coef_df_kernel(FineOp op, const double* __restrict__ kap, float4* __restrict__ cdf) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < op.g.size;
       p += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    node_coords(op.g, p, i, j, k);
    cdf[p] = cdd_store(cdd_make(fine_coef<double>(op, kap, p, i, j, k)));
  }
}


// Reduction of per-thread double-float accumulators sdf[i * blockDim + tid] (nval sums):
// warps reduce in double-float, the block partials go to part (as float4), and the last
// block adds the partials in block order and converts each sum to FP64 once.
// Returns true in the block that finished the sums (after they are in out, visible to
// the block's threads).
__device__ bool reduce_finish_df(float4* sdf, int nval, double2* __restrict__ part_raw,
                                 unsigned* __restrict__ counter, double2* __restrict__ out) {
  __shared__ bool s_last;
  float4* part = reinterpret_cast<float4*>(part_raw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  __syncthreads();
  for (int i = warp; i < nval; i += nwarp) {
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int t = lane; t < (int)blockDim.x; t += 32) df_acc_add(v, sdf[i * blockDim.x + t]);
    v = df_warp_sum(v);
    if (lane == 0) part[(long long)blockIdx.x * nval + i] = v;
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  for (int i = warp; i < nval; i += nwarp) {
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int b = lane; b < (int)gridDim.x; b += 32) df_acc_add(v, __ldcg(part + (long long)b * nval + i));
    v = df_warp_sum(v);
    if (lane == 0) out[i] = from_df(v);
  }
  if (tid == 0) *counter = 0u;
  __syncthreads();
  return true;
}

// r = b - H x and ||r||^2 (out[0].x) in double-float arithmetic on the FP32 pipes, from the
// double-float copy xd of x: H x by the exact-weight operator on x_hi plus the FP32
// stencil of x_lo (fine_apply_df_t), b split into double-float by bit operations, r
// returned as c128 (relative error about 2^-46 against FP64 arithmetic).
__global__ void __launch_bounds__(kThreads) true_residual_df_kernel(FineOp op, DfConsts K,
                                                                    const float4* __restrict__ cdf,
                                                                    const double2* __restrict__ b,
                                                                    const float4* __restrict__ xd,
                                                                    double2* __restrict__ r,
                                                                    double2* __restrict__ part,
                                                                    unsigned* __restrict__ counter,
                                                                    double2* __restrict__ out) {
  extern __shared__ double2 sacc[];
  float4* sdf = reinterpret_cast<float4*>(sacc);
  const int tid = threadIdx.x;
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  for (long long p = blockIdx.x * (long long)blockDim.x + tid; p < op.g.size;
       p += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    node_coords(op.g, p, i, j, k);
    const cdd hx = fine_apply_df_any<float4>(op, K.box, cdf, xd, p, i, j, k, K.ih2, K.ih2_6, K.inv24);
    const double2 bv = b[p];
    const dd br = split_d(bv.x), bi = split_d(bv.y);
    racc rr{br.hi, br.lo}, ri{bi.hi, bi.lo};
    racc_add(rr, -hx.re.hi);
    racc_add(rr, -hx.re.lo);
    racc_add(ri, -hx.im.hi);
    racc_add(ri, -hx.im.lo);
    const cdd rv{racc_dd(rr), racc_dd(ri)};
    r[p] = make_double2(f2d(rv.re.hi) + f2d(rv.re.lo), f2d(rv.im.hi) + f2d(rv.im.lo));
    const float4 r4 = cdd_store(rv);
    df_cmacc(acc, r4, r4);
  }
  sdf[tid] = acc;
  reduce_finish_df(sdf, 1, part, counter, out);
}

__global__ void __launch_bounds__(kThreads) arnoldi_matvec_df_kernel(
    FineOp op, DfConsts K, const float4* __restrict__ cdf, const float2* __restrict__ z, float4* __restrict__ w,
    const float4* __restrict__ V, long long vstride, int nv, double2* __restrict__ part,
    unsigned* __restrict__ counter, double2* __restrict__ out) {
  extern __shared__ double2 sacc[];
  float4* sdf = reinterpret_cast<float4*>(sacc);
  const int tid = threadIdx.x;
  for (int i = 0; i <= nv; ++i) sdf[i * blockDim.x + tid] = make_float4(0.f, 0.f, 0.f, 0.f);
  for (long long p = blockIdx.x * (long long)blockDim.x + tid; p < op.g.size; p += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    node_coords(op.g, p, i, j, k);
    const float4 wv = cdd_store(fine_apply_df(op, K.box, cdf, z, p, i, j, k, K.ih2, K.ih2_6, K.inv24));
    w[p] = wv;
    for (int q = 0; q < nv; ++q) df_cmacc(sdf[q * blockDim.x + tid], V[q * vstride + p], wv);
    df_cmacc(sdf[nv * blockDim.x + tid], wv, wv);
  }
  reduce_finish_df(sdf, nv + 1, part, counter, out);
}

__global__ void __launch_bounds__(kThreads) arnoldi_update_df_kernel(
    long long n, float4* __restrict__ w, const float4* __restrict__ V, long long vstride, int nv,
    const double2* __restrict__ h1, double2* __restrict__ part, unsigned* __restrict__ counter,
    double2* __restrict__ out) {
  extern __shared__ double2 sacc[];
  float4* sdf = reinterpret_cast<float4*>(sacc);
  __shared__ float4 sh[64];
  const int tid = threadIdx.x;
  for (int i = 0; i <= nv; ++i) sdf[i * blockDim.x + tid] = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int i = tid; i < nv; i += blockDim.x) sh[i] = cdd_store(cdd_make(h1[i]));
  __syncthreads();
  for (long long p = blockIdx.x * (long long)blockDim.x + tid; p < n; p += (long long)gridDim.x * blockDim.x) {
    const float4 w0 = w[p];
    racc re{w0.x, w0.z}, im{w0.y, w0.w};
    for (int q = 0; q < nv; ++q) cacc_sub_cdd(re, im, cdd_load(sh[q]), cdd_load(V[q * vstride + p]));
    const float4 w4 = cdd_store(cdd{racc_dd(re), racc_dd(im)});
    for (int q = 0; q < nv; ++q) df_cmacc(sdf[q * blockDim.x + tid], V[q * vstride + p], w4);
    df_cmacc(sdf[nv * blockDim.x + tid], w4, w4);
  }
  reduce_finish_df(sdf, nv + 1, part, counter, out);
}

__global__ void __launch_bounds__(kThreads) arnoldi_normalize_df_kernel(
    long long n, const float4* __restrict__ w, const float4* __restrict__ V, long long vstride, int nv,
    const double2* __restrict__ h2, const double* __restrict__ inv_hn, float4* __restrict__ vout) {
  __shared__ float4 sh[64];
  __shared__ dd s_inv;
  for (int i = threadIdx.x; i < nv; i += blockDim.x) sh[i] = cdd_store(cdd_make(h2[i]));
  if (threadIdx.x == 0) s_inv = dd_make(*inv_hn);
  __syncthreads();
  const dd sc = s_inv;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    const float4 w0 = w[p];
    racc re{w0.x, w0.z}, im{w0.y, w0.w};
    for (int q = 0; q < nv; ++q) cacc_sub_cdd(re, im, cdd_load(sh[q]), cdd_load(V[q * vstride + p]));
    vout[p] = cdd_store(cdd_scale(cdd{racc_dd(re), racc_dd(im)}, sc));
  }
}

// Arnoldi step for a basis of NV <= kMaxNV vectors with register accumulators.
// First CGS pass: w = H z in double-float, h1 = V^H w from the high parts in FP32.  The
// second pass (update kernel, double-float) orthogonalises against whatever the first
// pass left, so h1 needs only to remove the bulk of w's components along V; the stored
// column of the Hessenberg matrix is h1 + h2.
constexpr int kMaxNV = 10;

template <int NV>
__global__ void __launch_bounds__(kThreads, 4) arnoldi_matvec_df_t(FineOp op, DfConsts K, const float4* __restrict__ cdf,
                                                                const float2* __restrict__ z, float4* __restrict__ w,
                                                                const float4* __restrict__ V, long long vstride,
                                                                double2* __restrict__ part,
                                                                unsigned* __restrict__ counter,
                                                                double2* __restrict__ out) {
  extern __shared__ double2 sacc[];
  float4* sdf = reinterpret_cast<float4*>(sacc);
  const int tid = threadIdx.x;
  float2 acc[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) acc[q] = make_float2(0.f, 0.f);
  for (long long p = blockIdx.x * (long long)blockDim.x + tid; p < op.g.size; p += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    node_coords(op.g, p, i, j, k);
    const float4 wv = cdd_store(fine_apply_df(op, K.box, cdf, z, p, i, j, k, K.ih2, K.ih2_6, K.inv24));
    w[p] = wv;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      const float4 v = V[q * vstride + p];   // acc += conj(v) w, high parts
      acc[q].x = fmaf(v.x, wv.x, acc[q].x);
      acc[q].x = fmaf(v.y, wv.y, acc[q].x);
      acc[q].y = fmaf(v.x, wv.y, acc[q].y);
      acc[q].y = fmaf(-v.y, wv.x, acc[q].y);
    }
  }
#pragma unroll
  for (int q = 0; q < NV; ++q) sdf[q * blockDim.x + tid] = make_float4(acc[q].x, acc[q].y, 0.f, 0.f);
  reduce_finish_df(sdf, NV, part, counter, out);
}

// A load the compiler keeps in place (not merged with an earlier load of the same entry):
// the dot pass re-reads V from L1 instead of holding the subtraction's values in registers.
__device__ __forceinline__ float4 ld_reread(const float4* p) {
  float4 v;
  asm volatile("ld.global.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p));
  return v;
}

// Second CGS pass: w' = w - V h1 (not stored) and h2 = V^H w', |w'|^2 (double-float),
// accumulators in registers (the dot pass re-reads V right after the subtraction read it:
// L1 hits).
// The block that finishes the reduction also forms the Hessenberg column, its Givens
// rotation and the residual estimate (the small step, no separate launch).
// Three blocks per SM (80 registers) up to seven basis vectors, two above: no spills.
template <int NV>
__global__ void __launch_bounds__(kThreads, NV <= 7 ? 3 : 2) arnoldi_update_df_t(long long n, float4* __restrict__ w,
                                                                   const float4* __restrict__ V, long long vstride,
                                                                   const double2* __restrict__ h1,
                                                                   double2* __restrict__ part,
                                                                   unsigned* __restrict__ counter,
                                                                   double2* __restrict__ out, KrylovState st) {
  extern __shared__ double2 sacc[];
  float4* sdf = reinterpret_cast<float4*>(sacc);
  __shared__ float4 sh[NV];
  const int tid = threadIdx.x;
  float4 acc[NV + 1];
#pragma unroll
  for (int q = 0; q <= NV; ++q) acc[q] = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int i = tid; i < NV; i += blockDim.x) sh[i] = cdd_store(cdd_make(h1[i]));
  __syncthreads();
  for (long long p = blockIdx.x * (long long)blockDim.x + tid; p < n; p += (long long)gridDim.x * blockDim.x) {
    const float4 w0 = w[p];
    racc re{w0.x, w0.z}, im{w0.y, w0.w};
#pragma unroll
    for (int q = 0; q < NV; ++q) cacc_sub_cdd(re, im, cdd_load(sh[q]), cdd_load(V[q * vstride + p]));
    const float4 w4 = cdd_store(cdd{racc_dd(re), racc_dd(im)});
#pragma unroll
    for (int q = 0; q < NV; ++q) df_cmacc(acc[q], ld_reread(V + q * vstride + p), w4);
    df_cmacc(acc[NV], w4, w4);
  }
#pragma unroll
  for (int q = 0; q <= NV; ++q) sdf[q * blockDim.x + tid] = acc[q];
  if (reduce_finish_df(sdf, NV + 1, part, counter, out) && tid == 0) arnoldi_small_body(st, NV - 1, st.m);
}

// One-pass Arnoldi step (helm_opts.arnoldi_passes = 1): w = H z and the projections
// h = V^H w in double-float arithmetic (classical Gram-Schmidt once, about 48-bit) with
// ||w||^2, per-thread accumulators in registers.  The last block zeroes h1 and runs the
// small step, which reads h from h2 and ||w||^2 from h2[j + 1]: the new column's norm is
// sqrt(||w||^2 - ||h||^2), exact for an orthonormal V; the subtraction loses digits only
// when w lies almost inside span(V), where the Givens estimate drops to the level of
// convergence and the iteration ends.
template <int NV>
__global__ void __launch_bounds__(kThreads, 2) arnoldi_cgs_df_t(FineOp op, DfConsts K, const float4* __restrict__ cdf,
                                                                const float2* __restrict__ z, float4* __restrict__ w,
                                                                const float4* __restrict__ V, long long vstride,
                                                                KrylovState st) {
  extern __shared__ double2 sacc[];
  float4* sdf = reinterpret_cast<float4*>(sacc);
  const int tid = threadIdx.x;
  float4 acc[NV + 1];
#pragma unroll
  for (int q = 0; q <= NV; ++q) acc[q] = make_float4(0.f, 0.f, 0.f, 0.f);
  for (long long p = blockIdx.x * (long long)blockDim.x + tid; p < op.g.size; p += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    node_coords(op.g, p, i, j, k);
    const float4 wv = cdd_store(fine_apply_df(op, K.box, cdf, z, p, i, j, k, K.ih2, K.ih2_6, K.inv24));
    w[p] = wv;
#pragma unroll
    for (int q = 0; q < NV; ++q) df_cmacc(acc[q], V[q * vstride + p], wv);
    df_cmacc(acc[NV], wv, wv);
  }
#pragma unroll
  for (int q = 0; q <= NV; ++q) sdf[q * blockDim.x + tid] = acc[q];
  if (reduce_finish_df(sdf, NV + 1, st.part, st.counter, st.h2) && tid == 0) {
    for (int i = 0; i < NV; ++i) st.h1[i] = make_double2(0.0, 0.0);
    arnoldi_small_body(st, NV - 1, st.m);
  }
}

template <int NV>
int arnoldi_df_launch(int bl, size_t sm, const FineOp& op, const DfConsts& K, const float4* cdf, const float2* z,
                      float4* w, const float4* V, long long vstride, const KrylovState& st, int passes,
                      cudaStream_t s) {
  if (passes == 1) {
    // one wave of the blocks that fit (two per SM at most, by the launch bounds)
    static const int blc = [sm] {
      cudaFuncSetAttribute(arnoldi_cgs_df_t<NV>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      int per_sm = 0, dev = 0, sms = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, arnoldi_cgs_df_t<NV>, kThreads, sm);
      return std::max(1, per_sm * std::max(sms, 1));
    }();
    KernelTimer kt(HELM_K_ARNOLDI_MATVEC, s);
    arnoldi_cgs_df_t<NV><<<std::min(bl, blc), kThreads, sm, s>>>(op, K, cdf, z, w, V, vstride, st);
    HELM_LAUNCH_CHECK();
    return 0;
  }
  static std::atomic<bool> attr_set{false};
  if (!attr_set) {
    cudaFuncSetAttribute(arnoldi_matvec_df_t<NV>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(arnoldi_update_df_t<NV>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr_set = true;
  }
  {
    KernelTimer kt(HELM_K_ARNOLDI_MATVEC, s);
    arnoldi_matvec_df_t<NV><<<bl, kThreads, sm, s>>>(op, K, cdf, z, w, V, vstride, st.part, st.counter, st.h1);
    HELM_LAUNCH_CHECK();
  }
  {
    // one wave of resident blocks: three per SM up to seven basis vectors, two above
    const int blu = NV <= 7 ? std::min(bl, 152 * 3) : bl;
    KernelTimer kt(HELM_K_ARNOLDI_UPDATE, s);
    arnoldi_update_df_t<NV><<<blu, kThreads, sm, s>>>(op.g.size, w, V, vstride, st.h1, st.part, st.counter, st.h2, st);
    HELM_LAUNCH_CHECK();
  }
  return 0;
}

// v = r / beta into double-float storage; resets g = (beta, 0, ...)
__global__ void __launch_bounds__(kThreads) start_cycle_df_kernel(long long n, const double2* __restrict__ r,
                                                                  float4* __restrict__ v, KrylovState st, int m) {
  const double beta = st.scal[KS_BETA];
  // 1 / beta as double-float; r split by bit operations (no FP64 instruction per node)
  const dd s = dd_make(1.0 / beta);
  if (blockIdx.x == 0)
    for (int i = threadIdx.x; i <= m; i += blockDim.x) st.g[i] = make_double2(i == 0 ? beta : 0.0, 0.0);
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    const double2 a = r[p];
    v[p] = cdd_store(cdd_scale(cdd{split_d(a.x), split_d(a.y)}, s));
  }
}

int grid_blocks(long long n) {
  const long long want = (n + kThreads - 1) / kThreads;
  return (int)std::max<long long>(1, std::min<long long>(want, 152LL * 4));
}

}  // namespace

int krylov_alloc(KrylovState& st, int m, double* scal, double2* part, unsigned* counter) {
  st.m = m;
  st.owns_shared = false;
  HELM_CUDA_TRY(cudaMalloc(&st.H, sizeof(double2) * (m + 1) * m));
  HELM_CUDA_TRY(cudaMalloc(&st.g, sizeof(double2) * (m + 1)));
  HELM_CUDA_TRY(cudaMalloc(&st.sn, sizeof(double2) * m));
  HELM_CUDA_TRY(cudaMalloc(&st.cs, sizeof(double) * m));
  HELM_CUDA_TRY(cudaMalloc(&st.y, sizeof(double2) * m));
  HELM_CUDA_TRY(cudaMalloc(&st.h1, sizeof(double2) * (m + 2)));
  HELM_CUDA_TRY(cudaMalloc(&st.h2, sizeof(double2) * (m + 2)));
  HELM_CUDA_TRY(cudaMalloc(&st.red, sizeof(double2) * 4));
  st.scal = scal;
  st.part = part;
  st.counter = counter;
  HELM_CUDA_TRY(cudaMemset(st.H, 0, sizeof(double2) * (m + 1) * m));
  return 0;
}

void krylov_free(KrylovState& st) {
  cudaFree(st.H); cudaFree(st.g); cudaFree(st.sn); cudaFree(st.cs); cudaFree(st.y);
  cudaFree(st.h1); cudaFree(st.h2); cudaFree(st.red);
  st = KrylovState();
}

size_t krylov_part_entries(int m) { return (size_t)152 * 4 * (m + 2); }

int k_norm(const KrylovState& st, long long n, const double2* b, double2* copy_to, cudaStream_t s) {
  const int bl = grid_blocks(n);
  KernelTimer kt(HELM_K_KRYLOV_OTHER, s);
  norm2_kernel<<<bl, kThreads, kThreads * sizeof(double2), s>>>(n, b, copy_to, st.part, st.counter, st.red);
  HELM_LAUNCH_CHECK();
  set_scalar_kernel<<<1, 32, 0, s>>>(st.scal + KS_BNORM, st.red, 1);
  HELM_LAUNCH_CHECK();
  set_scalar_kernel<<<1, 32, 0, s>>>(st.scal + KS_BETA, st.red, 1);
  HELM_LAUNCH_CHECK();
  return 0;
}

int k_start_cycle(const KrylovState& st, long long n, const double2* r, double2* v0, cudaStream_t s) {
  KernelTimer kt(HELM_K_KRYLOV_OTHER, s);
  start_cycle_kernel<<<grid_blocks(n), kThreads, 0, s>>>(n, r, v0, st, st.m);
  HELM_LAUNCH_CHECK();
  return 0;
}

int k_arnoldi(const KrylovState& st, const FineOp& op, const double* kap64, const void* z, Prec zp,
              double2* w, const double2* V, long long vstride, int j, cudaStream_t s) {
  const long long n = op.g.size;
  const int bl = grid_blocks(n);
  const int nv = j + 1;
  const size_t sm = (size_t)(nv + 1) * kThreads * sizeof(double2);
  static std::atomic<bool> attr_set{false};
  if (!attr_set) {
    const int lim = 200 * 1024;
    cudaFuncSetAttribute(arnoldi_matvec_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(arnoldi_matvec_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(arnoldi_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    attr_set = true;
  }
  {
  KernelTimer kt(HELM_K_ARNOLDI_MATVEC, s);
  if (zp == P64)
    arnoldi_matvec_kernel<double><<<bl, kThreads, sm, s>>>(op, kap64, (const double2*)z, w, V, vstride, nv,
                                                          st.part, st.counter, st.h1);
  else
    arnoldi_matvec_kernel<float><<<bl, kThreads, sm, s>>>(op, kap64, (const float2*)z, w, V, vstride, nv,
                                                         st.part, st.counter, st.h1);
  HELM_LAUNCH_CHECK();
  }
  {
  KernelTimer kt(HELM_K_ARNOLDI_UPDATE, s);
  arnoldi_update_kernel<<<bl, kThreads, sm, s>>>(n, w, V, vstride, nv, st.h1, st.part, st.counter, st.h2);
  HELM_LAUNCH_CHECK();
  }
  KernelTimer kt(HELM_K_KRYLOV_OTHER, s);
  arnoldi_small_kernel<<<1, 32, 0, s>>>(st, j, st.m);
  HELM_LAUNCH_CHECK();
  return 0;
}

DfConsts df_consts(const FineOp& op, const RcBox& box) {
  DfConsts K;
  K.box = box;
  const double ih2 = op.inv_h2;
  auto mk_dd = [](double v) {
    const float hi = (float)v;
    return dd{hi, (float)(v - (double)hi)};
  };
  K.ih2 = mk_dd(ih2);
  K.ih2_6 = mk_dd(ih2 / 6.0);
  K.inv24 = mk_dd(1.0 / 24.0);
  return K;
}

int k_coef_df(const FineOp& op, const double* kap64, float4* cdf, cudaStream_t s) {
  KernelTimer kt(HELM_K_SETUP, s);
  coef_df_kernel<<<grid_blocks(op.g.size), kThreads, 0, s>>>(op, kap64, cdf);
  HELM_LAUNCH_CHECK();
  return 0;
}

int k_start_cycle_df(const KrylovState& st, long long n, const double2* r, float4* v0, cudaStream_t s) {
  KernelTimer kt(HELM_K_KRYLOV_OTHER, s);
  start_cycle_df_kernel<<<grid_blocks(n), kThreads, 0, s>>>(n, r, v0, st, st.m);
  HELM_LAUNCH_CHECK();
  return 0;
}

int k_arnoldi_df(const KrylovState& st, const FineOp& op, const RcBox& box, const float4* cdf, const float2* z,
                 float4* w, const float4* V, long long vstride, int j, int passes, cudaStream_t s) {
  const long long n = op.g.size;
  const int bl = grid_blocks(n);
  const int nv = j + 1;
  const size_t sm = (size_t)(nv + 1) * kThreads * sizeof(double2);
  static std::atomic<bool> attr_set{false};
  if (!attr_set) {
    const int lim = 200 * 1024;
    cudaFuncSetAttribute(arnoldi_matvec_df_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(arnoldi_update_df_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    attr_set = true;
  }
  const DfConsts K = df_consts(op, box);
  if (nv <= kMaxNV) {
    int st2 = 0;
    switch (nv) {
#define HELM_NV(N) \
  case N: st2 = arnoldi_df_launch<N>(bl, sm, op, K, cdf, z, w, V, vstride, st, passes, s); break;
      HELM_NV(1) HELM_NV(2) HELM_NV(3) HELM_NV(4) HELM_NV(5) HELM_NV(6) HELM_NV(7) HELM_NV(8) HELM_NV(9) HELM_NV(10)
#undef HELM_NV
    }
    if (st2) return st2;
  } else {
    {
      KernelTimer kt(HELM_K_ARNOLDI_MATVEC, s);
      arnoldi_matvec_df_kernel<<<bl, kThreads, sm, s>>>(op, K, cdf, z, w, V, vstride, nv, st.part, st.counter, st.h1);
      HELM_LAUNCH_CHECK();
    }
    {
      KernelTimer kt(HELM_K_ARNOLDI_UPDATE, s);
      arnoldi_update_df_kernel<<<bl, kThreads, sm, s>>>(n, w, V, vstride, nv, st.h1, st.part, st.counter, st.h2);
      HELM_LAUNCH_CHECK();
    }
    // the templated update kernels above do the small step in their last block
    KernelTimer kt(HELM_K_KRYLOV_OTHER, s);
    arnoldi_small_kernel<<<1, 32, 0, s>>>(st, j, st.m);
    HELM_LAUNCH_CHECK();
  }
  return 0;
}

int k_normalize_df(const KrylovState& st, long long n, const float4* w, const float4* V, long long vstride, int j,
                   float4* vout, cudaStream_t s) {
  KernelTimer kt(HELM_K_ARNOLDI_NORM, s);
  arnoldi_normalize_df_kernel<<<grid_blocks(n), kThreads, 0, s>>>(n, w, V, vstride, j + 1, st.h2,
                                                                  st.scal + KS_INV_HN, vout);
  HELM_LAUNCH_CHECK();
  return 0;
}

int k_normalize(const KrylovState& st, long long n, const double2* w, const double2* V, long long vstride,
                int j, double2* vout, cudaStream_t s) {
  KernelTimer kt(HELM_K_ARNOLDI_NORM, s);
  arnoldi_normalize_kernel<<<grid_blocks(n), kThreads, 0, s>>>(n, w, V, vstride, j + 1, st.h2,
                                                               st.scal + KS_INV_HN, vout);
  HELM_LAUNCH_CHECK();
  return 0;
}

int k_update_solution(const KrylovState& st, long long n, double2* x, const void* Z, Prec zp,
                      long long zstride, int k, float4* xd, cudaStream_t s) {
  KernelTimer kt(HELM_K_KRYLOV_OTHER, s);
  lsq_kernel<<<1, 32, 0, s>>>(st, k, st.m);
  HELM_LAUNCH_CHECK();
  if (zp == P64)
    solution_update_kernel<double><<<grid_blocks(n), kThreads, 0, s>>>(n, x, (const double2*)Z, zstride, k, st.y);
  else
    solution_update_df_kernel<<<grid_blocks(n), kThreads, 0, s>>>(n, x, (const float2*)Z, zstride, k, st.y, xd);
  HELM_LAUNCH_CHECK();
  return 0;
}

int k_add_correction(long long n, double2* x, const void* z, Prec zp, float4* xd, cudaStream_t s) {
  KernelTimer kt(HELM_K_KRYLOV_OTHER, s);
  if (zp == P64)
    add_correction_kernel<double><<<grid_blocks(n), kThreads, 0, s>>>(n, x, (const double2*)z, nullptr);
  else
    add_correction_kernel<float><<<grid_blocks(n), kThreads, 0, s>>>(n, x, (const float2*)z, xd);
  HELM_LAUNCH_CHECK();
  return 0;
}

int k_true_residual(const KrylovState& st, const FineOp& op, const double* kap64, const double2* b,
                    const double2* x, double2* r, cudaStream_t s) {
  const int bl = grid_blocks(op.g.size);
  KernelTimer kt(HELM_K_KRYLOV_OTHER, s);
  true_residual_kernel<<<bl, kThreads, kThreads * sizeof(double2), s>>>(op, kap64, b, x, r, st.part,
                                                                       st.counter, st.red);
  HELM_LAUNCH_CHECK();
  set_scalar_kernel<<<1, 32, 0, s>>>(st.scal + KS_BETA, st.red, 1);
  HELM_LAUNCH_CHECK();
  return 0;
}

int k_true_residual_df(const KrylovState& st, const FineOp& op, const RcBox& box, const float4* cdf, const double2* b,
                       const float4* xd, double2* r, cudaStream_t s) {
  const int bl = grid_blocks(op.g.size);
  KernelTimer kt(HELM_K_KRYLOV_OTHER, s);
  true_residual_df_kernel<<<bl, kThreads, kThreads * sizeof(float4), s>>>(op, df_consts(op, box), cdf, b, xd, r, st.part,
                                                                          st.counter, st.red);
  HELM_LAUNCH_CHECK();
  set_scalar_kernel<<<1, 32, 0, s>>>(st.scal + KS_BETA, st.red, 1);
  HELM_LAUNCH_CHECK();
  return 0;
}

}  // namespace helm
