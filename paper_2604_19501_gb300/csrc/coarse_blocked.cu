// Blocked Gauss-Jordan elimination of the large fronts of the coarsest-level factorisation
// (coarse.cu; Sec. 2 and 3.1 fix only that the coarsest level is solved exactly).
//
// A front's augmented matrix [F | I_S] (nF rows, ld = nF + nS columns, row-major) has its
// first nS columns eliminated with row pivoting among the eliminated rows S, exactly as the
// unblocked elimination does, but a panel of kNb columns at a time:
//   1. pivot rows: LU with partial pivoting of an FP32 copy of the panel's candidate rows
//      (rows k0 .. nS-1, columns k0 .. k1-1); the FP32 copy only chooses the rows, it takes
//      the same decisions as the unblocked elimination up to near ties;
//   2. the chosen rows are swapped in A (columns k0 .. ld-1), in order;
//   3. D = A_PP^-1 of the kNb x kNb pivot block (FP64 Gauss-Jordan with row pivoting);
//   4. X = D A_PR on the rest of the columns (k1 .. ld-1), then A_OR -= A_OP X for every
//      other row O (rows above k0 and below k1), and A_PR = X.
// Step 4 is two FP64 complex matrix products, which carry almost all of the work
// (about nS nF (ld - nS/2) complex multiply-adds per front); the columns of the eliminated
// panels are not updated, since nothing reads them afterwards.
//
// Large fronts are also assembled and extracted by grid-wide kernels instead of one block.
#include <algorithm>
#include <vector>
#include "coarse.cuh"
#include "df64.cuh"
#include "timer.cuh"

namespace helm {

namespace {

constexpr int kNb = 64;          // panel width
constexpr int kGT = 64;          // product tile (rows and columns of C per block)
constexpr int kGK = 8;           // product tile depth

// C = (accumulate ? C : 0) + sign * A B: C M x N, A M x K, B K x N, row-major with leading
// dimensions lda, ldb, ldc; complex FP64.  256 threads, each 4 x 4 entries of a 64 x 64 tile.
__global__ void __launch_bounds__(256) zgemm_kernel(int M, int N, int K, const double2* __restrict__ A, long long lda,
                                                    const double2* __restrict__ B, long long ldb, double2* __restrict__ C,
                                                    long long ldc, double sign, int accumulate) {
  __shared__ double2 sA[kGK][kGT + 1];
  __shared__ double2 sB[kGK][kGT];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int m0 = blockIdx.y * kGT, n0 = blockIdx.x * kGT;
  double2 acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_double2(0.0, 0.0);
  for (int k0 = 0; k0 < K; k0 += kGK) {
    for (int q = threadIdx.x; q < kGT * kGK; q += 256) {
      const int mm = q / kGK, kk = q % kGK, gm = m0 + mm, gk = k0 + kk;
      sA[kk][mm] = (gm < M && gk < K) ? A[gm * lda + gk] : make_double2(0.0, 0.0);
    }
    for (int q = threadIdx.x; q < kGK * kGT; q += 256) {
      const int kk = q / kGT, nn = q % kGT, gk = k0 + kk, gn = n0 + nn;
      sB[kk][nn] = (gk < K && gn < N) ? B[gk * ldb + gn] : make_double2(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kGK; ++kk) {
      double2 a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = sA[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = sB[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = cmac(acc[i][j], a[i], b[j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int m = m0 + ty + 16 * i, n = n0 + tx + 16 * j;
      if (m < M && n < N) {
        double2* c = C + m * ldc + n;
        const double2 v = make_double2(sign * acc[i][j].x, sign * acc[i][j].y);
        *c = accumulate ? make_double2(c->x + v.x, c->y + v.y) : v;
      }
    }
}

int zgemm(int M, int N, int K, const double2* A, long long lda, const double2* B, long long ldb, double2* C,
          long long ldc, double sign, bool accumulate, cudaStream_t s) {
  if (M <= 0 || N <= 0 || K <= 0) return 0;
  const dim3 grid((N + kGT - 1) / kGT, (M + kGT - 1) / kGT);
  if (grid.y > 65535u) {
    set_error("blocked factorisation: product too tall");
    return HELM_EINVAL;
  }
  zgemm_kernel<<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, sign, accumulate ? 1 : 0);
  HELM_LAUNCH_CHECK();
  return 0;
}

// W (nc x w, FP32 complex) = A rows r0 .. r0+nc-1, columns c0 .. c0+w-1
__global__ void panel_copy_kernel(const double2* __restrict__ A, long long ld, int r0, int c0, int nc, int w,
                                  float2* __restrict__ W) {
  const long long n = (long long)nc * w;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t / w), c = (int)(t % w);
    const double2 v = A[(long long)(r0 + i) * ld + c0 + c];
    W[t] = make_float2((float)v.x, (float)v.y);
  }
}

// LU with partial pivoting of W (nc x w, nc >= w) in one block: piv[j] = row swapped with
// row j at step j (ties: the lowest row).  Only the pivot choice is used.
__global__ void __launch_bounds__(1024) panel_lu_kernel(float2* __restrict__ W, int nc, int w, int* __restrict__ piv,
                                                        int* __restrict__ err) {
  __shared__ float s_val[32];
  __shared__ int s_idx[32];
  __shared__ int s_p;
  __shared__ float2 s_row[kNb];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  for (int j = 0; j < w; ++j) {
    float best = -1.f;
    int bi = nc;
    for (int i = j + tid; i < nc; i += blockDim.x) {
      const float2 a = W[(long long)i * w + j];
      const float v = a.x * a.x + a.y * a.y;
      if (v > best) { best = v; bi = i; }
    }
    for (int off = 16; off > 0; off >>= 1) {
      const float ov = __shfl_down_sync(0xffffffffu, best, off);
      const int oi = __shfl_down_sync(0xffffffffu, bi, off);
      if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    if (lane == 0) { s_val[warp] = best; s_idx[warp] = bi; }
    __syncthreads();
    if (tid == 0) {
      float bv = s_val[0];
      int bidx = s_idx[0];
      for (int q = 1; q < nwarp; ++q)
        if (s_val[q] > bv || (s_val[q] == bv && s_idx[q] < bidx)) { bv = s_val[q]; bidx = s_idx[q]; }
      if (!(bv > 0.f) || !isfinite(bv) || bidx >= nc) {
        atomicExch(err, kErrPivot);
        bidx = j;
      }
      s_p = bidx;
      piv[j] = bidx;
    }
    __syncthreads();
    const int p = s_p;
    for (int c = tid; c < w; c += blockDim.x) {
      const float2 t = W[(long long)j * w + c];
      const float2 u = W[(long long)p * w + c];
      W[(long long)j * w + c] = u;
      W[(long long)p * w + c] = t;
      s_row[c] = u;
    }
    __syncthreads();
    const float2 d = s_row[j];
    const float m2 = d.x * d.x + d.y * d.y;
    const float2 inv = m2 > 0.f ? make_float2(d.x / m2, -d.y / m2) : make_float2(0.f, 0.f);
    for (int i = j + 1 + tid; i < nc; i += blockDim.x) {
      float2* Wi = W + (long long)i * w;
      const float2 f = cmul(Wi[j], inv);
      for (int c = j + 1; c < w; ++c) {
        const float2 r = s_row[c];
        Wi[c] = make_float2(Wi[c].x - (f.x * r.x - f.y * r.y), Wi[c].y - (f.x * r.y + f.y * r.x));
      }
    }
    __syncthreads();
  }
}

// Row swaps of A in order (rows r0 + j and r0 + piv[j], j < w), columns c0 .. ld-1.
__global__ void row_swap_kernel(double2* __restrict__ A, long long ld, int r0, int c0, int w, const int* __restrict__ piv) {
  __shared__ int sp[kNb];
  for (int j = threadIdx.x; j < w; j += blockDim.x) sp[j] = piv[j];
  __syncthreads();
  for (long long c = c0 + blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ld; c += (long long)gridDim.x * blockDim.x) {
    for (int j = 0; j < w; ++j) {
      const int p = sp[j];
      if (p == j) continue;
      double2* a = A + (long long)(r0 + j) * ld + c;
      double2* b = A + (long long)(r0 + p) * ld + c;
      const double2 t = *a;
      *a = *b;
      *b = t;
    }
  }
}

// D = (A_PP)^-1 for the w x w block at (r0, r0) of A, by Gauss-Jordan with row pivoting on
// [A_PP | I] in shared memory (one block).
__global__ void __launch_bounds__(256) pivot_inverse_kernel(const double2* __restrict__ A, long long ld, int r0, int w,
                                                            double2* __restrict__ D, int* __restrict__ err) {
  extern __shared__ double2 sm[];   // [w][2w]
  __shared__ double s_val[32];
  __shared__ int s_idx[32];
  __shared__ int s_p;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  const int L = 2 * w;
  for (int t = tid; t < w * L; t += blockDim.x) {
    const int i = t / L, c = t % L;
    sm[t] = c < w ? A[(long long)(r0 + i) * ld + r0 + c] : make_double2(c - w == i ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  for (int k = 0; k < w; ++k) {
    double best = -1.0;
    int bi = w;
    for (int i = k + tid; i < w; i += blockDim.x) {
      const double2 a = sm[i * L + k];
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
      for (int q = 1; q < nwarp; ++q)
        if (s_val[q] > bv || (s_val[q] == bv && s_idx[q] < bidx)) { bv = s_val[q]; bidx = s_idx[q]; }
      if (!(bv > 0.0) || !isfinite(bv) || bidx >= w) {
        atomicExch(err, kErrPivot);
        bidx = k;
      }
      s_p = bidx;
    }
    __syncthreads();
    const int p = s_p;
    if (p != k)
      for (int c = tid; c < L; c += blockDim.x) {
        const double2 t = sm[k * L + c];
        sm[k * L + c] = sm[p * L + c];
        sm[p * L + c] = t;
      }
    __syncthreads();
    const double2 a = sm[k * L + k];
    const double m = a.x * a.x + a.y * a.y;
    const double2 inv = m > 0.0 ? make_double2(a.x / m, -a.y / m) : make_double2(0.0, 0.0);
    __syncthreads();
    for (int c = tid; c < L; c += blockDim.x) sm[k * L + c] = cmul(sm[k * L + c], inv);
    __syncthreads();
    for (int t = tid; t < w * L; t += blockDim.x) {
      const int i = t / L, c = t % L;
      if (i == k || c == k) continue;
      const double2 f = sm[i * L + k];
      const double2 r = sm[k * L + c];
      sm[t] = make_double2(sm[t].x - (f.x * r.x - f.y * r.y), sm[t].y - (f.x * r.y + f.y * r.x));
    }
    __syncthreads();
    for (int i = tid; i < w; i += blockDim.x)
      if (i != k) sm[i * L + k] = make_double2(0.0, 0.0);
    __syncthreads();
  }
  for (int t = tid; t < w * w; t += blockDim.x) {
    const int i = t / w, c = t % w;
    D[t] = sm[i * L + w + c];
  }
}

// A rows r0 .. r0+w-1, columns c0 .. c0+n-1 = X (w x n, leading dimension n)
__global__ void copy_rows_kernel(double2* __restrict__ A, long long ld, int r0, int c0, int w, int n,
                                 const double2* __restrict__ X) {
  const long long tot = (long long)w * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t / n), c = (int)(t % n);
    A[(long long)(r0 + i) * ld + c0 + c] = X[t];
  }
}

// ---- grid-wide assembly and extraction of one large front
__global__ void set_identity_kernel(double2* __restrict__ A, long long ld, int nS, int nF) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nS; i += gridDim.x * blockDim.x)
    A[(long long)i * ld + nF + i] = make_double2(1.0, 0.0);
}
__global__ void scatter_entries_kernel(double2* __restrict__ A, const int2* __restrict__ ents, int cnt,
                                       const double2* __restrict__ coef) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < cnt; e += gridDim.x * blockDim.x) {
    const int2 en = ents[e];
    const double2 v = coef[en.y];
    A[en.x].x += v.x;
    A[en.x].y += v.y;
  }
}
__global__ void extend_add_kernel(double2* __restrict__ A, long long ld, const double2* __restrict__ U, int nB,
                                  const int* __restrict__ map) {
  const long long n2 = (long long)nB * nB;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n2; t += (long long)gridDim.x * blockDim.x) {
    const int a = (int)(t / nB), b = (int)(t % nB);
    double2& dst = A[(long long)map[a] * ld + map[b]];
    const double2 v = U[t];
    dst.x += v.x;
    dst.y += v.y;
  }
}
__device__ __forceinline__ void store_entry(double2* base, long long i, double2 v, bool df) {
  if (df) reinterpret_cast<float4*>(base)[i] = to_df(v);
  else base[i] = v;
}
__global__ void extract_front_kernel(const double2* __restrict__ A, int nS, int nB, int bsign, double2* __restrict__ M,
                                     double2* __restrict__ GT, double2* __restrict__ U, bool df) {
  const int nF = nS + nB;
  const long long ld = nF + nS;
  const long long nm = (long long)nS * nF, ng = (long long)nS * nB, nu = (long long)nB * nB;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nm; t += stride) {
    const int row = (int)(t / nF), col = (int)(t % nF);
    if (bsign < 0) store_entry(M, t, A[row * ld + (col < nS ? nF + col : col)], df);
    else store_entry(M, t, A[(long long)col * ld + nF + row], df);
  }
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < ng; t += stride) {
    const int c = (int)(t / nS), row = (int)(t % nS);
    store_entry(GT, t, A[row * ld + nS + c], df);
  }
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nu; t += stride) {
    const int row = (int)(t / nB), col = (int)(t % nB);
    U[t] = A[(nS + row) * ld + nS + col];
  }
}

int grid_for(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 152LL * 16)); }

}  // namespace

int big_front_assemble(const FrontDesc& d, const std::vector<FrontDesc>& desc, const std::vector<int>& kids,
                       double2* aug, const int2* d_ents, const double2* coef, const double2* upool, const int* d_cmap,
                       cudaStream_t s) {
  const int nF = d.nS + d.nB;
  const long long ld = nF + d.nS;
  double2* A = aug + d.aug_off;
  HELM_CUDA_TRY(cudaMemsetAsync(A, 0, (size_t)nF * ld * sizeof(double2), s));
  set_identity_kernel<<<grid_for(d.nS), 256, 0, s>>>(A, ld, d.nS, nF);
  HELM_LAUNCH_CHECK();
  if (d.ent_cnt > 0) {
    scatter_entries_kernel<<<grid_for(d.ent_cnt), 256, 0, s>>>(A, d_ents + d.ent_off, d.ent_cnt, coef);
    HELM_LAUNCH_CHECK();
  }
  for (int c = 0; c < d.nkids; ++c) {
    const FrontDesc& kd = desc[kids[d.kid_off + c]];
    extend_add_kernel<<<grid_for((long long)kd.nB * kd.nB), 256, 0, s>>>(A, ld, upool + kd.U_off, kd.nB, d_cmap + kd.cmap_off);
    HELM_LAUNCH_CHECK();
  }
  return 0;
}

int big_front_extract(const FrontDesc& d, const double2* aug, double2* factors, double2* upool, bool df, cudaStream_t s) {
  const long long n = (long long)d.nS * (d.nS + d.nB);
  extract_front_kernel<<<grid_for(n), 256, 0, s>>>(aug + d.aug_off, d.nS, d.nB, d.bsign, factors + d.M_off,
                                                   factors + d.G_off, upool + d.U_off, df);
  HELM_LAUNCH_CHECK();
  return 0;
}

int big_front_eliminate(const FrontDesc& d, double2* aug, float2* w32, int* piv, double2* dinv, double2* xbuf, int* err,
                        cudaStream_t s) {
  const int nS = d.nS, nF = nS + d.nB;
  const long long ld = nF + nS;
  double2* A = aug + d.aug_off;
  static std::atomic<bool> attr{false};
  if (!attr) {
    HELM_CUDA_TRY(cudaFuncSetAttribute(pivot_inverse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kNb * 2 * kNb * (int)sizeof(double2)));
    attr = true;
  }
  for (int k0 = 0; k0 < nS; k0 += kNb) {
    const int w = std::min(kNb, nS - k0), k1 = k0 + w, nc = nS - k0;
    const int nrest = (int)(ld - k1);
    panel_copy_kernel<<<grid_for((long long)nc * w), 256, 0, s>>>(A, ld, k0, k0, nc, w, w32);
    HELM_LAUNCH_CHECK();
    panel_lu_kernel<<<1, 1024, 0, s>>>(w32, nc, w, piv, err);
    HELM_LAUNCH_CHECK();
    row_swap_kernel<<<grid_for(ld - k0), 256, 0, s>>>(A, ld, k0, k0, w, piv);
    HELM_LAUNCH_CHECK();
    pivot_inverse_kernel<<<1, 256, (size_t)w * 2 * w * sizeof(double2), s>>>(A, ld, k0, w, dinv, err);
    HELM_LAUNCH_CHECK();
    // X = D A_PR
    if (int st = zgemm(w, nrest, w, dinv, w, A + (long long)k0 * ld + k1, ld, xbuf, nrest, 1.0, false, s)) return st;
    // A_OR -= A_OP X, rows above and below the panel
    if (int st = zgemm(k0, nrest, w, A + k0, ld, xbuf, nrest, A + k1, ld, -1.0, true, s)) return st;
    if (int st = zgemm(nF - k1, nrest, w, A + (long long)k1 * ld + k0, ld, xbuf, nrest, A + (long long)k1 * ld + k1,
                       ld, -1.0, true, s))
      return st;
    copy_rows_kernel<<<grid_for((long long)w * nrest), 256, 0, s>>>(A, ld, k0, k1, w, nrest, xbuf);
    HELM_LAUNCH_CHECK();
  }
  return 0;
}

}  // namespace helm
