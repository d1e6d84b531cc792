// The fine-grid operator H_h = -Lap_h - omega^2 kappa^2 (1 - i gamma) M_h at one node
// (Sec. 1 Eq. acousitcHelm; Sec. 3.1), shared by the cycle and the Krylov kernels.
#pragma once
#include "common.cuh"
#include "df64.cuh"

namespace helm {

// Coefficient c = omega^2 kappa^2 (1 - i gamma) at node (i, j, k).
template <typename T>
__device__ __forceinline__ c2<T> fine_coef(const FineOp& op, const T* __restrict__ kap, long long idx, int i,
                                           int j, int k) {
  const T gam = GamTab<T>::at(op, 0, i) + GamTab<T>::at(op, 1, j) + (op.g.dim == 3 ? GamTab<T>::at(op, 2, k) : T(0));
  const T cre = (T)op.omega2 * kap[idx];
  return mk<T>(cre, -cre * gam);
}

// Diagonal of the fine operator: 2d/h^2 - c (2nd order), or the centre of the compact
// 4th-order stencils, 20/(6h^2) - (8/12) c in 2D (Eq. disc4thCompact) and
// 24/(6h^2) - (6/12) c in 3D (Eq. disc4thCompact3D).
template <typename T>
__device__ __forceinline__ c2<T> fine_diag(const FineOp& op, const T* __restrict__ kap, long long idx,
                                           int i, int j, int k) {
  const c2<T> c = fine_coef<T>(op, kap, idx, i, j, k);
  const T ih2 = (T)op.inv_h2;
  if (op.order == 0) return mk<T>(T(2 * op.g.dim) * ih2 - c.x, -c.y);
  if (op.g.dim == 2) return mk<T>(T(20.0 / 6.0) * ih2 - T(8.0 / 12.0) * c.x, -T(8.0 / 12.0) * c.y);
  return mk<T>(T(4.0) * ih2 - T(0.5) * c.x, -T(0.5) * c.y);
}

// (H x) at flat position p of a vector x, node idx = (i, j, k); zero beyond the boundary.
// 4th order: Laplacian weights per offset class (centre / face / edge), mass weight 1/12
// on the faces with the coefficient mean (c_i + c_j) / 2 of the coupled nodes.
template <typename T, typename TX>
__device__ __forceinline__ c2<T> fine_apply_at(const FineOp& op, c2<T> diag, const c2<TX>* __restrict__ x,
                                               long long p, long long idx, int i, int j, int k,
                                               const T* __restrict__ kap) {
  const long long sy = op.g.N[0];
  const long long sz = (long long)op.g.N[0] * op.g.N[1];
  const T ih2 = (T)op.inv_h2;
  if (op.order == 0) {
    c2<T> s = mk<T>(0, 0);
    if (i > 0) s = s + cvt<T>(x[p - 1]);
    if (i < op.g.N[0] - 1) s = s + cvt<T>(x[p + 1]);
    if (j > 0) s = s + cvt<T>(x[p - sy]);
    if (j < op.g.N[1] - 1) s = s + cvt<T>(x[p + sy]);
    if (op.g.dim == 3) {
      if (k > 0) s = s + cvt<T>(x[p - sz]);
      if (k < op.g.N[2] - 1) s = s + cvt<T>(x[p + sz]);
    }
    return cmul(diag, cvt<T>(x[p])) - cscale(s, ih2);
  }
  const c2<T> ci = fine_coef<T>(op, kap, idx, i, j, k);
  c2<T> acc = cmul(diag, cvt<T>(x[p]));
  const bool is3 = op.g.dim == 3;
  const T wface = is3 ? T(-2.0 / 6.0) * ih2 : T(-4.0 / 6.0) * ih2;
  const T wedge = is3 ? T(-1.0 / 6.0) * ih2 : T(-1.0 / 6.0) * ih2;   // 2D: corners; 3D: edges
  const int zlo = is3 ? -1 : 0, zhi = is3 ? 1 : 0;
  for (int dz = zlo; dz <= zhi; ++dz) {
    const int kk = k + dz;
    if (kk < 0 || kk >= op.g.N[2]) continue;
    for (int dy = -1; dy <= 1; ++dy) {
      const int jj = j + dy;
      if (jj < 0 || jj >= op.g.N[1]) continue;
      for (int dx = -1; dx <= 1; ++dx) {
        const int ii = i + dx;
        if (ii < 0 || ii >= op.g.N[0]) continue;
        const int nz = (dx != 0) + (dy != 0) + (dz != 0);
        if (nz == 0 || (is3 && nz == 3) ) continue;
        const long long q = p + dx + dy * sy + dz * sz;
        const c2<T> xv = cvt<T>(x[q]);
        if (nz == 1) {
          // face: Laplacian weight and mass (1/12) (c_i + c_j) / 2
          const c2<T> cj = fine_coef<T>(op, kap, idx + (q - p), ii, jj, kk);
          const c2<T> m = mk<T>(wface - T(1.0 / 24.0) * (ci.x + cj.x), -T(1.0 / 24.0) * (ci.y + cj.y));
          acc = cmac(acc, m, xv);
        } else {
          acc = acc + cscale(xv, wedge);
        }
      }
    }
  }
  return acc;
}

// (H z) at node p in double-float arithmetic for a vector z of exact floats (c64), with
// the coefficients c as double-float per node (cdf).  The operator is regrouped with
// small integer weights so that every weighted sum of z is formed exactly:
//   2nd order:  H z = ih2 (2d z_c - sum_f z_f) - c_c z_c
//   4th order:  H z = (ih2 / 6) L - (1/24) (c_c Mz + Mcz),
//     L   = wc z_c - wf sum_f z_f - sum_e z_e       (wc, wf = 20, 4 in 2D; 24, 2 in 3D)
//     Mz  = mc z_c + sum_f z_f,  Mcz = mc c_c z_c + sum_f c_f z_f   (mc = 8 in 2D, 6 in 3D)
// (f: face neighbours, e: the other non-zero offsets, i.e. 2D corners and 3D edges).
// Sums are running accumulators (racc, df64.cuh), normalised once where they leave the sum.
//
// With z in double-float (TZ = float4: hi, lo per component), H z = H z_hi + H z_lo: the
// high parts go through the exact-weight form above, the low parts (below 2^-23 |z_hi|)
// through the same stencil in FP32, whose rounding is then of order 2^-47 |H| |z|.
__device__ __forceinline__ float2 df_hi(float2 v) { return v; }
__device__ __forceinline__ float2 df_hi(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 df_lo(float4 v) { return make_float2(v.z, v.w); }

//
// RC: every coefficient c the node reads (its own and its face neighbours') is real, i.e.
// the absorbing profile is zero there (df_real_coef_warp); the products with the imaginary
// parts, exact zeros, are then left out: the result has the same value (at most the sign
// of a zero differs).
template <bool RC>
__device__ __forceinline__ void cacc_add_c(racc& re, racc& im, cdd x, float2 z, float s) {
  if (RC) {
    racc_add_ddf(re, x.re, s * z.x);
    racc_add_ddf(im, x.re, s * z.y);
  } else {
    cacc_add_cz(re, im, x, z, s);
  }
}

template <typename TZ, bool RC = false>
__device__ __forceinline__ cdd fine_apply_df_t(const FineOp& op, const float4* __restrict__ cdf,
                                               const TZ* __restrict__ z, long long p, int i, int j, int k,
                                               dd ih2, dd ih2_6, dd inv24) {
  constexpr bool LO = sizeof(TZ) == sizeof(float4);
  const long long sy = op.g.N[0];
  const long long sz = (long long)op.g.N[0] * op.g.N[1];
  const cdd cc = cdd_load(cdf[p]);
  const TZ zc4 = z[p];
  const float2 zc = df_hi(zc4);
  const bool is3 = op.g.dim == 3;
  // low parts: Laplacian-type sum, mass sums (FP32)
  float2 l_lo = make_float2(0.f, 0.f), z_lo = make_float2(0.f, 0.f), m_lo = make_float2(0.f, 0.f);
  if (op.order == 0) {
    const float wc = 2.0f * op.g.dim;
    racc Lr{0.f, 0.f}, Li{0.f, 0.f};
    racc_add_prod(Lr, wc, zc.x);
    racc_add_prod(Li, wc, zc.y);
    if constexpr (LO) l_lo = cscale(df_lo(zc4), wc);
    auto face = [&](long long q) {
      const TZ zq4 = z[q];
      const float2 zq = df_hi(zq4);
      racc_add(Lr, -zq.x);
      racc_add(Li, -zq.y);
      if constexpr (LO) l_lo = l_lo - df_lo(zq4);
    };
    if (i > 0) face(p - 1);
    if (i < op.g.N[0] - 1) face(p + 1);
    if (j > 0) face(p - sy);
    if (j < op.g.N[1] - 1) face(p + sy);
    if (is3) {
      if (k > 0) face(p - sz);
      if (k < op.g.N[2] - 1) face(p + sz);
    }
    const dd lr = dd_mul(racc_dd(Lr), ih2), li = dd_mul(racc_dd(Li), ih2);
    racc Wr{lr.hi, lr.lo}, Wi{li.hi, li.lo};
    cacc_add_c<RC>(Wr, Wi, cc, zc, -1.f);
    if constexpr (LO) {
      // ih2 L_lo - c_c z_c,lo
      const float2 h = cscale(l_lo, ih2.hi) - cmul(make_float2(cc.re.hi, cc.im.hi), df_lo(zc4));
      racc_add(Wr, h.x);
      racc_add(Wi, h.y);
    }
    return cdd{racc_dd(Wr), racc_dd(Wi)};
  }
  const float wc = is3 ? 24.f : 20.f, wf = is3 ? 2.f : 4.f, mc = is3 ? 6.f : 8.f;
  racc Lr{0.f, 0.f}, Li{0.f, 0.f}, Zr{0.f, 0.f}, Zi{0.f, 0.f}, Mr{0.f, 0.f}, Mi{0.f, 0.f};
  racc_add_prod(Lr, wc, zc.x);
  racc_add_prod(Li, wc, zc.y);
  racc_add_prod(Zr, mc, zc.x);
  racc_add_prod(Zi, mc, zc.y);
  // mc c_c z_c with mc z_c = p + e exact: c_c p + c_c e
  {
    const float pr = mc * zc.x, pi = mc * zc.y;
    const float2 ez = make_float2(fmaf(mc, zc.x, -pr), fmaf(mc, zc.y, -pi));
    cacc_add_c<RC>(Mr, Mi, cc, make_float2(pr, pi), 1.f);
    cacc_add_c<RC>(Mr, Mi, cc, ez, 1.f);
  }
  if constexpr (LO) {
    const float2 zl = df_lo(zc4);
    l_lo = cscale(zl, wc);
    z_lo = cscale(zl, mc);
    m_lo = cmul(make_float2(cc.re.hi, cc.im.hi), z_lo);
  }
  const int zlo = is3 ? -1 : 0, zhi = is3 ? 1 : 0;
  for (int dz = zlo; dz <= zhi; ++dz) {
    const int kk = k + dz;
    if (kk < 0 || kk >= op.g.N[2]) continue;
    for (int dy = -1; dy <= 1; ++dy) {
      const int jj = j + dy;
      if (jj < 0 || jj >= op.g.N[1]) continue;
      for (int dx = -1; dx <= 1; ++dx) {
        const int ii = i + dx;
        if (ii < 0 || ii >= op.g.N[0]) continue;
        const int nz = (dx != 0) + (dy != 0) + (dz != 0);
        if (nz == 0 || nz == 3) continue;
        const long long q = p + dx + dy * sy + dz * sz;
        const TZ zq4 = z[q];
        const float2 zq = df_hi(zq4);
        if (nz == 1) {
          racc_add(Lr, -wf * zq.x);   // wf a power of two: exact
          racc_add(Li, -wf * zq.y);
          racc_add(Zr, zq.x);
          racc_add(Zi, zq.y);
          const cdd cq = cdd_load(cdf[q]);
          cacc_add_c<RC>(Mr, Mi, cq, zq, 1.f);
          if constexpr (LO) {
            const float2 zl = df_lo(zq4);
            l_lo = l_lo - cscale(zl, wf);
            z_lo = z_lo + zl;
            m_lo = m_lo + cmul(make_float2(cq.re.hi, cq.im.hi), zl);
          }
        } else {
          racc_add(Lr, -zq.x);
          racc_add(Li, -zq.y);
          if constexpr (LO) l_lo = l_lo - df_lo(zq4);
        }
      }
    }
  }
  // mass = c_c Mz + Mcz
  racc_add_dd(Mr, cc.re, dd_of(Zr));
  if (!RC) racc_add_dd(Mr, dd_neg(cc.im), dd_of(Zi));
  racc_add_dd(Mi, cc.re, dd_of(Zi));
  if (!RC) racc_add_dd(Mi, cc.im, dd_of(Zr));
  const cdd L{racc_dd(Lr), racc_dd(Li)};
  const cdd mass{racc_dd(Mr), racc_dd(Mi)};
  cdd h = cdd_sub(cdd_scale(L, ih2_6), cdd_scale(mass, inv24));
  if constexpr (LO) {
    // (ih2 / 6) L_lo - (1/24) (c_c Mz_lo + Mcz_lo)
    const float2 hl = cscale(l_lo, ih2_6.hi) - cscale(cmul(make_float2(cc.re.hi, cc.im.hi), z_lo) + m_lo, inv24.hi);
    h.re = dd_add(h.re, dd{hl.x, 0.f});
    h.im = dd_add(h.im, dd{hl.y, 0.f});
  }
  return h;
}

// True when the 32 consecutive nodes of a warp (lane l at x index i, the warp starting at
// x = i - l) lie in one row inside the real-coefficient box: the absorbing profile is zero
// at each of them and at its face neighbours, so that the coefficients
// c = omega^2 kappa^2 (1 - i gamma) the operator reads there are real.  Every
// lane computes the same value (a warp that spans two rows gets false in both), so the
// choice of form never splits a warp.
__device__ __forceinline__ bool df_real_coef_warp(const RcBox& box, int dim, int i, int j, int k) {
  const int xs = i - (int)(threadIdx.x & 31);
  return xs >= box.lo[0] && xs + 31 <= box.hi[0] && j >= box.lo[1] && j <= box.hi[1] &&
         (dim == 2 || (k >= box.lo[2] && k <= box.hi[2]));
}

// H z for a node, with the real-coefficient form where it applies.  The callers are 1D
// grid-stride kernels, so the lanes of a warp hold consecutive nodes and the form is
// chosen per warp (df_real_coef_warp): a per-node choice made the warps at the layer's
// inner edge run both forms, which cost more in 3D than the form saves.
template <typename TZ>
__device__ __forceinline__ cdd fine_apply_df_any(const FineOp& op, const RcBox& box, const float4* __restrict__ cdf,
                                                 const TZ* __restrict__ z, long long p, int i, int j, int k,
                                                 dd ih2, dd ih2_6, dd inv24) {
  if (df_real_coef_warp(box, op.g.dim, i, j, k))
    return fine_apply_df_t<TZ, true>(op, cdf, z, p, i, j, k, ih2, ih2_6, inv24);
  return fine_apply_df_t<TZ, false>(op, cdf, z, p, i, j, k, ih2, ih2_6, inv24);
}

__device__ __forceinline__ cdd fine_apply_df(const FineOp& op, const RcBox& box, const float4* __restrict__ cdf,
                                             const float2* __restrict__ z, long long p, int i, int j, int k,
                                             dd ih2, dd ih2_6, dd inv24) {
  return fine_apply_df_any<float2>(op, box, cdf, z, p, i, j, k, ih2, ih2_6, inv24);
}

}  // namespace helm
