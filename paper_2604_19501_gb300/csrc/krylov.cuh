// Host-side launchers of the FGMRES kernels.
#pragma once
#include "common.cuh"
#include "gridops.cuh"

namespace helm {

enum { KS_BNORM = 0, KS_BETA = 1, KS_HN = 2, KS_INV_HN = 3, KS_EST = 4, KS_COUNT = 8 };

// Device-resident state of one FGMRES(m) solve (FP64).
struct KrylovState {
  int m = 0;
  double2* H = nullptr;      // (m+1) x m Hessenberg, rotated in place
  double2* g = nullptr;      // m+1 right-hand side of the least-squares problem
  double2* sn = nullptr;     // m Givens sines
  double* cs = nullptr;      // m Givens cosines
  double2* y = nullptr;      // m least-squares solution
  double2* h1 = nullptr;     // first Gram-Schmidt pass (+ ||w||^2)
  double2* h2 = nullptr;     // second pass (+ ||w'||^2); h1 + h2 after the small step
  double2* red = nullptr;    // reduction outputs
  double* scal = nullptr;    // KS_* scalars
  double2* part = nullptr;   // per-block partial sums (shared by the states of a context)
  unsigned* counter = nullptr;
  bool owns_shared = false;
};

// The small per-right-hand-side arrays; scal (KS_COUNT doubles), the partial-sum buffer
// (krylov_part_entries(m) entries) and the zeroed counter are supplied by the caller:
// the states of one context run on one stream, one after the other, and share them.
int krylov_alloc(KrylovState& st, int m, double* scal, double2* part, unsigned* counter);
void krylov_free(KrylovState& st);
size_t krylov_part_entries(int m);

// scal[KS_BNORM] = scal[KS_BETA] = ||b||; if copy_to, copy_to = b.
int k_norm(const KrylovState& st, long long n, const double2* b, double2* copy_to, cudaStream_t s);
// v0 = r / beta (beta = scal[KS_BETA]); g = (beta, 0, ...).
int k_start_cycle(const KrylovState& st, long long n, const double2* r, double2* v0, cudaStream_t s);
// Arnoldi step j from z_j (c128 or c64): w, H(:, j), rotations, estimate scal[KS_EST].
int k_arnoldi(const KrylovState& st, const FineOp& op, const double* kap64, const void* z, Prec zp,
              double2* w, const double2* V, long long vstride, int j, cudaStream_t s);
// v_{j+1} = (w - V h) / hn, h = h1 + h2 (stored in h2 by the Arnoldi step's small step).
int k_normalize(const KrylovState& st, long long n, const double2* w, const double2* V, long long vstride,
                int j, double2* vout, cudaStream_t s);
// Double-float variants (mixed precision): V and w stored as float4 (hi, lo) pairs.
int k_coef_df(const FineOp& op, const double* kap64, float4* cdf, cudaStream_t s);
int k_start_cycle_df(const KrylovState& st, long long n, const double2* r, float4* v0, cudaStream_t s);
// passes: 2 = CGS2 (FP32 first pass, double-float second pass), 1 = one double-float pass.
// box: the real-coefficient box of op (nodes whose coefficients and face neighbours' are real).
int k_arnoldi_df(const KrylovState& st, const FineOp& op, const RcBox& box, const float4* cdf, const float2* z,
                 float4* w, const float4* V, long long vstride, int j, int passes, cudaStream_t s);
int k_normalize_df(const KrylovState& st, long long n, const float4* w, const float4* V, long long vstride, int j,
                   float4* vout, cudaStream_t s);
// y = R^-1 g (k x k) and x += Z y; for a c64 basis (zp = P32) also xd = x as double-float.
int k_update_solution(const KrylovState& st, long long n, double2* x, const void* Z, Prec zp,
                      long long zstride, int k, float4* xd, cudaStream_t s);
// x += z (z c128 or c64), summed in FP64; for c64 z and a non-null xd also xd = x as
// double-float.
int k_add_correction(long long n, double2* x, const void* z, Prec zp, float4* xd, cudaStream_t s);
// r = b - H x in FP64, scal[KS_BETA] = ||r||.
int k_true_residual(const KrylovState& st, const FineOp& op, const double* kap64, const double2* b,
                    const double2* x, double2* r, cudaStream_t s);
// The same in double-float arithmetic from xd (x as double-float) and the double-float
// coefficients cdf; r is c128.
int k_true_residual_df(const KrylovState& st, const FineOp& op, const RcBox& box, const float4* cdf, const double2* b,
                       const float4* xd, double2* r, cudaStream_t s);

}  // namespace helm
