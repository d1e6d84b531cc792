// Shared device helpers and internal types of the RS-CGC Helmholtz library.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <string>
#include <algorithm>
#include <atomic>

#include "../../include/helm.h"

namespace helm {

// ---------------------------------------------------------------- complex types
template <typename T> struct Cplx;
template <> struct Cplx<double> { using type = double2; };
template <> struct Cplx<float> { using type = float2; };
template <typename T> using c2 = typename Cplx<T>::type;

template <typename T> __host__ __device__ __forceinline__ c2<T> mk(T r, T i) {
  c2<T> z; z.x = r; z.y = i; return z;
}
template <typename T, typename S> __host__ __device__ __forceinline__ c2<T> cvt(S a) {
  return mk<T>(static_cast<T>(a.x), static_cast<T>(a.y));
}
// double-float storage (re_hi, im_hi, re_lo, im_lo): FP32 arithmetic takes the high parts
// (the value rounded to float), FP64 arithmetic the sum.
template <typename T> struct DfLoad;
template <> struct DfLoad<float> {
  __host__ __device__ static c2<float> get(float4 a) { return mk<float>(a.x, a.y); }
};
template <> struct DfLoad<double> {
  __host__ __device__ static c2<double> get(float4 a) {
    return mk<double>((double)a.x + (double)a.z, (double)a.y + (double)a.w);
  }
};
template <typename T> __host__ __device__ __forceinline__ c2<T> cvt(float4 a) { return DfLoad<T>::get(a); }
// Arithmetic on the interleaved complex types (overloads for double2 and float2; the
// template parameter of the call sites only selects the type).
#define HELM_COMPLEX_OPS(C, R)                                                             \
  __host__ __device__ __forceinline__ C operator+(C a, C b) { C z; z.x = a.x + b.x; z.y = a.y + b.y; return z; } \
  __host__ __device__ __forceinline__ C operator-(C a, C b) { C z; z.x = a.x - b.x; z.y = a.y - b.y; return z; } \
  __device__ __forceinline__ C cmul(C a, C b) {                                             \
    C z; z.x = a.x * b.x - a.y * b.y; z.y = a.x * b.y + a.y * b.x; return z;                 \
  }                                                                                          \
  __device__ __forceinline__ C cmac(C acc, C a, C b) {                                      \
    acc.x = fma(a.x, b.x, acc.x); acc.x = fma(-a.y, b.y, acc.x);                             \
    acc.y = fma(a.x, b.y, acc.y); acc.y = fma(a.y, b.x, acc.y);                              \
    return acc;                                                                              \
  }                                                                                          \
  __device__ __forceinline__ C cmacc(C acc, C a, C b) {                                     \
    acc.x = fma(a.x, b.x, acc.x); acc.x = fma(a.y, b.y, acc.x);                              \
    acc.y = fma(a.x, b.y, acc.y); acc.y = fma(-a.y, b.x, acc.y);                             \
    return acc;                                                                              \
  }                                                                                          \
  __device__ __forceinline__ C cscale(C a, R s) { C z; z.x = a.x * s; z.y = a.y * s; return z; } \
  __device__ __forceinline__ C crecip(C a) {                                                \
    R d = a.x * a.x + a.y * a.y; C z; z.x = a.x / d; z.y = -a.y / d; return z;               \
  }
HELM_COMPLEX_OPS(double2, double)
HELM_COMPLEX_OPS(float2, float)
#undef HELM_COMPLEX_OPS


// ---------------------------------------------------------------- grids
struct GridDims {
  int dim;
  int N[3];          // nodes per axis (cells + 1); N[2] = 1 in 2D
  long long size;    // total nodes
  // division by N[0] and N[1] as a multiply and shift: n / d = (n * m) >> (32 + s) with
  // s = ceil(log2 d), m = ceil(2^(32+s) / d), exact for every n < 2^31
  unsigned long long m0, m1;
  int s0, s1;
};

// Fills the division constants of a GridDims whose N[] is set.
inline void finish_dims(GridDims& g) {
  auto magic = [](unsigned d, unsigned long long& m, int& s) {
    s = 0;
    while ((1ull << s) < d) ++s;
    const unsigned long long num = 1ull << (32 + s);
    m = (num + d - 1) / d;
  };
  magic((unsigned)g.N[0], g.m0, g.s0);
  magic((unsigned)g.N[1], g.m1, g.s1);
}

__host__ __device__ __forceinline__ unsigned fast_div(unsigned n, unsigned long long m, int s) {
  return (unsigned)((n * m) >> (32 + s));
}

// (i, j, k) of node idx < 2^31.
__host__ __device__ __forceinline__ void node_coords(const GridDims& g, long long idx, int& i, int& j,
                                                     int& k) {
  const unsigned n = (unsigned)idx;
  const unsigned t = fast_div(n, g.m0, g.s0);
  i = (int)(n - t * (unsigned)g.N[0]);
  const unsigned kk = fast_div(t, g.m1, g.s1);
  j = (int)(t - kk * (unsigned)g.N[1]);
  k = (int)kk;
}

// Fine (level-1) operator parameters: -Lap_h - omega^2 kappa^2 (1 - i gamma) with
// gamma = sum over axes of a per-axis profile (already scaled by gamma_max).
struct FineOp {
  GridDims g;
  int order;               // 0 = 2nd-order 5/7-point, 1 = compact 4th-order 9/19-point
  double inv_h2;
  double omega2;
  const double* gam[3];    // per-axis gamma tables (device), length N[a]
  const float* gam32[3];   // the same tables in FP32 (FP32 kernels read these)
};

// Per axis, the index range [lo, hi] where the absorbing profile is zero at the index and
// at both neighbours, so that a node inside the box and its face neighbours have real
// coefficients c (lo > hi: an empty range).  Kept apart from FineOp: a larger FineOp
// parameter changed the register allocation of the FP64 operator kernels.
struct RcBox {
  int lo[3], hi[3];
};

// The per-axis absorbing profile in the arithmetic type of a kernel.
template <typename T> struct GamTab;
template <> struct GamTab<double> {
  __device__ static double at(const FineOp& op, int a, int i) { return op.gam[a][i]; }
};
template <> struct GamTab<float> {
  __device__ static float at(const FineOp& op, int a, int i) { return op.gam32[a][i]; }
};

// Assembled stencil on a coarse level: coef[o * size + node], o in [0, (2r+1)^d).
template <typename T> struct StencilOp {
  GridDims g;
  int r;
  int ncoef;
  const c2<T>* coef;
  const c2<T>* dinv;       // 1 / diagonal
};

// 1D transfer weights, radius 1 (full weighting) or 2 (cubic).
struct Transfer {
  int radius;
  double w[5];             // w[o + radius]
};

// ---------------------------------------------------------------- launch accounting
extern thread_local long long* g_launch_counter;
inline void count_launch() { if (g_launch_counter) ++(*g_launch_counter); }

std::string& last_error_ref();
void set_error(const std::string& s);

#define HELM_CUDA_TRY(call)                                                              \
  do {                                                                                   \
    cudaError_t _e = (call);                                                             \
    if (_e != cudaSuccess) {                                                             \
      ::helm::set_error(std::string(#call) + ": " + cudaGetErrorString(_e));            \
      return HELM_ECUDA;                                                                 \
    }                                                                                    \
  } while (0)

#define HELM_LAUNCH_CHECK()                                                              \
  do {                                                                                   \
    ::helm::count_launch();                                                              \
    cudaError_t _e = cudaGetLastError();                                                 \
    if (_e != cudaSuccess) {                                                             \
      ::helm::set_error(std::string("kernel launch: ") + cudaGetErrorString(_e));       \
      return HELM_ECUDA;                                                                 \
    }                                                                                    \
  } while (0)

inline int blocks_for(long long n, int threads) { return (int)((n + threads - 1) / threads); }

// ---------------------------------------------------------------- programmatic dependent launch
// Kernels launched with launch_pdl may start while the previous kernel of the stream is
// still running.  They call pdl_trigger() early (which lets the next kernel launch once
// every block of this one has started) and pdl_wait() before they read anything an
// earlier kernel wrote; pdl_wait returns once the previous kernel has completed and its
// memory is visible.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

}  // namespace helm
