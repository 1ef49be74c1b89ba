// Shared device-side definitions for the Frobenius inversion kernels.
//
// Scalar types: double / float for the real planes A and B of M = A + iB
// (Sec. 1.3 of Dai, Lim and Ye: Frobenius inversion works on the real and
// imaginary parts as separate real matrices), and zd / zf, interleaved complex
// numbers, for the complex-arithmetic baselines (Algorithms "Inversion with LU
// decomposition" and "Inversion with Cholesky decomposition").
//
// All matrices are row-major with an element leading dimension and an element
// batch stride.  Batched kernels take the matrix index from blockIdx.z.
#pragma once

#include <cstdint>
#include <mutex>
#include <set>
#include <tuple>
#include <type_traits>
#include <cuda_runtime.h>

#include "../../include/frobinv.h"

namespace frob {

struct __align__(16) zd {
  double x, y;
};
struct __align__(8) zf {
  float x, y;
};

template <typename T> struct real_of { using type = T; };
template <> struct real_of<zd> { using type = double; };
template <> struct real_of<zf> { using type = float; };

template <typename T> struct is_cplx { static constexpr bool value = false; };
template <> struct is_cplx<zd> { static constexpr bool value = true; };
template <> struct is_cplx<zf> { static constexpr bool value = true; };

// ---------------------------------------------------------------- arithmetic
__host__ __device__ __forceinline__ double zero_of(double) { return 0.0; }
__host__ __device__ __forceinline__ float zero_of(float) { return 0.0f; }
__host__ __device__ __forceinline__ zd zero_of(zd) { return zd{0.0, 0.0}; }
__host__ __device__ __forceinline__ zf zero_of(zf) { return zf{0.0f, 0.0f}; }

template <typename T> __host__ __device__ __forceinline__ T one_v();
template <> __host__ __device__ __forceinline__ double one_v<double>() { return 1.0; }
template <> __host__ __device__ __forceinline__ float one_v<float>() { return 1.0f; }
template <> __host__ __device__ __forceinline__ zd one_v<zd>() { return zd{1.0, 0.0}; }
template <> __host__ __device__ __forceinline__ zf one_v<zf>() { return zf{1.0f, 0.0f}; }

template <typename T> __host__ __device__ __forceinline__ T zero_v() { return zero_of(T{}); }

// acc += a * b
// warp shuffle of a scalar or an interleaved complex number
__device__ __forceinline__ double shfl_(unsigned m, double v, int src) { return __shfl_sync(m, v, src); }
__device__ __forceinline__ float shfl_(unsigned m, float v, int src) { return __shfl_sync(m, v, src); }
__device__ __forceinline__ zd shfl_(unsigned m, zd v, int src) {
  return zd{__shfl_sync(m, v.x, src), __shfl_sync(m, v.y, src)};
}
__device__ __forceinline__ zf shfl_(unsigned m, zf v, int src) {
  return zf{__shfl_sync(m, v.x, src), __shfl_sync(m, v.y, src)};
}

__device__ __forceinline__ void mac(double& acc, double a, double b) { acc = fma(a, b, acc); }
__device__ __forceinline__ void mac(float& acc, float a, float b) { acc = fmaf(a, b, acc); }
__device__ __forceinline__ void mac(zd& acc, zd a, zd b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
__device__ __forceinline__ void mac(zf& acc, zf a, zf b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
}

__host__ __device__ __forceinline__ double conj_(double a) { return a; }
__host__ __device__ __forceinline__ float conj_(float a) { return a; }
__host__ __device__ __forceinline__ zd conj_(zd a) { return zd{a.x, -a.y}; }
__host__ __device__ __forceinline__ zf conj_(zf a) { return zf{a.x, -a.y}; }

__host__ __device__ __forceinline__ double add_(double a, double b) { return a + b; }
__host__ __device__ __forceinline__ float add_(float a, float b) { return a + b; }
__host__ __device__ __forceinline__ zd add_(zd a, zd b) { return zd{a.x + b.x, a.y + b.y}; }
__host__ __device__ __forceinline__ zf add_(zf a, zf b) { return zf{a.x + b.x, a.y + b.y}; }

__host__ __device__ __forceinline__ double sub_(double a, double b) { return a - b; }
__host__ __device__ __forceinline__ float sub_(float a, float b) { return a - b; }
__host__ __device__ __forceinline__ zd sub_(zd a, zd b) { return zd{a.x - b.x, a.y - b.y}; }
__host__ __device__ __forceinline__ zf sub_(zf a, zf b) { return zf{a.x - b.x, a.y - b.y}; }

__host__ __device__ __forceinline__ double mul_(double a, double b) { return a * b; }
__host__ __device__ __forceinline__ float mul_(float a, float b) { return a * b; }
__host__ __device__ __forceinline__ zd mul_(zd a, zd b) { return zd{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
__host__ __device__ __forceinline__ zf mul_(zf a, zf b) { return zf{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }

__host__ __device__ __forceinline__ double neg_(double a) { return -a; }
__host__ __device__ __forceinline__ float neg_(float a) { return -a; }
__host__ __device__ __forceinline__ zd neg_(zd a) { return zd{-a.x, -a.y}; }
__host__ __device__ __forceinline__ zf neg_(zf a) { return zf{-a.x, -a.y}; }

// |a|^2 (the pivot key: the squared modulus for complex numbers)
__device__ __forceinline__ double abs2_(double a) { return a * a; }
__device__ __forceinline__ float abs2_(float a) { return a * a; }
__device__ __forceinline__ double abs2_(zd a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ float abs2_(zf a) { return a.x * a.x + a.y * a.y; }

// exact reciprocal by division (IEEE division for reals; for complex numbers
// 1/z = conj(z)/|z|^2, evaluated with a scaling that avoids overflow)
__device__ __forceinline__ double recip_(double a) { return 1.0 / a; }
__device__ __forceinline__ float recip_(float a) { return 1.0f / a; }
__device__ __forceinline__ zd recip_(zd a) {
  double s = fmax(fabs(a.x), fabs(a.y));
  double ar = a.x / s, ai = a.y / s;
  double d = (ar * ar + ai * ai) * s;
  return zd{ar / d, -ai / d};
}
__device__ __forceinline__ zf recip_(zf a) {
  float s = fmaxf(fabsf(a.x), fabsf(a.y));
  float ar = a.x / s, ai = a.y / s;
  float d = (ar * ar + ai * ai) * s;
  return zf{ar / d, -ai / d};
}

__host__ __device__ __forceinline__ double real_(double a) { return a; }
__host__ __device__ __forceinline__ float real_(float a) { return a; }
__host__ __device__ __forceinline__ double real_(zd a) { return a.x; }
__host__ __device__ __forceinline__ float real_(zf a) { return a.x; }

template <typename T> __device__ __forceinline__ T from_real(typename real_of<T>::type r);
template <> __device__ __forceinline__ double from_real<double>(double r) { return r; }
template <> __device__ __forceinline__ float from_real<float>(float r) { return r; }
template <> __device__ __forceinline__ zd from_real<zd>(double r) { return zd{r, 0.0}; }
template <> __device__ __forceinline__ zf from_real<zf>(float r) { return zf{r, 0.0f}; }

__device__ __forceinline__ bool finite_(double a) { return isfinite(a); }
__device__ __forceinline__ bool finite_(float a) { return isfinite(a); }

// ---------------------------------------------------------------- views
// A batch of equally sized row-major matrices: element (b, i, j) lives at
// p[b * bs + i * ld + j].
template <typename T> struct MatB {
  T* p;
  int64_t ld;
  int64_t bs;
  __host__ __device__ __forceinline__ T* at(int b) const { return p + (int64_t)b * bs; }
  __host__ __device__ __forceinline__ MatB sub(int64_t i, int64_t j) const { return MatB{p + i * ld + j, ld, bs}; }
  // the batch starting at matrix `first`
  __host__ __device__ __forceinline__ MatB at_batch(int64_t first) const { return MatB{p + first * bs, ld, bs}; }
};

template <typename T> __host__ __device__ inline MatB<T> matb(T* p, int64_t ld, int64_t bs) { return MatB<T>{p, ld, bs}; }

// Operand access modes of a GEMM / triangular operand.
enum Op : int { OP_N = 0, OP_T = 1, OP_C = 2 };

// Launch bookkeeping (host): every kernel launch of the library is bracketed
// by launch_begin / launch_end, which count launches and, when the
// environment variable FROB_DEBUG_SYNC is set to 1, log each launch to stderr,
// synchronise the stream after it and log the CUDA status.
// When profiling is on (frob_profile_enable), launch_begin / launch_end also
// record a CUDA event pair on the launching stream, so that per-kernel device
// time can be read back with frob_profile_report.
void launch_begin(const char* name, cudaStream_t st);
void launch_end(const char* name, cudaStream_t st);
// The algorithmic flops of the next launch of this host thread (2 M N K for
// a product, over the tiles it computes), kept in its profile record and
// summed per kernel variant by frob_profile_report; 0 when not set.
void set_launch_flops(double flops);
// cudaFuncSetAttribute(kernel, MaxDynamicSharedMemorySize, bytes) once per
// (kernel, device, bytes): the attribute belongs to the function on the
// current device, so a process that drives several GPUs sets it on each.
inline bool smem_attr_needed(const void* fn, int bytes) {
  static std::mutex mu;
  static std::set<std::tuple<const void*, int, int>> seen;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  return seen.insert(std::make_tuple(fn, dev, bytes)).second;
}
template <typename F> inline void set_smem_attr(F* kernel, int bytes) {
  if (smem_attr_needed(reinterpret_cast<const void*>(kernel), bytes))
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

// SMs that persistent kernels launched by this host thread leave free (a
// panel factorization running beside them on another stream), and the grid
// of such a kernel: at most one CTA per tile and per remaining SM.
inline thread_local int t_sm_reserve = 0;
inline unsigned persistent_grid(int64_t tiles) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int avail = sms - t_sm_reserve;
  if (avail < 1) avail = 1;
  return (unsigned)(tiles < avail ? tiles : avail);
}

// Scope of an SM reservation (restores the previous value).
class SmReserve {
 public:
  explicit SmReserve(int n) : prev_(t_sm_reserve) { t_sm_reserve = n; }
  ~SmReserve() { t_sm_reserve = prev_; }
  SmReserve(const SmReserve&) = delete;
  SmReserve& operator=(const SmReserve&) = delete;

 private:
  int prev_;
};

// Element-wise GEMM epilogues applied to W consecutive columns j0 .. j0 + W - 1
// of row i (those below ncols): a functor with a row<W>() method (kRow) reads
// every input of the W elements before it writes any, so that the loads are
// in flight together; other functors are called element by element.
template <class E, class = void> struct epi_has_row : std::false_type {};
template <class E> struct epi_has_row<E, std::void_t<decltype(E::kRow)>> : std::true_type {};

template <int W, class Epi, typename T>
__device__ __forceinline__ void epi_row(const Epi& epi, int b, int i, int j0, const T (&v)[W], int ncols) {
  if constexpr (epi_has_row<Epi>::value) {
    epi.template row<W>(b, i, j0, v, ncols);
  } else {
#pragma unroll
    for (int q = 0; q < W; ++q)
      if (j0 + q < ncols) epi(b, i, j0 + q, v[q]);
  }
}

#define FROB_LAUNCH(NAME, ST, ...)    \
  do {                                \
    ::frob::launch_begin(NAME, ST);   \
    __VA_ARGS__;                      \
    ::frob::launch_end(NAME, ST);     \
  } while (0)

template <typename T> constexpr const char* type_tag();
template <> constexpr const char* type_tag<double>() { return "f64"; }
template <> constexpr const char* type_tag<float>() { return "f32"; }
template <> constexpr const char* type_tag<zd>() { return "c128"; }
template <> constexpr const char* type_tag<zf>() { return "c64"; }

// Per-matrix status written by the kernels (first failure wins).
__device__ __forceinline__ void report(frob_info* info, int b, int status, int bad_index) {
  if (info == nullptr) return;
  frob_info* f = info + b;
  if (f->status == FROB_OK) {
    f->status = status;
    f->bad_index = bad_index;
  }
}

}  // namespace frob
