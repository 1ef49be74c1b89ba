// Mixed-precision Frobenius inversion with Newton-Schulz refinement.
//
//   X_0      = Frobenius inversion of M in FP32 (Sec. 4.1, on the CUDA cores);
//              for the control runs, complex LU / Cholesky inversion in FP32
//              instead (the refinement below is the same for both starts)
//   repeat:  R = I - M X        FP64-accurate (digit-split products on the
//                               BF16 tensor cores, ozaki.cuh)
//            stop when ||R||_F / (||M||_F ||X||_F) <= tol
//            X <- X + X R       (4 digits per operand in the first
//                               correction, 5 after it: see S_CORR)
//
// X is kept in FP64 (planes X and X^T, so that both products only ever split
// rows).  Matrices that have converged, or whose FP32 inversion failed, are
// skipped by every later kernel through a per-matrix flag, so the loop needs
// no host synchronisation and a fixed launch sequence.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include "../../include/frobinv.h"
#include "common.cuh"
#include "ops.h"
#include "ozaki.cuh"

namespace frob {
namespace mixed {

// Digits of M and X in the residual I - M X.  A computed residual R~_k =
// R_k + E_k feeds the next one as R_{k+1} = R_k^2 - E_k + R_k E_k, so the
// error of every residual but the first bounds what the refinement can reach.
// Seven digits (pairs s + t <= 8) leave dropped terms of weight 2^-63 times
// the row and column scales: a relative residual floor near 1e-16 for
// matrices whose entries are alike in size, and up to about 1e-14 when a
// large diagonal sets the row scale (Hermitian positive definite input with a
// wide spectrum).  Eight digits (pairs s + t <= 9) lower that floor by 2^7 and
// are used when the requested tolerance is below 1e-14.
constexpr int S_RESID = 7;
constexpr int S_RESID_FINE = 8;
constexpr int S_RESID_FIRST = 5;  // the first residual's error adds to ||R_0||^2: 2^-36 suffices
// The correction X R is computed from S_CORR-digit splits of X and R (pairs
// s + t <= S_CORR + 1), a relative error near 2^(-7 S_CORR - 1) of X R, so the
// next residual is R^2 + O(2^(-7 S_CORR - 1) ||R||).  Four digits suffice for
// the first correction (||R_0|| ~ FP32 accuracy, R_0^2 dominates); later
// ones use five, or the 2^-29 ||R_1|| term would stall the relative residual
// near 1e-14.
constexpr int S_CORR = 5;
constexpr int S_CORR_FIRST = 4;

namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    tried = true;
  }
  return fn;
}

// digits [2][S][batch][n][Kp] BF16 as a rank-3 map (Kp, n, 2 S batch)
bool digit_map(CUtensorMap* map, const __nv_bfloat16* ptr, int n, int Kp, int S, int batch, int box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)n, (cuuint64_t)(2 * S * batch)};
  cuuint64_t strides[2] = {(cuuint64_t)Kp * 2, (cuuint64_t)n * Kp * 2};
  cuuint32_t box[3] = {(cuuint32_t)oz::KB, (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<__nv_bfloat16*>(ptr), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Precision conversions with integer operations (this GPU's FP64 unit, which
// also converts, retires about two lanes per clock per SM).
// FP64 -> FP32, round to nearest even; magnitudes below the FP32 normal range
// flush to zero, above it saturate to infinity; NaN stays NaN.
__device__ __forceinline__ float d2f_int(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const unsigned sign = (unsigned)(u >> 32) & 0x80000000u;
  const int ex = (int)((u >> 52) & 0x7FF);
  const unsigned long long m = u & 0xFFFFFFFFFFFFFull;
  if (ex == 0x7FF) return __uint_as_float(sign | 0x7F800000u | (m ? 0x400000u : 0u));
  const int e = ex - 1023 + 127;
  if (e <= 0) return __uint_as_float(sign);
  const unsigned q = (unsigned)(m >> 29);
  const unsigned long long rem = m & 0x1FFFFFFFull;
  unsigned bits = e >= 255 ? 0x7F800000u : (((unsigned)e << 23) + q);
  if (e < 255 && (rem > 0x10000000ull || (rem == 0x10000000ull && (q & 1u)))) bits += 1;  // a carry bumps the exponent
  if (bits > 0x7F800000u) bits = 0x7F800000u;
  return __uint_as_float(sign | bits);
}
// FP32 -> FP64, exact (FP32 subnormals flush to zero).
__device__ __forceinline__ double f2d_int(float x) {
  const unsigned u = __float_as_uint(x);
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  const unsigned e = (u >> 23) & 0xFFu;
  const unsigned long long m = u & 0x7FFFFFu;
  if (e == 0) return __longlong_as_double((long long)sign);
  const unsigned long long de = e == 0xFFu ? 0x7FFull : (unsigned long long)(e - 127 + 1023);
  return __longlong_as_double((long long)(sign | (de << 52) | (m << 29)));
}

// M (c128) -> M32 (c64) and FP64 planes [2][batch][n][n]; ||M||_F^2 per
// matrix (FP32 partial sums, one atomic per block)
__global__ void conv_in_kernel(int n, MatB<const zd> M, MatB<zf> M32, double* Mp, double* nM2, int hpd) {
  const int b = blockIdx.z;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nn = (int64_t)n * n;
  float ss = 0.f;
  if (e < nn) {
    const int i = (int)(e / n), j = (int)(e % n);
    zd v;
    if (!hpd || i > j) {
      v = M.at(b)[(int64_t)i * M.ld + j];
    } else if (i == j) {
      v = zd{M.at(b)[(int64_t)i * M.ld + j].x, 0.0};  // Hermitian: real diagonal
    } else {
      const zd w = M.at(b)[(int64_t)j * M.ld + i];   // upper triangle from the lower one
      v = zd{w.x, -w.y};
    }
    const zf v32{d2f_int(v.x), d2f_int(v.y)};
    M32.at(b)[(int64_t)i * M32.ld + j] = v32;
    Mp[(int64_t)b * nn + e] = v.x;
    Mp[((int64_t)gridDim.z + b) * nn + e] = v.y;
    ss = fmaf(v32.x, v32.x, v32.y * v32.y);
  }
  for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
  __shared__ float part[32];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = ss;
  __syncthreads();
  if (threadIdx.x < 32) {
    float w = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.f;
    for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
    if (threadIdx.x == 0 && w != 0.f) atomicAdd(nM2 + b, (double)w);
  }
}

// X32 (c64) -> planes X, X^T (FP64)
__global__ void conv_x_kernel(int n, MatB<const zf> X32, double* Xp, double* XTp, int batch) {
  const int b = blockIdx.z;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nn = (int64_t)n * n;
  if (e >= nn) return;
  const int i = (int)(e / n), j = (int)(e % n);
  const zf v = X32.at(b)[(int64_t)i * X32.ld + j];
  const double re = f2d_int(v.x), im = f2d_int(v.y);
  Xp[(int64_t)b * nn + e] = re;
  Xp[((int64_t)batch + b) * nn + e] = im;
  XTp[(int64_t)b * nn + (int64_t)j * n + i] = re;
  XTp[((int64_t)batch + b) * nn + (int64_t)j * n + i] = im;
}

// planes X -> interleaved c128 output
__global__ void conv_out_kernel(int n, const double* Xp, MatB<zd> X, int batch) {
  const int b = blockIdx.z;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nn = (int64_t)n * n;
  if (e >= nn) return;
  const int i = (int)(e / n), j = (int)(e % n);
  X.at(b)[(int64_t)i * X.ld + j] = zd{Xp[(int64_t)b * nn + e], Xp[((int64_t)batch + b) * nn + e]};
}

// ||X||_F^2 per matrix into nX2.  FP32 is ample for the norm in a relative
// residual and keeps the work off the FP64 pipe; each block reduces 16
// elements per thread before a single atomic.
constexpr int XN_PER_THREAD = 16;
__global__ void xnorm_kernel(int n, const double* Xp, double* nX2, int batch, const int* skip) {
  const int b = blockIdx.z;
  if (skip[b]) return;
  const int64_t nn = (int64_t)n * n;
  const int64_t e0 = (int64_t)blockIdx.x * blockDim.x * XN_PER_THREAD + threadIdx.x;
  float ss = 0.f;
  for (int k = 0; k < XN_PER_THREAD; ++k) {
    const int64_t e = e0 + (int64_t)k * blockDim.x;
    if (e < nn) {
      const float a = d2f_int(Xp[(int64_t)b * nn + e]), c = d2f_int(Xp[((int64_t)batch + b) * nn + e]);
      ss = fmaf(a, a, fmaf(c, c, ss));
    }
  }
  for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
  __shared__ float part[32];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = ss;
  __syncthreads();
  if (threadIdx.x < 32) {
    float v = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.f;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0 && v != 0.f) atomicAdd(nX2 + b, (double)v);
  }
}

__global__ void zero_kernel(double* a, double* c, int batch, const int* skip) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < batch && !skip[b]) {
    a[b] = 0.0;
    c[b] = 0.0;
  }
}

// skip matrices whose FP32 inversion failed
__global__ void init_skip_kernel(const frob_info* info, int* skip, int batch) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < batch) skip[b] = info[b].status != FROB_OK;
}

// relative residual, convergence and iteration bookkeeping
__global__ void check_kernel(int batch, int it, int last, double tol, const double* rn2, const double* nM2,
                             const double* nX2, int* skip, frob_info* info) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch || skip[b]) return;
  const double res = sqrt(rn2[b]) / (sqrt(nM2[b]) * sqrt(nX2[b]));
  info[b].residual = res;
  info[b].ns_iters = it;
  if (res <= tol) {
    skip[b] = 1;
  } else if (last || !(res < 0.5)) {
    // not converged within the budget, or the start was too poor for the
    // iteration to contract (rho(I - M X_0) must be below 1)
    info[b].status = FROB_ERR_NOT_CONVERGED;
    skip[b] = 1;
  }
}

// The digit products, persistent: one CTA per SM (the shared memory admits
// no second), at most one per tile.
template <int MODE>
void launch_cgemm(const CUtensorMap& ma, const CUtensorMap& mb, const oz::OzArgs& a, cudaStream_t st) {
  set_smem_attr(oz::oz_cgemm_kernel<MODE>, oz::SMEM_BYTES);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t tiles =
      (int64_t)((a.n + oz::BN - 1) / oz::BN) * ((a.n + tc::BM - 1) / tc::BM) * 2 * a.batch;
  const unsigned grid = (unsigned)(tiles < sms ? tiles : (sms > 0 ? sms : 1));
  FROB_LAUNCH(MODE == oz::RESID ? "oz_cgemm<resid>" : "oz_cgemm<corr>", st,
              oz::oz_cgemm_kernel<MODE><<<grid, oz::THREADS, oz::SMEM_BYTES, st>>>(ma, mb, a));
}

void launch_split(int n, int Kp, int batch, int S, const double* src, __nv_bfloat16* dst, int* exps,
                  const int* skip, cudaStream_t st) {
  const int64_t warps = (int64_t)batch * n;  // one warp per (real, imaginary) row pair
  const int threads = 256;
  const unsigned blocks = (unsigned)((warps * 32 + threads - 1) / threads);
  const int64_t nn = (int64_t)n * n, ps = (int64_t)batch * n * n;
#define FROB_SPLIT_S(SV)                                                                                        \
  FROB_LAUNCH("oz_split", st,                                                                                  \
              oz::oz_split_rows_kernel<SV><<<blocks, threads, 0, st>>>(n, n, Kp, batch, src, n, nn, ps, dst, exps, \
                                                                         skip))
  switch (S) {  // the digit counts this driver uses
    case S_CORR: FROB_SPLIT_S(S_CORR); break;
    case S_RESID: FROB_SPLIT_S(S_RESID); break;
    case S_RESID_FINE: FROB_SPLIT_S(S_RESID_FINE); break;
    default: break;
  }
#undef FROB_SPLIT_S
}

struct Layout {
  zf *M32, *X32;
  void* ws32;
  double *Mp, *Xp, *XTp, *RTp;
  __nv_bfloat16 *Mdig, *Xdig, *Bdig;
  int *expM, *expX, *expB;
  double *rn2, *nM2, *nX2;
  int *skip, *err;
  size_t bytes;
};

Layout carve(int n, int batch, void* ws) {
  Layout L{};
  unsigned char* base = static_cast<unsigned char*>(ws);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    void* p = base ? base + off : nullptr;
    off += (bytes + 255) & ~(size_t)255;
    return p;
  };
  const size_t nn = (size_t)n * n;
  const int Kp = (n + oz::KP_ALIGN - 1) / oz::KP_ALIGN * oz::KP_ALIGN;
  L.M32 = static_cast<zf*>(take(nn * batch * sizeof(zf)));
  L.X32 = static_cast<zf*>(take(nn * batch * sizeof(zf)));
  // the FP32 start runs without tensor-core products (TcOff below): its
  // workspace ends with their scratch, which is left out
  const size_t tcb = tc_scratch_for(n, batch);
  size_t w32 = frob_lu_ws<float>(n, batch, nullptr, nullptr) - tcb;
  w32 = std::max(w32, frob_chol_ws<float>(n, batch, nullptr, nullptr) - tcb);
  w32 = std::max(w32, cplx_lu_ws<zf>(n, batch, nullptr, nullptr));
  w32 = std::max(w32, cplx_chol_ws<zf>(n, batch, nullptr, nullptr));
  L.ws32 = take(w32);
  L.Mp = static_cast<double*>(take(2 * nn * batch * 8));
  L.Xp = static_cast<double*>(take(2 * nn * batch * 8));
  L.XTp = static_cast<double*>(take(2 * nn * batch * 8));
  L.RTp = static_cast<double*>(take(2 * nn * batch * 8));
  const size_t dig = (size_t)2 * oz::S_MAX * batch * n * Kp * 2;
  L.Mdig = static_cast<__nv_bfloat16*>(take(dig));
  L.Xdig = static_cast<__nv_bfloat16*>(take(dig));
  L.Bdig = static_cast<__nv_bfloat16*>(take(dig));
  L.expM = static_cast<int*>(take((size_t)2 * batch * n * 4));
  L.expX = static_cast<int*>(take((size_t)2 * batch * n * 4));
  L.expB = static_cast<int*>(take((size_t)2 * batch * n * 4));
  L.rn2 = static_cast<double*>(take((size_t)batch * 8));
  L.nM2 = static_cast<double*>(take((size_t)batch * 8));
  L.nX2 = static_cast<double*>(take((size_t)batch * 8));
  L.skip = static_cast<int*>(take((size_t)batch * 4));
  L.err = static_cast<int*>(take(256));
  L.bytes = off;
  return L;
}

}  // namespace

size_t mixed_ws(int n, int batch) { return carve(n, batch, nullptr).bytes; }

frob_status mixed_run(int n, int batch, MatB<const zd> M, MatB<zd> X, const frob_opts& o, void* ws, frob_info* info,
                      cudaStream_t st, bool hpd, bool complex_start) {
  if (n > oz::K_MAX) return FROB_ERR_UNSUPPORTED;
  Layout L = carve(n, batch, ws);
  const int Kp = (n + oz::KP_ALIGN - 1) / oz::KP_ALIGN * oz::KP_ALIGN;
  const int64_t nn = (int64_t)n * n;
  const dim3 eg((unsigned)((nn + 255) / 256), 1, batch);
  const double tol = o.ns_tol > 0 ? o.ns_tol : 1e-14;
  const int max_iter = o.ns_max_iter > 0 ? o.ns_max_iter : 8;

  cudaMemsetAsync(L.nM2, 0, (size_t)batch * 8, st);
  cudaMemsetAsync(L.err, 0, 4, st);
  FROB_LAUNCH("mixed_conv_in", st,
              conv_in_kernel<<<eg, 256, 0, st>>>(n, M, MatB<zf>{L.M32, n, nn}, L.Mp, L.nM2, hpd ? 1 : 0));
  // X_0: Frobenius inversion in FP32, with LU (Sec. 4.1) or, for Hermitian
  // positive definite input, with Cholesky (Sec. 4.3); or, for the control,
  // complex LU / Cholesky inversion in FP32; also initialises info
  frob_opts o32 = o;
  o32.prec = FROB_FP32;
  const MatB<const zf> M32{L.M32, n, nn};
  const MatB<zf> X32{L.X32, n, nn};
  TcOff no_tensor_core_start;
  if (complex_start && hpd)
    cplx_chol_run<zf>(n, batch, M32, X32, L.ws32, info, st);
  else if (complex_start)
    cplx_lu_run<zf>(n, batch, M32, X32, L.ws32, info, st);
  else if (hpd)
    frob_chol_run<float>(n, batch, M32, X32, L.ws32, info, st);
  else
    frob_lu_run<float>(n, batch, M32, X32, o32, L.ws32, info, st);
  FROB_LAUNCH("mixed_conv_x", st, conv_x_kernel<<<eg, 256, 0, st>>>(n, MatB<const zf>{L.X32, n, nn}, L.Xp, L.XTp, batch));
  FROB_LAUNCH("mixed_init_skip", st, init_skip_kernel<<<(batch + 127) / 128, 128, 0, st>>>(info, L.skip, batch));
  const int s_resid = tol < 1e-14 ? S_RESID_FINE : S_RESID;
  launch_split(n, Kp, batch, s_resid, L.Mp, L.Mdig, L.expM, L.skip, st);

  CUtensorMap mapM, mapXTr, mapXc, mapRTc;
  if (!digit_map(&mapM, L.Mdig, n, Kp, s_resid, batch, tc::BM) ||
      !digit_map(&mapXTr, L.Bdig, n, Kp, s_resid, batch, oz::BN) ||
      !digit_map(&mapXc, L.Xdig, n, Kp, S_CORR, batch, tc::BM) ||
      !digit_map(&mapRTc, L.Bdig, n, Kp, S_CORR, batch, oz::BN))
    return FROB_ERR_CUDA;

  oz::OzArgs ra{};
  ra.n = n;
  ra.Kp = Kp;
  ra.batch = batch;
  ra.S = s_resid;
  ra.Su = s_resid;
  ra.expA = L.expM;
  ra.expB = L.expB;
  ra.outR = L.RTp;
  ra.rnorm2 = L.rn2;
  ra.skip = L.skip;
  ra.err = L.err;
  oz::OzArgs ca = ra;
  ca.S = S_CORR;
  ca.Su = S_CORR;
  ca.expA = L.expX;
  ca.X = L.Xp;
  ca.XT = L.XTp;

  for (int it = 0; it <= max_iter; ++it) {
    FROB_LAUNCH("mixed_zero", st, zero_kernel<<<(batch + 127) / 128, 128, 0, st>>>(L.rn2, L.nX2, batch, L.skip));
    const dim3 xg((unsigned)((nn + 256 * XN_PER_THREAD - 1) / (256 * XN_PER_THREAD)), 1, batch);
    FROB_LAUNCH("mixed_xnorm", st, xnorm_kernel<<<xg, 256, 0, st>>>(n, L.Xp, L.nX2, batch, L.skip));
    launch_split(n, Kp, batch, s_resid, L.XTp, L.Bdig, L.expB, L.skip, st);
    ra.Su = it == 0 ? S_RESID_FIRST : s_resid;
    launch_cgemm<oz::RESID>(mapM, mapXTr, ra, st);                                   // R = I - M X
    FROB_LAUNCH("mixed_check", st,
                check_kernel<<<(batch + 127) / 128, 128, 0, st>>>(batch, it, it == max_iter, tol, L.rn2, L.nM2, L.nX2,
                                                                  L.skip, info));
    if (it == max_iter) break;
    launch_split(n, Kp, batch, S_CORR, L.Xp, L.Xdig, L.expX, L.skip, st);
    launch_split(n, Kp, batch, S_CORR, L.RTp, L.Bdig, L.expB, L.skip, st);
    ca.Su = it == 0 ? S_CORR_FIRST : S_CORR;
    launch_cgemm<oz::CORR>(mapXc, mapRTc, ca, st);                                   // X <- X + X R
  }
  FROB_LAUNCH("mixed_conv_out", st, conv_out_kernel<<<eg, 256, 0, st>>>(n, L.Xp, X, batch));
  return cudaGetLastError() == cudaSuccess ? FROB_OK : FROB_ERR_CUDA;
}

}  // namespace mixed
}  // namespace frob
