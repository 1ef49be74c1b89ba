// Host side of the FP64-accurate real products on the BF16 tensor cores
// (ozr.cuh): the exponent kernel, the digit split of both operands into the
// caller's scratch, the TMA tensor maps and the kernel arguments.
#include <cstdint>
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <mutex>

#include "../../include/frobinv.h"
#include "common.cuh"
#include "ozr.cuh"

namespace frob {
namespace ozr {

namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// digits [S][batch][rows][Kp] BF16 as a rank-3 map (Kp, rows, S batch), boxes
// of 64 K x box_rows rows, 128-byte swizzle
bool digit_map(CUtensorMap* map, const __nv_bfloat16* ptr, int rows, int Kp, int S, int batch, int box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)rows, (cuuint64_t)(S * batch)};
  cuuint64_t strides[2] = {(cuuint64_t)Kp * 2, (cuuint64_t)rows * Kp * 2};
  cuuint32_t box[3] = {(cuuint32_t)oz::KB, (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<__nv_bfloat16*>(ptr), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// e_r of the logical R x K matrix X (element (r, k) = src[r ld + k], or
// src[k ld + r] with trans): the smallest integer with max_k |X_rk| < 2^e_r
// (0 for an all-zero row, after ozr_exp_final), from the FP64 bit patterns;
// NONFINITE_EXP when the row holds an infinity or a NaN.  Partial maxima of
// the bit patterns (non-negative doubles, infinities and NaNs above every
// finite value, order as unsigned integers) are combined with atomicMax into
// mx[b][r] (zeroed first).  !trans: one warp per row; trans: 32 x 8 threads
// per 32 consecutive r and a 256-row slice of k, consecutive threads on
// consecutive addresses.
__global__ void __launch_bounds__(256) ozr_absmax_kernel(int R, int K, int batch, const double* src, int64_t ld,
                                                         int64_t sb, int trans, unsigned long long* mx) {
  if (!trans) {
    const int64_t item = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (item >= (int64_t)R * batch) return;
    const int lane = threadIdx.x & 31;
    const int b = (int)(item / R), r = (int)(item % R);
    const double* row = src + (int64_t)b * sb + (int64_t)r * ld;
    unsigned long long m = 0;
    for (int k = lane; k < K; k += 32) {
      const unsigned long long a = (unsigned long long)__double_as_longlong(row[k]) & 0x7FFFFFFFFFFFFFFFull;
      m = a > m ? a : m;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long other = __shfl_xor_sync(0xffffffffu, m, o);
      m = other > m ? other : m;
    }
    if (lane == 0) mx[item] = m;
    return;
  }
  __shared__ unsigned long long red[8][32];
  const int b = blockIdx.z;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int r = blockIdx.x * 32 + tx;
  const int k0 = blockIdx.y * 256;
  unsigned long long m = 0;
  if (r < R) {
    const double* col = src + (int64_t)b * sb + r;
    const int k1 = k0 + 256 < K ? k0 + 256 : K;
    for (int k = k0 + ty; k < k1; k += 8) {
      const unsigned long long a = (unsigned long long)__double_as_longlong(col[(int64_t)k * ld]) & 0x7FFFFFFFFFFFFFFFull;
      m = a > m ? a : m;
    }
  }
  red[ty][tx] = m;
  __syncthreads();
  if (ty == 0 && r < R) {
#pragma unroll
    for (int i = 1; i < 8; ++i) m = red[i][tx] > m ? red[i][tx] : m;
    if (m != 0) atomicMax(mx + (int64_t)b * R + r, m);
  }
}

// exps[i] from the maxima: 0 for zero, NONFINITE_EXP for infinities / NaNs;
// mx[i] is zeroed for the digit kernel's sums of squares
__global__ void ozr_exp_final_kernel(int64_t count, unsigned long long* mx, int* exps) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const unsigned long long m = mx[i];
  mx[i] = 0;
  const int mex = (int)(m >> 52);
  int e = 0;
  if (mex == 0x7FF) e = NONFINITE_EXP;
  else if (m != 0) e = (mex == 0) ? -1022 : mex - 1022;
  exps[i] = e;
}

}  // namespace

int64_t kp_of(int K) { return ((int64_t)K + oz::KP_ALIGN - 1) / oz::KP_ALIGN * oz::KP_ALIGN; }

size_t scratch_bytes(int M, int N, int K, int batch) {
  const int64_t kp = kp_of(K);
  auto a256 = [](size_t x) { return (x + 255) & ~(size_t)255; };
  return 256 + a256((size_t)S_DIG * batch * M * kp * 2) + a256((size_t)S_DIG * batch * N * kp * 2) +
         a256((size_t)batch * M * 4) + a256((size_t)batch * N * 4) + a256((size_t)batch * (M + N) * 8);
}

bool prepare(int M, int N, int K, int batch, const double* A, int64_t lda, int64_t sa, bool transA,
             const double* B, int64_t ldb, int64_t sb, bool b_rows_are_k_major, void* scratch, int* err,
             CUtensorMap* ma, CUtensorMap* mb, RArgs* args, cudaStream_t st) {
  const int64_t kp = kp_of(K);
  auto a256 = [](size_t x) { return (x + 255) & ~(size_t)255; };
  unsigned char* p = static_cast<unsigned char*>(scratch) + 256;
  __nv_bfloat16* da = reinterpret_cast<__nv_bfloat16*>(p);
  p += a256((size_t)S_DIG * batch * M * kp * 2);
  __nv_bfloat16* db = reinterpret_cast<__nv_bfloat16*>(p);
  p += a256((size_t)S_DIG * batch * N * kp * 2);
  int* ea = reinterpret_cast<int*>(p);
  p += a256((size_t)batch * M * 4);
  int* eb = reinterpret_cast<int*>(p);
  p += a256((size_t)batch * N * 4);
  // [batch][M] then [batch][N]: the maxima' bit patterns, then the digits'
  // sums of squares
  unsigned long long* mxa = reinterpret_cast<unsigned long long*>(p);
  unsigned long long* mxb = mxa + (size_t)batch * M;
  // op(B)'s column j as a K-major row: B[k][j] (transposed read) unless the
  // caller's B already stores op(B)^T row-major
  const int tb = b_rows_are_k_major ? 0 : 1;
  const int ta = transA ? 1 : 0;
  if (kp <= SMALL_KP) {
    // thin operands: exponents, digits and sums of squares in one pass each
    FROB_LAUNCH("ozr_digits", st,
                ozr_digits_small_kernel<S_DIG><<<dim3((unsigned)((M + 31) / 32), (unsigned)batch), 256, 0, st>>>(
                    M, K, batch, A, lda, sa, ta, ea, da, mxa));
    FROB_LAUNCH("ozr_digits", st,
                ozr_digits_small_kernel<S_DIG><<<dim3((unsigned)((N + 31) / 32), (unsigned)batch), 256, 0, st>>>(
                    N, K, batch, B, ldb, sb, tb, eb, db, mxb));
  } else {
    auto exp_grid = [K](int R, int bt, int trans) {
      if (trans) return dim3((unsigned)((R + 31) / 32), (unsigned)((K + 255) / 256), (unsigned)bt);
      return dim3((unsigned)(((int64_t)R * bt * 32 + 255) / 256));
    };
    cudaMemsetAsync(mxa, 0, (size_t)batch * (M + N) * 8, st);
    FROB_LAUNCH("ozr_exp", st,
                ozr_absmax_kernel<<<exp_grid(M, batch, ta), 256, 0, st>>>(M, K, batch, A, lda, sa, ta, mxa));
    FROB_LAUNCH("ozr_exp", st,
                ozr_absmax_kernel<<<exp_grid(N, batch, tb), 256, 0, st>>>(N, K, batch, B, ldb, sb, tb, mxb));
    FROB_LAUNCH("ozr_exp", st,
                ozr_exp_final_kernel<<<(unsigned)(((int64_t)batch * M + 255) / 256), 256, 0, st>>>((int64_t)batch * M,
                                                                                                    mxa, ea));
    FROB_LAUNCH("ozr_exp", st,
                ozr_exp_final_kernel<<<(unsigned)(((int64_t)batch * N + 255) / 256), 256, 0, st>>>((int64_t)batch * N,
                                                                                                    mxb, eb));
    const unsigned gk = (unsigned)((kp + 32 * DIG_KT - 1) / (32 * DIG_KT));
    const dim3 ga(gk, (unsigned)((M + 31) / 32), (unsigned)batch);
    const dim3 gb(gk, (unsigned)((N + 31) / 32), (unsigned)batch);
    FROB_LAUNCH("ozr_digits", st,
                ozr_digits_kernel<S_DIG><<<ga, 256, 0, st>>>(M, K, (int)kp, batch, A, lda, sa, ta, ea, da, mxa));
    FROB_LAUNCH("ozr_digits", st,
                ozr_digits_kernel<S_DIG><<<gb, 256, 0, st>>>(N, K, (int)kp, batch, B, ldb, sb, tb, eb, db, mxb));
  }
  if (!digit_map(ma, da, M, (int)kp, S_DIG, batch, tc::BM) || !digit_map(mb, db, N, (int)kp, S_DIG, batch, oz::BN))
    return false;
  args->M = M;
  args->N = N;
  args->Kp = (int)kp;
  args->batch = batch;
  args->S = S_DIG;
  args->Su = S_DIG;
  args->expA = ea;
  args->expB = eb;
  args->sqA = mxa;
  args->sqB = mxb;
  args->err = err;
  return true;
}

}  // namespace ozr
}  // namespace frob

namespace {
// D = alpha * v + beta * C (C may alias D; not read when beta == 0)
struct EpiAlphaBeta {
  double* D;
  int64_t ldd, sd;
  double alpha, beta;
  __device__ __forceinline__ void operator()(int b, int i, int j, double v) const {
    double* d = D + (int64_t)b * sd + (int64_t)i * ldd + j;
    *d = beta == 0.0 ? alpha * v : alpha * v + beta * *d;
  }
  static constexpr bool kRow = true;
  template <int W>
  __device__ __forceinline__ void row(int b, int i, int j0, const double (&v)[W], int ncols) const {
    double* d = D + (int64_t)b * sd + (int64_t)i * ldd + j0;
    double c[W];
#pragma unroll
    for (int q = 0; q < W; ++q) c[q] = (beta != 0.0 && j0 + q < ncols) ? d[q] : 0.0;
#pragma unroll
    for (int q = 0; q < W; ++q)
      if (j0 + q < ncols) d[q] = beta == 0.0 ? alpha * v[q] : alpha * v[q] + beta * c[q];
  }
};
}  // namespace

using namespace frob;

extern "C" size_t frob_gemm_f64_workspace_bytes(int M, int N, int K, int batch) {
  if (M < ozr::MIN_MN_THIN || N < ozr::MIN_MN_THIN || K < 1 || batch < 1) return 0;
  return ozr::scratch_bytes(M, N, K, batch);
}

extern "C" frob_status frob_gemm_f64(int M, int N, int K, int batch, const double* A, int64_t lda, int64_t sa,
                                     int transA, const double* B, int64_t ldb, int64_t sb, int transB, double* C,
                                     int64_t ldc, int64_t sc, double alpha, double beta, void* ws, size_t wsb,
                                     int* err, void* stream) {
  if (M < ozr::MIN_MN_THIN || N < ozr::MIN_MN_THIN || K < 1 || batch < 1 || batch > 65535 || !A || !B || !C || !err)
    return FROB_ERR_ARG;
  if ((transA != 0 && transA != 1) || (transB != 0 && transB != 1)) return FROB_ERR_ARG;
  if (lda < (transA ? M : K) || ldb < (transB ? K : N) || ldc < N) return FROB_ERR_ARG;
  const size_t need = ozr::scratch_bytes(M, N, K, batch);
  if (!ws || wsb < need || (reinterpret_cast<uintptr_t>(ws) & 255)) return FROB_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  (void)cudaGetLastError();  // an earlier call's pending error is not this call's
  CUtensorMap ma, mb;
  ozr::RArgs ra;
  // op(B)'s columns are B's rows when transB
  if (!ozr::prepare(M, N, K, batch, A, lda, sa, transA != 0, B, ldb, sb, transB != 0, ws, err, &ma, &mb, &ra, st))
    return FROB_ERR_CUDA;
  const cudaError_t e = ozr::launch(ma, mb, ra, EpiAlphaBeta{C, ldc, sc, alpha, beta}, st);
  return e == cudaSuccess ? FROB_OK : FROB_ERR_CUDA;
}
