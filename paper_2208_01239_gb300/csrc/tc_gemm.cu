// Host side of the tensor-core GEMM: operand conversion (FP32 -> BF16 or
// TF32, round to nearest, K-major with a 16-byte aligned row pitch), TMA
// tensor maps, launch, and the C-ABI entry point frob_gemm_tc.
#include <cstdint>
#include <cstring>
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <mutex>

#include "../../include/frobinv.h"
#include "common.cuh"
#include "tc_gemm.cuh"
#include "ops.h"

namespace frob {
namespace tc {

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

// rank-3 map over [batch][rows][K] with row pitch `pitch` elements
bool make_map(CUtensorMap* map, const void* ptr, int kind, int K, int rows, int batch, int64_t pitch,
              int64_t bpitch, int box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  const int elem = kind == 0 ? 2 : 4;
  cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)batch};
  cuuint64_t strides[2] = {(cuuint64_t)(pitch * elem), (cuuint64_t)(bpitch * elem)};
  cuuint32_t box[3] = {(cuuint32_t)(BK_BYTES / elem), (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(map, kind == 0 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_TFLOAT32, 3,
                  const_cast<void*>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// src (rows x K, row-major, ld) -> dst (rows x pitch), BF16 or TF32-rounded FP32
template <int KIND>
__global__ void convert_kernel(int rows, int K, const float* src, int64_t ld, int64_t sb, void* dst, int64_t pitch) {
  const int b = blockIdx.z;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)rows * pitch) return;
  const int r = (int)(e / pitch), k = (int)(e % pitch);
  const float v = k < K ? src[(int64_t)b * sb + (int64_t)r * ld + k] : 0.f;
  const int64_t o = (int64_t)b * rows * pitch + e;
  if (KIND == 0)
    static_cast<__nv_bfloat16*>(dst)[o] = __float2bfloat16_rn(v);
  else
    static_cast<float*>(dst)[o] = to_tf32(v);
}

template <int KIND, int BN, int STAGES, class Epi>
cudaError_t launch(const CUtensorMap& ma, const CUtensorMap& mb, int M, int N, int K, int batch, Epi epi, int* err,
                   cudaStream_t st) {
  using S = TcSmem<BN, STAGES>;
  set_smem_attr(tc_gemm_kernel<KIND, BN, STAGES, Epi>, S::BYTES);
  // persistent: one CTA per SM (the shared memory admits no second), at most one per tile
  const int64_t tiles = (int64_t)((N + BN - 1) / BN) * ((M + BM - 1) / BM) * batch;
  if (tiles > INT32_MAX) return cudaErrorInvalidValue;  // the kernel counts tiles in int
  const unsigned grid = persistent_grid(tiles);
  FROB_LAUNCH(KIND == 0 ? "tc_gemm<bf16>" : "tc_gemm<tf32>", st,
              tc_gemm_kernel<KIND, BN, STAGES, Epi><<<grid, NUM_THREADS, S::BYTES, st>>>(ma, mb, M, N, K, batch, epi,
                                                                                           err));
  return cudaGetLastError();
}

// Split-TF32 operand rows (see tc3_prepare): dst[b][r][blk * Kp + k] for the
// three blocks, from the element (r, k) of the source, src[r * ld + k] or,
// with trans, src[k * ld + r]; k in [K, Kp) is written as zero.  32 x 32
// tiles through shared memory, so both the source and the destination are
// read / written along their contiguous dimension.  pattern 0 (A operand):
// hi, hi, lo; pattern 1 (B operand): hi, lo, hi.
__global__ void __launch_bounds__(256) split3_kernel(int R, int K, int64_t Kp, const float* src, int64_t ld,
                                                     int64_t sb, int trans, int pattern, float* dst) {
  __shared__ float tile[32][33];
  const int b = blockIdx.z;
  const int r0 = blockIdx.y * 32, k0 = blockIdx.x * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  const float* sbp = src + (int64_t)b * sb;
  for (int i = ty; i < 32; i += 8) {
    if (trans) {  // tile[k][r] from source row k0 + i, columns r0 + tx
      const int k = k0 + i, r = r0 + tx;
      tile[i][tx] = (k < K && r < R) ? sbp[(int64_t)k * ld + r] : 0.f;
    } else {      // tile[r][k] from source row r0 + i, columns k0 + tx
      const int r = r0 + i, k = k0 + tx;
      tile[i][tx] = (k < K && r < R) ? sbp[(int64_t)r * ld + k] : 0.f;
    }
  }
  __syncthreads();
  float* db = dst + (int64_t)b * R * 3 * Kp;
  for (int i = ty; i < 32; i += 8) {
    const int r = r0 + i, k = k0 + tx;
    if (r >= R || k >= Kp) continue;
    const float x = trans ? tile[tx][i] : tile[i][tx];
    const float hi = to_tf32(x);
    const float lo = to_tf32(x - hi);
    float* row = db + (int64_t)r * 3 * Kp;
    row[k] = hi;
    row[Kp + k] = pattern == 0 ? hi : lo;
    row[2 * Kp + k] = pattern == 0 ? lo : hi;
  }
}

}  // namespace

int64_t tc3_kp(int K) { return ((int64_t)K + 3) / 4 * 4; }

size_t tc3_scratch_bytes(int M, int N, int K, int batch) {
  const int64_t kp = tc3_kp(K);
  auto a256 = [](size_t x) { return (x + 255) & ~(size_t)255; };
  return 256 + a256((size_t)batch * M * 3 * kp * 4) + a256((size_t)batch * N * 3 * kp * 4);
}

bool tc3_prepare(int M, int N, int K, int batch, const float* A, int64_t lda, int64_t sa, bool transA,
                 const float* B, int64_t ldb, int64_t sb, bool transB, void* scratch, CUtensorMap* ma,
                 CUtensorMap* mb, cudaStream_t st) {
  const int64_t kp = tc3_kp(K);
  unsigned char* base = static_cast<unsigned char*>(scratch) + 256;
  float* wa = reinterpret_cast<float*>(base);
  float* wb = reinterpret_cast<float*>(base + (((size_t)batch * M * 3 * kp * 4 + 255) & ~(size_t)255));
  const dim3 ga((unsigned)((kp + 31) / 32), (unsigned)((M + 31) / 32), (unsigned)batch);
  const dim3 gb((unsigned)((kp + 31) / 32), (unsigned)((N + 31) / 32), (unsigned)batch);
  FROB_LAUNCH("tc_split3", st, split3_kernel<<<ga, 256, 0, st>>>(M, K, kp, A, lda, sa, transA ? 1 : 0, 0, wa));
  FROB_LAUNCH("tc_split3", st, split3_kernel<<<gb, 256, 0, st>>>(N, K, kp, B, ldb, sb, transB ? 1 : 0, 1, wb));
  return make_map(ma, wa, 1, (int)(3 * kp), M, batch, 3 * kp, (int64_t)M * 3 * kp, BM) &&
         make_map(mb, wb, 1, (int)(3 * kp), N, batch, 3 * kp, (int64_t)N * 3 * kp, 256);
}

int64_t pitch_for(int kind, int K) {
  const int q = kind == 0 ? 8 : 4;  // 16 bytes
  return ((int64_t)K + q - 1) / q * q;
}

size_t gemm_tc_ws(int kind, int M, int N, int K, int batch) {
  const int64_t p = pitch_for(kind, K);
  const size_t elem = kind == 0 ? 2 : 4;
  auto a256 = [](size_t x) { return (x + 255) & ~(size_t)255; };
  return a256((size_t)batch * M * p * elem) + a256((size_t)batch * N * p * elem) + 256;
}

}  // namespace tc

size_t tc_scratch_for(int n, int batch) {
  return n >= tc::TC3_MIN_K ? tc::tc3_scratch_bytes(n, n, n, batch) : 0;
}

}  // namespace frob

using namespace frob;

extern "C" frob_status frob_gemm_tc(int kind, int M, int N, int K, int batch, const float* A, int64_t lda, int64_t sa,
                                    const float* B, int64_t ldb, int64_t sb, float* C, int64_t ldc, int64_t sc,
                                    void* ws, size_t wsb, int* err, void* stream) {
  if ((kind != 0 && kind != 1) || M < 1 || N < 1 || K < 1 || batch < 1 || batch > 65535) return FROB_ERR_ARG;
  if (!A || !B || !C || !err || lda < K || ldb < K || ldc < N) return FROB_ERR_ARG;
  const size_t need = tc::gemm_tc_ws(kind, M, N, K, batch);
  if (!ws || wsb < need || (reinterpret_cast<uintptr_t>(ws) & 255)) return FROB_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t p = tc::pitch_for(kind, K);
  const size_t elem = kind == 0 ? 2 : 4;
  unsigned char* wa = static_cast<unsigned char*>(ws);
  unsigned char* wb = wa + (((size_t)batch * M * p * elem + 255) & ~(size_t)255);
  {
    dim3 ga((unsigned)(((int64_t)M * p + 255) / 256), 1, batch), gb((unsigned)(((int64_t)N * p + 255) / 256), 1, batch);
    if (kind == 0) {
      FROB_LAUNCH("tc_convert<bf16>", st, tc::convert_kernel<0><<<ga, 256, 0, st>>>(M, K, A, lda, sa, wa, p));
      FROB_LAUNCH("tc_convert<bf16>", st, tc::convert_kernel<0><<<gb, 256, 0, st>>>(N, K, B, ldb, sb, wb, p));
    } else {
      FROB_LAUNCH("tc_convert<tf32>", st, tc::convert_kernel<1><<<ga, 256, 0, st>>>(M, K, A, lda, sa, wa, p));
      FROB_LAUNCH("tc_convert<tf32>", st, tc::convert_kernel<1><<<gb, 256, 0, st>>>(N, K, B, ldb, sb, wb, p));
    }
  }
  CUtensorMap ma, mb;
  if (!tc::make_map(&ma, wa, kind, K, M, batch, p, (int64_t)M * p, tc::BM) ||
      !tc::make_map(&mb, wb, kind, K, N, batch, p, (int64_t)N * p, 256))
    return FROB_ERR_CUDA;
  tc::TcEpiStoreF32 epi{C, ldc, sc, 1.f, 0.f};
  // 128 x 256 output tiles: the widest UMMA N for cta_group::1; persistent
  // CTAs with two TMEM accumulators overlap each tile's epilogue with the
  // next tile's main loop
  cudaError_t e = kind == 0 ? tc::launch<0, 256, 4>(ma, mb, M, N, K, batch, epi, err, st)
                            : tc::launch<1, 256, 4>(ma, mb, M, N, K, batch, epi, err, st);
  return e == cudaSuccess ? FROB_OK : FROB_ERR_CUDA;
}

extern "C" size_t frob_gemm_tc_workspace_bytes(int kind, int M, int N, int K, int batch) {
  if ((kind != 0 && kind != 1) || M < 1 || N < 1 || K < 1 || batch < 1) return 0;
  return frob::tc::gemm_tc_ws(kind, M, N, K, batch);
}
