// Tensor-core GEMM for sm_103a: TMA-fed, tcgen05.mma with the accumulator in
// tensor memory (TMEM), BF16 or TF32 operands, FP32 accumulation.
//
//   D[b] (M x N) = epilogue( A[b] (M x K) . B[b] (N x K)^T )
//
// Both operands are K-major (row-major with K contiguous), so that each
// operand tile is a plain TMA box with the 128-byte swizzle that the UMMA
// shared-memory descriptors expect.  The conversion kernels that produce the
// BF16 / TF32 operands write them in this layout.
//
// CTA: 192 threads = 6 warps.  Warp 0 (one elected lane) issues TMA loads
// into a STAGES-deep ring of shared-memory stages; warp 1 allocates TMEM and
// (one elected lane) issues tcgen05.mma, committing each stage back to the
// producer through an mbarrier; warps 2..5 read the 128 x BN FP32 accumulator
// out of TMEM (warp w reads lanes 32 (w % 4) .. 32 (w % 4) + 31) and run the
// epilogue.  The kernel is persistent (one CTA per SM, tiles strided by the
// grid) and TMEM holds two accumulators, so that the epilogue of one tile
// runs while the tensor core computes the next.
//
// Every wait on an mbarrier is bounded by the global timer: a wait that runs
// out sets an error flag (the caller's `err` word) and the thread stops
// waiting; before the CTA releases its TMEM and returns, the producer waits
// (bounded again) for the copies it issued that were not consumed.  The flag
// is best-effort: after FROB_ERR_TIMEOUT the results are unusable and the
// context should be treated as suspect.
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "common.cuh"

namespace frob {
namespace tc {

constexpr int BM = 128;
constexpr int BK_BYTES = 128;  // one 128-byte swizzle row of K per stage
constexpr int NUM_THREADS = 192;
constexpr uint64_t WAIT_NS = 2000000000ull;  // 2 s

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase with the given parity; false after WAIT_NS.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (!mbar_try_wait(bar, parity))
    if (global_ns() - t0 > WAIT_NS) return false;
  return true;
}

// 3-D tiled TMA load (x = K offset in elements, y = row, z = matrix index)
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], "
      "[%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
      : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

template <int KIND>  // 0: kind::f16 (BF16 operands), 1: kind::tf32
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
  if constexpr (KIND == 0) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
  }
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// 32 lanes x 32 bits, 16 consecutive columns per thread
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
      "[%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// UMMA shared-memory descriptor of a K-major tile stored with the 128-byte
// swizzle (rows of 128 bytes, 8-row groups 1024 bytes apart).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);      // start address
  d |= (uint64_t)1 << 16;                        // leading-dimension offset (unused for this layout)
  d |= (uint64_t)(1024 >> 4) << 32;              // stride-dimension offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;                        // fixed 0b001
  d |= (uint64_t)2 << 61;                        // 128-byte swizzle
  return d;
}

// Instruction descriptor: dense, FP32 accumulator, both operands K-major.
template <int KIND, int BN> __host__ __device__ constexpr uint32_t instr_desc() {
  return (1u << 4)                                   // D format F32
         | ((KIND == 0 ? 1u : 2u) << 7)              // A format: BF16 (kind::f16) / TF32
         | ((KIND == 0 ? 1u : 2u) << 10)             // B format
         | ((uint32_t)(BN >> 3) << 17)               // N >> 3
         | ((uint32_t)(BM >> 4) << 24);              // M >> 4
}

template <int BN, int STAGES> struct TcSmem {
  static constexpr int A_BYTES = BM * BK_BYTES;
  static constexpr int B_BYTES = BN * BK_BYTES;
  static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
  static constexpr int BYTES = STAGES * STAGE_BYTES + 1024 /*align slack*/ + 256 /*barriers*/;
};

// Epilogue functor interface: operator()(b, row, col0, v[16], nvalid) for 16
// consecutive columns col0 .. col0 + 15 of one output row (nvalid of them in
// range).
struct TcEpiStoreF32 {
  float* D;
  int64_t ldd, sd;
  float alpha, beta;  // D = alpha * acc + beta * D
  __device__ __forceinline__ void operator()(int b, int row, int col0, const float (&v)[16], int nvalid) const {
    float* p = D + (int64_t)b * sd + (int64_t)row * ldd + col0;
#pragma unroll
    for (int i = 0; i < 16; ++i)
      if (i < nvalid) p[i] = (beta == 0.f) ? alpha * v[i] : alpha * v[i] + beta * p[i];
  }
};

// Adapter for the element-wise epilogues of the CUDA-core GEMM
// (operator()(b, i, j, v)): the tensor-core kernel hands it 16 columns of one
// row at a time.
template <class Epi> struct TcEpiElem {
  Epi e;
  __device__ __forceinline__ void operator()(int b, int row, int col0, const float (&v)[16], int nvalid) const {
#pragma unroll
    for (int i = 0; i < 16; ++i)
      if (i < nvalid) e(b, row, col0 + i, v[i]);
  }
};

// Persistent: CTA c takes output tiles c, c + gridDim.x, ... (x fastest, then
// y, then the batch).  TMEM holds two BN-column accumulators; the MMA issuer
// fills one while the epilogue warps drain the other, so a tile's epilogue
// overlaps the next tile's main loop.
template <int KIND, int BN, int STAGES, class Epi>
__global__ void __launch_bounds__(NUM_THREADS, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, int M, int N,
                   int K, int batch, Epi epi, int* err) {
  using S = TcSmem<BN, STAGES>;
  constexpr int ELEM = (KIND == 0) ? 2 : 4;
  constexpr int BK = BK_BYTES / ELEM;          // K elements per stage (64 BF16 / 32 TF32)
  constexpr int MMA_K = 32 / ELEM;             // K per instruction (16 BF16 / 8 TF32)
  constexpr uint32_t IDESC = instr_desc<KIND, BN>();
  constexpr uint32_t ACC_COLS = BN < 32 ? 32 : BN;
  constexpr uint32_t TMEM_COLS = 2 * ACC_COLS;

  extern __shared__ __align__(1024) unsigned char smraw[];
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(base + STAGES * S::STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* acc_full = empty + STAGES;  // [2]
  uint64_t* acc_empty = acc_full + 2;   // [2]
  uint64_t* mma_done = acc_empty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mma_done + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int kblocks = (K + BK - 1) / BK;
  const int nx = (N + BN - 1) / BN, ny = (M + BM - 1) / BM;
  const int ntiles = nx * ny * batch;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&acc_full[i], 1);
      mbar_init(&acc_empty[i], 4);  // the four epilogue warps
    }
    mbar_init(mma_done, 1);
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  int filled = 0;  // producer: stages filled

  if (warp == 0) {
    if (lane == 0) {
      // producer
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        const int xt = t % nx, yt = (t / nx) % ny, b = t / (nx * ny);
        for (int kb = 0; kb < kblocks; ++kb) {
          const int s = filled % STAGES;
          if (filled >= STAGES && !mbar_wait(&empty[s], ((filled / STAGES) - 1) & 1)) {
            atomicExch(err, FROB_ERR_TIMEOUT);
            ok = false;
            break;
          }
          unsigned char* sa = base + s * S::STAGE_BYTES;
          mbar_arrive_expect_tx(&full[s], S::STAGE_BYTES);
          tma_load_3d(sa, &mapA, &full[s], kb * BK, yt * BM, b);
          tma_load_3d(sa + S::A_BYTES, &mapB, &full[s], kb * BK, xt * BN, b);
          ++filled;
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issuer
      bool ok = true;
      int used = 0;  // stages consumed
      int it = 0;    // tiles of this CTA
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++it) {
        const int buf = it & 1;
        if (it >= 2 && !mbar_wait(&acc_empty[buf], ((it >> 1) - 1) & 1)) {
          atomicExch(err, FROB_ERR_TIMEOUT);
          break;
        }
        tc_fence_after();
        const uint32_t acc = tmem + (uint32_t)(buf * ACC_COLS);
        for (int kb = 0; kb < kblocks; ++kb) {
          const int s = used % STAGES;
          if (!mbar_wait(&full[s], (used / STAGES) & 1)) {
            atomicExch(err, FROB_ERR_TIMEOUT);
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = smem_u32(base + s * S::STAGE_BYTES);
          const uint32_t sb = sa + S::A_BYTES;
#pragma unroll
          for (int k = 0; k < BK / MMA_K; ++k) {
            const uint64_t ad = sw128_desc(sa + k * 32);
            const uint64_t bd = sw128_desc(sb + k * 32);
            mma<KIND>(acc, ad, bd, IDESC, (kb > 0 || k > 0) ? 1u : 0u);
          }
          mma_commit(&empty[s]);
          ++used;
        }
        if (ok) mma_commit(&acc_full[buf]);
      }
      // every MMA this thread issued has finished before TMEM is released
      mma_commit(mma_done);
      if (!mbar_wait(mma_done, 0)) atomicExch(err, FROB_ERR_TIMEOUT);
    }
  } else {
    // epilogue warps 2..5: TMEM lanes 32 (warp % 4) ...
    const int sub = warp & 3;
    int it = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
      const int xt = t % nx, yt = (t / nx) % ny, b = t / (nx * ny);
      const int buf = it & 1;
      if (!mbar_wait(&acc_full[buf], (it >> 1) & 1)) {
        if (lane == 0) atomicExch(err, FROB_ERR_TIMEOUT);
        break;
      }
      tc_fence_after();
      const int row = yt * BM + sub * 32 + lane;
#pragma unroll 1
      for (int c = 0; c < BN; c += 16) {
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(sub * 32) << 16) + (uint32_t)(buf * ACC_COLS + c), v);
        const int col0 = xt * BN + c;
        int nvalid = N - col0;
        nvalid = nvalid > 16 ? 16 : nvalid;
        if (row < M && nvalid > 0) epi(b, row, col0, v, nvalid);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acc_empty[buf])) : "memory");
    }
  }
  tc_fence_before();
  __syncthreads();
  // the producer waits for any stage it filled that the MMA did not consume,
  // so that no TMA write lands in shared memory after the CTA exits
  if (warp == 0 && lane == 0) {
    for (int j = (filled > STAGES ? filled - STAGES : 0); j < filled; ++j)
      mbar_wait(&full[j % STAGES], (j / STAGES) & 1);
  }
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, TMEM_COLS);
  }
}

// ---------------------------------------------------------------- split TF32
// FP32 products on the TF32 tensor cores with FP32-level accuracy: every
// operand value x is split into hi = tf32(x) and lo = tf32(x - hi) (both
// rounded to nearest; x - hi has at most 13 significant bits, so
// |x - hi - lo| <= 2^-23 |x|), and a b ~ hi_a hi_b + hi_a lo_b + lo_a hi_b
// (the dropped lo_a lo_b is below 2^-22 |a b|).  The three products are one
// tensor-core GEMM over a K three times as long: the A operand row holds
// [hi | hi | lo] and the B operand row [hi | lo | hi], each block of Kp
// (K padded to a 16-byte multiple with zeros) values, so that the FP32
// accumulator in TMEM sums all three.
constexpr int TC3_MIN_MN = 128;  // smaller products stay on the CUDA cores
constexpr int TC3_MIN_K = 256;   // as do short ones (an epilogue-bound rank-K update)

int64_t tc3_kp(int K);
// scratch for one product: both split operands (plus the timeout flag's 256 B)
size_t tc3_scratch_bytes(int M, int N, int K, int batch);
// Splits op(A) (M x K; A[i][k], or A[k][i] when transA) and op(B)^T (N x K;
// B[k][j] when transB, else B[j][k]) into the scratch after its first 256
// bytes and encodes the two tensor maps; false if the maps cannot be made.
bool tc3_prepare(int M, int N, int K, int batch, const float* A, int64_t lda, int64_t sa, bool transA,
                 const float* B, int64_t ldb, int64_t sb, bool transB, void* scratch, CUtensorMap* ma,
                 CUtensorMap* mb, cudaStream_t st);

// One persistent launch of tc_gemm_kernel over the split operands with an
// element-wise epilogue; `err` receives FROB_ERR_TIMEOUT if a bounded wait
// gave up.
template <class Epi>
inline cudaError_t tc3_launch(const CUtensorMap& ma, const CUtensorMap& mb, int M, int N, int K, int batch, Epi epi,
                              int* err, cudaStream_t st) {
  constexpr int BN = 256, STAGES = 4;
  using S = TcSmem<BN, STAGES>;
  using E = TcEpiElem<Epi>;
  set_smem_attr(tc_gemm_kernel<1, BN, STAGES, E>, S::BYTES);
  const int64_t tiles = (int64_t)((N + BN - 1) / BN) * ((M + BM - 1) / BM) * batch;
  if (tiles > INT32_MAX) return cudaErrorInvalidValue;
  const unsigned grid = persistent_grid(tiles);
  const int K3 = (int)(3 * tc3_kp(K));
  FROB_LAUNCH("tc_gemm<3xtf32>", st,
              tc_gemm_kernel<1, BN, STAGES, E><<<grid, NUM_THREADS, S::BYTES, st>>>(ma, mb, M, N, K3, batch, E{epi},
                                                                                  err));
  return cudaGetLastError();
}

}  // namespace tc
}  // namespace frob
