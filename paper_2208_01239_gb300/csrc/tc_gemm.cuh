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
// epilogue.  One output tile of 128 x BN per CTA.
//
// Every wait on an mbarrier is bounded by the global timer: a wait that runs
// out sets an error flag (the caller's `err` word) and the thread stops
// waiting; the CTA still releases its TMEM and returns.
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

template <int KIND, int BN, int STAGES, class Epi>
__global__ void __launch_bounds__(NUM_THREADS, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, int M, int N,
                   int K, Epi epi, int* err) {
  using S = TcSmem<BN, STAGES>;
  constexpr int ELEM = (KIND == 0) ? 2 : 4;
  constexpr int BK = BK_BYTES / ELEM;          // K elements per stage (64 BF16 / 32 TF32)
  constexpr int MMA_K = 32 / ELEM;             // K per instruction (16 BF16 / 8 TF32)
  constexpr uint32_t IDESC = instr_desc<KIND, BN>();
  constexpr uint32_t TMEM_COLS = BN < 32 ? 32 : BN;

  extern __shared__ __align__(1024) unsigned char smraw[];
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(base + STAGES * S::STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* done = empty + STAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int b = blockIdx.z;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int kblocks = (K + BK - 1) / BK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
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

  if (warp == 0) {
    if (lane == 0) {
      // producer
      for (int kb = 0; kb < kblocks; ++kb) {
        const int s = kb % STAGES;
        const uint32_t round = kb / STAGES;
        if (kb >= STAGES && !mbar_wait(&empty[s], (round - 1) & 1)) {
          atomicExch(err, FROB_ERR_TIMEOUT);
          break;
        }
        unsigned char* sa = base + s * S::STAGE_BYTES;
        mbar_arrive_expect_tx(&full[s], S::STAGE_BYTES);
        tma_load_3d(sa, &mapA, &full[s], kb * BK, m0, b);
        tma_load_3d(sa + S::A_BYTES, &mapB, &full[s], kb * BK, n0, b);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issuer
      bool ok = true;
      for (int kb = 0; kb < kblocks && ok; ++kb) {
        const int s = kb % STAGES;
        if (!mbar_wait(&full[s], (kb / STAGES) & 1)) {
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
          mma<KIND>(tmem, ad, bd, IDESC, (kb > 0 || k > 0) ? 1u : 0u);
        }
        mma_commit(&empty[s]);
      }
      mma_commit(done);
    }
  } else {
    // epilogue warps 2..5: TMEM lanes 32 (warp % 4) ...
    const int sub = warp & 3;
    const int row = m0 + sub * 32 + lane;
    const bool ok = mbar_wait(done, 0);
    if (!ok && lane == 0) atomicExch(err, FROB_ERR_TIMEOUT);
    tc_fence_after();
    if (ok) {
#pragma unroll 1
      for (int c = 0; c < BN; c += 16) {
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(sub * 32) << 16) + (uint32_t)c, v);
        const int col0 = n0 + c;
        int nvalid = N - col0;
        nvalid = nvalid > 16 ? 16 : nvalid;
        if (row < M && nvalid > 0) epi(b, row, col0, v, nvalid);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  // the producer waits for any stage it filled that the MMA did not consume,
  // so that no TMA write lands in shared memory after the CTA exits
  if (warp == 0 && lane == 0) {
    for (int s = 0; s < STAGES && s < kblocks; ++s) {
      const int last = ((kblocks - 1 - s) / STAGES) * STAGES + s;  // last k-block that used stage s
      mbar_wait(&full[s], (last / STAGES) & 1);
    }
  }
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, TMEM_COLS);
  }
}

}  // namespace tc
}  // namespace frob
