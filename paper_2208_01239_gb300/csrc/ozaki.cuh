// FP64-accurate complex matrix products on the BF16 tensor cores, by exact
// splitting of the operands (Ozaki, Ogita, Oishi and Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication", Numer. Algorithms 2012, scheme I).
//
// Splitting (oz_split_rows_kernel).  Each row i of a real FP64 matrix is
// scaled by 2^-e_i, where 2^e_i is the smallest power of two above the row's
// largest magnitude, so the scaled entries r lie in (-1, 1).  Then S signed
// digits are taken by repeated round-to-nearest:
//     d_1 = rint(128 r),  r <- 128 r - d_1,  d_2 = rint(128 r), ...
// |d_1| <= 128 and |d_s| <= 64 for s >= 2, so every digit is exact in BF16,
// and  r = sum_s d_s 2^{-7 s} + (remainder below 2^{-7 S - 1}).
//
// Products.  For digit matrices D_s (of A, row-scaled) and E_t (of B,
// column-scaled), every entry of D_s E_t^T is an integer below 2^23 in
// magnitude when K <= 512, so the tensor core's FP32 accumulation is exact.
// All pairs with the same weight 2^{-7 (s + t)} are accumulated into one TMEM
// accumulator; for s + t <= 7 the sum stays at most 2^24 and is exact.  The
// weights 2^-56 and 2^-63 (s + t = 8, 9) lie below the FP64 unit of the
// result, so one FP32 rounding of their group sums (relative 2^-24) is
// harmless there.  Pairs with s + t > S + 1 are dropped (their weight is
// below 2^{-7 (S + 2)}).
//
// Complex product C = A B with A = Ar + i Ai, B = Br + i Bi:
//   Re C = Ar Br - Ai Bi,  Im C = Ar Bi + Ai Br;
// each output part is two real terms.  The kernel computes one 128 x 64 tile
// of one part: for each term, for each digit s of the A operand, for each
// 256-wide K chunk, the 128 x 256 chunk of the digit slice stays resident in
// shared memory (two chunk buffers, so that the next chunk loads while the
// current one is used) while the matching K chunks of the digit slices of B
// stream through a 6-stage TMA ring of 128-wide K stages (8 MMAs per barrier
// round: the per-round barrier and commit cost is fixed, so wider stages keep
// the tensor pipe busier); tcgen05.mma accumulates into the group
// accumulators in TMEM; after each term the epilogue warps add the groups,
// scaled by their powers of two, into a register accumulator per output
// element (see the epilogues below).  The final value goes to FP64.
//
// Epilogues:
//   RESID:  writes R^T with R = I - A B (transposed store, coalesced) and
//           adds sum |R_ij|^2 into a per-matrix FP64 accumulator.  The
//           operands are split with joint real / imaginary exponents and the
//           groups are summed exactly in 64-bit fixed point, so that the
//           residual carries FP64 rounding only (float-float would leave an
//           error near 2^-48 of sum_k |a_ik b_kj|, which is the floor the
//           refinement would stall at).
//   CORR:   X <- X + A B, written to X (row-major) and X^T.
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "common.cuh"
#include "tc_gemm.cuh"

namespace frob {
namespace oz {

constexpr int S_MAX = 8;
constexpr int BN = 64;        // output tile columns
constexpr int KB = 64;        // BF16 elements per k-block (one 128-byte row)
constexpr int KP_ALIGN = 128; // the padded K (digit-array pitch) is a multiple of this
constexpr int K_MAX = 512;    // largest inner dimension with exact FP32 accumulation
constexpr int A_CHUNK_KB = 4;                              // k-blocks per resident A chunk
constexpr int A_CHUNK_BYTES = tc::BM * KB * 2 * A_CHUNK_KB;  // 64 KB: 128 rows x 256 K
constexpr int A_RES_BYTES = 2 * A_CHUNK_BYTES;               // double-buffered
constexpr int KSTAGE = 2;                                   // 64-wide K boxes per B stage
constexpr int B_BOX_BYTES = BN * KB * 2;                    // 8 KB
constexpr int B_STAGE_BYTES = B_BOX_BYTES * KSTAGE;         // 16 KB: 8 MMAs per barrier round
constexpr int B_STAGES = 6;
constexpr int NUM_GROUPS = 8;
constexpr int THREADS = 192;
constexpr int SMEM_BYTES = A_RES_BYTES + B_STAGES * B_STAGE_BYTES + 1024 + 512 + 4 * BN * 4;

// weight group of the digit pair (s, t), 1-based digits, s + t <= 9: one
// group per weight 2^(-7 (s + t))
__host__ __device__ constexpr int group_of(int s, int t) { return s + t - 2; }
__host__ __device__ constexpr int weight_of_group(int g) { return g + 2; }

// ---------------------------------------------------------------- split
// src: two real FP64 matrices per batch entry (rows x K, row-major, ld, batch
// stride bs, part stride ps); dst digits: BF16 [part][s][b][row][Kp]
// (zero-padded to Kp, Kp a multiple of 128, K <= K_MAX); exps: int
// [part][b][row].  With JOINT the real and imaginary rows share one exponent
// (the larger), so that the two real products of one complex output part
// carry the same row and column scales.
//
// Integer arithmetic only (the FP64 pipe is slow on this GPU): with
// x = +-m 2^(ex - 1075) (m the 53-bit significand, ex the biased exponent),
// the scaled value x 2^(7S - e) is rounded once to an integer F by a shift with
// round-to-nearest, |F| <= 2^(7S), and F is written in balanced base 128:
// with G = F + 64 (1 + 128 + ... + 128^(S-2)), the S - 1 trailing digits are
// ((G >> 7j) mod 128) - 64 in [-64, 63] and the leading digit is
// G >> 7(S-1) (arithmetic shift), |d_1| <= 128.  Then
// x 2^-e = sum_s d_s 2^(-7 s) up to 2^(-7 S - 1).
__device__ __forceinline__ long long scaled_fixed(double x, int shift_exp) {
  // returns rint(x * 2^shift_exp) for |x * 2^shift_exp| < 2^62, without FP64 math
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((u >> 52) & 0x7FF);
  if (ex == 0) return 0;                      // zero or subnormal (below every digit)
  const unsigned long long m = (u & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int sh = ex - 1075 + shift_exp;       // x * 2^shift = m * 2^sh
  long long v;
  if (sh >= 0) {
    v = (long long)(m << sh);                 // sh < 10 here because |result| < 2^62
  } else if (sh > -64) {
    const unsigned long long half = 1ull << (-sh - 1);
    const unsigned long long q = m >> (-sh);
    const unsigned long long rem = m & ((1ull << (-sh)) - 1ull);
    unsigned long long r = q;
    if (rem > half || (rem == half && (q & 1ull))) r = q + 1;  // nearest, ties to even
    v = (long long)r;
  } else {
    v = 0;
  }
  return (u >> 63) ? -v : v;
}

// BF16 bit pattern of a small integer d (|d| <= 256): 2^23 + 256 + d is an
// exact FP32 number, subtracting 2^23 + 256 leaves d exactly, and the low 16
// bits of an FP32 integer below 2^9 are zero.
__device__ __forceinline__ uint32_t bf16_bits_of_int(int d) {
  const float f = __int_as_float(0x4B000000 | (d + 256)) - 8388864.0f;
  return (uint32_t)__float_as_uint(f) >> 16;
}

// One warp per row (JOINT: per row pair, real and imaginary).  Each lane keeps
// its 16 entries of the row (4 consecutive columns in each 128-wide block) in
// registers between the maximum and the digit passes.
template <bool JOINT>
__global__ void __launch_bounds__(256) oz_split_rows_kernel(int rows, int K, int Kp, int batch, int S,
                                                            const double* src, int64_t ld, int64_t bs, int64_t ps,
                                                            __nv_bfloat16* dst, int* exps, const int* skip) {
  constexpr int NP = JOINT ? 2 : 1;
  constexpr int NJ = K_MAX / 128;
  const int warp = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  const int row = warp % rows;
  const int b = (warp / rows) % batch;
  const int w2 = warp / (rows * batch);
  if (w2 >= (JOINT ? 1 : 2)) return;
  if (skip && skip[b]) return;
  const int part0 = JOINT ? 0 : w2;
  double v[NP][NJ][4];
  unsigned long long mx = 0;  // largest |x| of the row(s), compared on the bit patterns (sign cleared)
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    const double* r = src + (int64_t)(part0 + p) * ps + (int64_t)b * bs + (int64_t)row * ld;
#pragma unroll
    for (int j = 0; j < NJ; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int k = 128 * j + 4 * lane + q;
        v[p][j][q] = k < K ? r[k] : 0.0;
        const unsigned long long a = (unsigned long long)__double_as_longlong(v[p][j][q]) & 0x7FFFFFFFFFFFFFFFull;
        mx = a > mx ? a : mx;
      }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long other = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = other > mx ? other : mx;
  }
  // e: smallest integer with max |x| < 2^e (0 for an all-zero row)
  int e = 0;
  const int mex = (int)(mx >> 52);
  if (mx != 0 && mex < 0x7FF) e = (mex == 0) ? -1022 : mex - 1022;
  if (lane == 0)
#pragma unroll
    for (int p = 0; p < NP; ++p) exps[((int64_t)(part0 + p) * batch + b) * rows + row] = e;
  long long off = 0;  // 64 (1 + 128 + ... + 128^(S-2))
  for (int j = 0; j < S - 1; ++j) off = (off << 7) + 64;
  const int64_t plane = (int64_t)batch * rows * Kp;  // one digit slice
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    __nv_bfloat16* out = dst + (int64_t)(part0 + p) * S * plane + ((int64_t)b * rows + row) * Kp;
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      const int k0 = 128 * j + 4 * lane;
      if (128 * j >= Kp) break;
      long long G[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) G[q] = scaled_fixed(v[p][j][q], 7 * S - e) + off;
      for (int sl = 0; sl < S; ++sl) {  // slice sl holds the digit of weight 2^(-7 (sl + 1))
        const int sh = 7 * (S - 1 - sl);
        uint32_t bits[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int d = sl == 0 ? (int)(G[q] >> sh) : (int)((G[q] >> sh) & 127) - 64;
          bits[q] = bf16_bits_of_int(d);
        }
        const uint2 w = make_uint2(bits[0] | (bits[1] << 16), bits[2] | (bits[3] << 16));
        *reinterpret_cast<uint2*>(out + (int64_t)sl * plane + k0) = w;
      }
    }
  }
}

// ---------------------------------------------------------------- product
enum Mode : int { RESID = 0, CORR = 1 };

struct OzArgs {
  int n;          // square matrices: rows = cols = K = n
  int Kp;         // K padded to KP_ALIGN
  int batch;
  int S;          // digits per operand in the digit arrays (their layout)
  int Su;         // leading digits used (<= S): pairs s, t <= Su with s + t <= Su + 1
  const int* expA;  // [2][batch][n]
  const int* expB;  // [2][batch][n]
  // RESID: RT planes (re, im): R^T, plus per-matrix sum of squares
  double* outR;     // [2][batch][n][n]
  double* rnorm2;   // [batch]
  // CORR: X planes (re, im) updated in place, and X^T planes written
  double* X;        // [2][batch][n][n]
  double* XT;       // [2][batch][n][n]
  const int* skip;  // per-matrix: nonzero = skip (converged or failed); may be NULL
  int* err;
};

// 2^k as an FP32 number, exact for -126 <= k <= 127 (built from the IEEE
// exponent field); 0 below, +inf above.
__device__ __forceinline__ float pow2f(int k) {
  if (k < -126) return 0.f;
  if (k > 127) return __int_as_float(0x7F800000);
  return __int_as_float((k + 127) << 23);
}

__device__ __forceinline__ void two_sum(float& hi, float& lo, float x) {
  const float s = hi + x;
  const float bb = s - hi;
  const float e = (hi - (s - bb)) + (x - bb);
  hi = s;
  lo += e;
}

template <int MODE>
__global__ void __launch_bounds__(THREADS, 1)
    oz_cgemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, OzArgs args) {
  using namespace tc;
  extern __shared__ __align__(1024) unsigned char smraw[];
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
  unsigned char* a_res = base;
  unsigned char* b_ring = base + A_RES_BYTES;
  uint64_t* bars = reinterpret_cast<uint64_t*>(b_ring + B_STAGES * B_STAGE_BYTES);
  uint64_t* b_full = bars;
  uint64_t* b_empty = bars + B_STAGES;
  uint64_t* a_full = bars + 2 * B_STAGES;  // [2]
  uint64_t* a_empty = a_full + 2;          // [2]
  uint64_t* term_done = a_empty + 2;
  uint64_t* drained = term_done + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drained + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n = args.n, S = args.S, batch = args.batch;
  const int Su = args.Su;
  const int b = blockIdx.z >> 1;
  const int part = blockIdx.z & 1;  // 0: real part of the product, 1: imaginary part
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int nkb = args.Kp / KB;
  // a converged or failed matrix: the whole CTA leaves before it allocates TMEM
  if (args.skip && args.skip[b]) return;
  // terms: (A operand part, B operand part, sign)
  const int ta0 = 0, tb0 = part;              // Ar Br (re) / Ar Bi (im)
  const int ta1 = 1, tb1 = part ^ 1;          // Ai Bi (re) / Ai Br (im)
  const float sg1 = part == 0 ? -1.f : 1.f;   // - Ai Bi (re), + Ai Br (im)

  if (threadIdx.x == 0) {
    for (int s = 0; s < B_STAGES; ++s) {
      mbar_init(&b_full[s], 1);
      mbar_init(&b_empty[s], 1);
    }
    mbar_init(&a_full[0], 1);
    mbar_init(&a_full[1], 1);
    mbar_init(&a_empty[0], 1);
    mbar_init(&a_empty[1], 1);
    mbar_init(term_done, 1);
    mbar_init(drained, 4);
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  {
    if (warp == 0 && lane == 0) {
      // ---------------- producer
      const int nch = (nkb + A_CHUNK_KB - 1) / A_CHUNK_KB;
      int bi = 0;   // B stage fill counter
      int ai = 0;   // A chunk fill counter
      bool ok = true;
      for (int term = 0; term < 2 && ok; ++term) {
        const int ap = term ? ta1 : ta0, bp = term ? tb1 : tb0;
        for (int s = 1; s <= Su && ok; ++s) {
          const int za = (ap * S + (s - 1)) * batch + b;
          for (int ch = 0; ch < nch && ok; ++ch) {
            const int kb0 = ch * A_CHUNK_KB;
            const int kb1 = (kb0 + A_CHUNK_KB < nkb) ? kb0 + A_CHUNK_KB : nkb;
            const int slot = ai & 1;
            if (ai >= 2 && !mbar_wait(&a_empty[slot], ((ai >> 1) - 1) & 1)) { ok = false; break; }
            mbar_arrive_expect_tx(&a_full[slot], (uint32_t)((kb1 - kb0) * BM * KB * 2));
            unsigned char* abuf = a_res + slot * A_CHUNK_BYTES;
            for (int kb = kb0; kb < kb1; ++kb)
              tma_load_3d(abuf + (kb - kb0) * (BM * KB * 2), &mapA, &a_full[slot], kb * KB, m0, za);
            ++ai;
            for (int t = 1; t <= Su + 1 - s && ok; ++t) {
              const int zb = (bp * S + (t - 1)) * batch + b;
              for (int kb = kb0; kb < kb1; kb += KSTAGE) {
                const int st = bi % B_STAGES;
                if (bi >= B_STAGES && !mbar_wait(&b_empty[st], ((bi / B_STAGES) - 1) & 1)) { ok = false; break; }
                mbar_arrive_expect_tx(&b_full[st], B_STAGE_BYTES);
#pragma unroll
                for (int q = 0; q < KSTAGE; ++q)
                  tma_load_3d(b_ring + st * B_STAGE_BYTES + q * B_BOX_BYTES, &mapB, &b_full[st], (kb + q) * KB, n0, zb);
                ++bi;
              }
            }
          }
        }
      }
      if (!ok) atomicExch(args.err, FROB_ERR_TIMEOUT);
    } else if (warp == 1 && lane == 0) {
      // ---------------- MMA issuer
      constexpr uint32_t IDESC = instr_desc<0, BN>();
      const int nch = (nkb + A_CHUNK_KB - 1) / A_CHUNK_KB;
      int bi = 0, ai = 0;
      bool ok = true;
      for (int term = 0; term < 2 && ok; ++term) {
        if (term == 1 && !mbar_wait(drained, 0)) { ok = false; break; }  // groups drained after term 0
        tc_fence_after();
        uint32_t started = 0;
        for (int s = 1; s <= Su && ok; ++s) {
          for (int ch = 0; ch < nch && ok; ++ch) {
            const int kb0 = ch * A_CHUNK_KB;
            const int kb1 = (kb0 + A_CHUNK_KB < nkb) ? kb0 + A_CHUNK_KB : nkb;
            const int slot = ai & 1;
            if (!mbar_wait(&a_full[slot], (ai >> 1) & 1)) { ok = false; break; }
            ++ai;
            tc_fence_after();
            const uint32_t sa = smem_u32(a_res + slot * A_CHUNK_BYTES);
            for (int t = 1; t <= Su + 1 - s && ok; ++t) {
              const int g = group_of(s, t);
              const uint32_t dt = tmem + (uint32_t)(g * BN);
              for (int kb = kb0; kb < kb1; kb += KSTAGE) {
                const int st = bi % B_STAGES;
                if (!mbar_wait(&b_full[st], (bi / B_STAGES) & 1)) { ok = false; break; }
                tc_fence_after();
                const uint32_t sb = smem_u32(b_ring + st * B_STAGE_BYTES);
#pragma unroll
                for (int q = 0; q < KSTAGE; ++q)
#pragma unroll
                  for (int kk = 0; kk < KB / 16; ++kk) {
                    const uint64_t ad = sw128_desc(sa + (kb + q - kb0) * (BM * KB * 2) + kk * 32);
                    const uint64_t bd = sw128_desc(sb + q * B_BOX_BYTES + kk * 32);
                    const uint32_t acc = ((started >> g) & 1u) ? 1u : 0u;
                    mma<0>(dt, ad, bd, IDESC, acc);
                    started |= 1u << g;
                  }
                mma_commit(&b_empty[st]);
                ++bi;
              }
            }
            mma_commit(&a_empty[slot]);  // chunk buffer free once these MMAs complete
          }
        }
        mma_commit(term_done);  // phase `term` of term_done
      }
      if (!ok) atomicExch(args.err, FROB_ERR_TIMEOUT);
    } else if (warp >= 2) {
      // ---------------- epilogue: warps 2..5 -> TMEM lanes 32 (warp % 4) ..
      const int sub = warp & 3;
      const int row = m0 + sub * 32 + lane;
      const int ngroups = Su;  // weights 2 .. Su + 1
      int* colexp = reinterpret_cast<int*>(tmem_slot + 4) + sub * BN;  // this warp's column exponents
      const int64_t nn = (int64_t)n * n;
      bool ok = true;
      if constexpr (MODE == RESID) {
        // Exact accumulation: both terms share the row and column exponents
        // (joint splits), every group value is an integer in FP32, and the
        // sum over groups and terms is kept in 64-bit fixed point, in units of
        // 2^-52 of the scaled product (|scaled product| < 2^11).  Groups of
        // weight 2^-56 and 2^-63 are rounded to that unit (at most 2^-53).
        long long acc[BN];
#pragma unroll
        for (int c = 0; c < BN; ++c) acc[c] = 0;
        for (int term = 0; term < 2; ++term) {
          if (!mbar_wait(term_done, term)) { ok = false; break; }
          tc_fence_after();
          const float sgn = term ? sg1 : 1.f;
          for (int g = 0; g < ngroups; ++g) {
            const int sh = 52 - 7 * weight_of_group(g);
            const float pre = sh < 0 ? sgn * pow2f(sh) : sgn;
            const int lsh = sh < 0 ? 0 : sh;
#pragma unroll
            for (int c0 = 0; c0 < BN; c0 += 16) {
              float v[16];
              tmem_ld16(tmem + ((uint32_t)(sub * 32) << 16) + (uint32_t)(g * BN + c0), v);
#pragma unroll
              for (int i = 0; i < 16; ++i)
                acc[c0 + i] += (long long)((unsigned long long)(long long)__float2int_rn(v[i] * pre) << lsh);
            }
          }
          __syncwarp();
          tc_fence_before();
          __syncwarp();
          if (term == 0 && lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(drained)) : "memory");
        }
        if (!ok && lane == 0) atomicExch(args.err, FROB_ERR_TIMEOUT);
        for (int c = lane; c < BN; c += 32) {
          const int col = n0 + c;
          colexp[c] = col < n ? args.expB[((int64_t)tb0 * batch + b) * n + col] : 0;
        }
        __syncwarp();
        const int ea = row < n ? args.expA[((int64_t)ta0 * batch + b) * n + row] : 0;
        double ss = 0.0;  // every lane takes part in the reduction below
        if (ok && row < n) {
          double* RT = args.outR + ((int64_t)part * batch + b) * nn;
#pragma unroll
          for (int c = 0; c < BN; ++c) {
            const int col = n0 + c;
            if (col < n) {
              const double pr = ldexp((double)acc[c], ea + colexp[c] - 52);
              const double r = (part == 0 && col == row ? 1.0 : 0.0) - pr;
              RT[(int64_t)col * n + row] = r;
              ss += r * r;
            }
          }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
        if (lane == 0 && ss != 0.0) atomicAdd(args.rnorm2 + b, ss);
      } else {
        // float-float (hi + lo) accumulation with error-free two-sums; the
        // terms carry their own row and column scales
        float hi[BN], lo[BN];
#pragma unroll
        for (int c = 0; c < BN; ++c) {
          hi[c] = 0.f;
          lo[c] = 0.f;
        }
        float* colscale = reinterpret_cast<float*>(colexp);
        for (int term = 0; term < 2; ++term) {
          if (!mbar_wait(term_done, term)) { ok = false; break; }
          tc_fence_after();
          const int ap = term ? ta1 : ta0, bp = term ? tb1 : tb0;
          const float sgn = term ? sg1 : 1.f;
          // column scales 2^(e_B[col]) of this term, staged in shared memory
          for (int c = lane; c < BN; c += 32) {
            const int col = n0 + c;
            const int eb = col < n ? args.expB[((int64_t)bp * batch + b) * n + col] : 0;
            colscale[c] = pow2f(eb);
          }
          __syncwarp();
          const int ea = row < n ? args.expA[((int64_t)ap * batch + b) * n + row] : 0;
          for (int g = 0; g < ngroups; ++g) {
            const int w = weight_of_group(g);
            // sign x 2^(e_A - 7 w): exact power of two (within FP32 range for the data seen here)
            const float rs = sgn * pow2f(ea - 7 * w);
#pragma unroll
            for (int c0 = 0; c0 < BN; c0 += 16) {
              float v[16];
              tmem_ld16(tmem + ((uint32_t)(sub * 32) << 16) + (uint32_t)(g * BN + c0), v);
#pragma unroll
              for (int i = 0; i < 16; ++i) two_sum(hi[c0 + i], lo[c0 + i], (v[i] * rs) * colscale[c0 + i]);
            }
          }
          __syncwarp();
          tc_fence_before();
          __syncwarp();
          if (term == 0 && lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(drained)) : "memory");
        }
        if (!ok && lane == 0) atomicExch(args.err, FROB_ERR_TIMEOUT);
        if (ok && row < n) {
          double* Xp = args.X + ((int64_t)part * batch + b) * nn;
          double* XTp = args.XT + ((int64_t)part * batch + b) * nn;
#pragma unroll
          for (int c = 0; c < BN; ++c) {
            const int col = n0 + c;
            if (col < n) {
              const double v = Xp[(int64_t)row * n + col] + ((double)hi[c] + (double)lo[c]);
              Xp[(int64_t)row * n + col] = v;
              XTp[(int64_t)col * n + row] = v;
            }
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

}  // namespace oz
}  // namespace frob
