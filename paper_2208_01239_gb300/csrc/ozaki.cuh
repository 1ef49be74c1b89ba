// FP64-accurate complex matrix products on the BF16 tensor cores, by exact
// splitting of the operands (Ozaki, Ogita, Oishi and Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication", Numer. Algorithms 2012, scheme I).
//
// Splitting (oz_split_rows_kernel).  Each row i of a real FP64 matrix pair
// (the real and imaginary parts) is scaled by 2^-e_i, where 2^e_i is the
// smallest power of two above the largest magnitude in the two rows, so the
// scaled entries r lie in (-1, 1).  Then r is written with S signed digits
// in base 128, r = sum_s d_s 2^{-7 s} + (remainder below 2^{-7 S - 1}),
// |d_1| <= 128 and |d_s| <= 64 for s >= 2, so every digit is exact in BF16.
//
// Products.  For digit matrices D_s (of A, row-scaled) and E_t (of B,
// column-scaled), every entry of D_s E_t^T is an integer below 2^23 in
// magnitude when K <= 512, so the tensor core's FP32 accumulation is exact.
// All pairs with the same weight 2^{-7 (s + t)} are accumulated into one TMEM
// accumulator ("group"); for s + t <= 7 the sum stays at most 2^24 and is
// exact.  The weights 2^-56 and 2^-63 (s + t = 8, 9) lie below the FP64 unit
// of the result, so one FP32 rounding of their group sums (relative 2^-24) is
// harmless there.  Pairs with s + t > S + 1 are dropped (their weight is
// below 2^{-7 (S + 2)}).
//
// Complex product C = A B with A = Ar + i Ai, B = Br + i Bi:
//   Re C = Ar Br - Ai Bi,  Im C = Ar Bi + Ai Br;
// each output part is two real terms, and with the joint exponents both
// terms carry the same row and column scales.
//
// Kernel (oz_cgemm_kernel): 128 x 128 tiles of one part, persistent CTAs.  The
// tensor pipe spends about the same time on a 128 x 64 x 16 MMA as on a
// 128 x 128 x 16 one, so the tile is 128 wide; TMEM (512 columns) then holds
// four 128-column accumulator slots, fewer than the up to 8 groups of a term.
// The groups are therefore issued in bands of four weights, {2 .. 5} and
// {6 .. S + 1}; group g of the tile (per term and weight, in order) lives in
// slot g mod 4, and its first MMA waits until the epilogue has drained group
// g - 4.  Within a band the pairs go by pairs of A digits, smallest first, so
// that each group's last pair (its largest s) comes in order of weight and
// the groups complete, and are drained, one after another while the tensor
// core works on the rest of the band.
// Operands: for each pair of consecutive digits (s, s + 1) of A and each
// 128-wide K chunk, the two 128 x 128 chunks of those digit slices stay in
// shared memory (four chunk buffers) while the matching chunks of the B digit
// slices t of the union of their runs stream once through a 3-stage TMA ring,
// each stage feeding the pairs (s, t) and (s + 1, t) (8 MMAs each).
//
// Epilogue (8 warps; warp w reads TMEM lanes 32 (w mod 4) .. + 31 and one
// 64-column half): each group is added, exactly, into a 64-bit fixed-point
// accumulator per element in units of 2^-52 of the scaled product
// (|scaled product| < 2^11), and the sum is converted to FP64 once:
//   RESID:  writes R^T with R = I - A B (transposed store, coalesced) and
//           adds sum |R_ij|^2 into a per-matrix FP64 accumulator.
//   CORR:   X <- X + A B, written to X (row-major) and X^T; the old value is
//           read from X^T, whose accesses are coalesced across the lanes.
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
constexpr int BN = 128;       // output tile columns (rows: tc::BM = 128)
constexpr int KB = 64;        // BF16 elements per k-block (one 128-byte row)
constexpr int KP_ALIGN = 128; // the padded K (digit-array pitch) is a multiple of this
constexpr int K_MAX = 512;    // largest inner dimension with exact FP32 accumulation
constexpr int CHUNK_KB = 2;                                // k-blocks per K chunk (128 K)
constexpr int A_BOX_BYTES = tc::BM * KB * 2;               // 16 KB
constexpr int A_CHUNK_BYTES = A_BOX_BYTES * CHUNK_KB;      // 32 KB
constexpr int A_BUFS = 4;                                  // A chunk buffers (two digits in use, two loading)
constexpr int A_RES_BYTES = A_BUFS * A_CHUNK_BYTES;
constexpr int B_BOX_BYTES = BN * KB * 2;                   // 16 KB
constexpr int B_STAGE_BYTES = B_BOX_BYTES * CHUNK_KB;      // 32 KB: 8 MMAs per stage
constexpr int B_STAGES = 3;
constexpr int SLOTS = 4;                                   // 128-column TMEM accumulators
constexpr int EPI_WARPS = 8;
constexpr int THREADS = 64 + 32 * EPI_WARPS;               // producer, MMA, epilogue warps
constexpr int NUM_BARS = 2 * B_STAGES + 2 * A_BUFS + 2 * SLOTS + 1;
constexpr int SMEM_BYTES = A_RES_BYTES + B_STAGES * B_STAGE_BYTES + 1024 + NUM_BARS * 8 + 16;
static_assert(SMEM_BYTES <= 232448, "shared memory per CTA");
static_assert(KP_ALIGN == KB * CHUNK_KB, "one B stage per (digit pair, K chunk)");

// ---------------------------------------------------------------- split
// src: two real FP64 matrices per batch entry (rows x K, row-major, ld, batch
// stride bs, part stride ps); dst digits: BF16 [part][s][b][row][Kp]
// (zero-padded to Kp, Kp a multiple of 128, K <= K_MAX); exps: int
// [part][b][row].  The real and imaginary rows share one exponent (the
// larger), so that the two real products of one complex output part carry
// the same row and column scales.
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

// One warp per row pair (real and imaginary).  Each lane keeps its 16
// entries of each row (4 consecutive columns in each 128-wide block) in
// registers between the maximum and the digit passes.  S is a template
// parameter so that every digit shift is a constant.
template <int S>
__global__ void __launch_bounds__(256) oz_split_rows_kernel(int rows, int K, int Kp, int batch, const double* src,
                                                            int64_t ld, int64_t bs, int64_t ps, __nv_bfloat16* dst,
                                                            int* exps, const int* skip) {
  constexpr int NP = 2;
  constexpr int NJ = K_MAX / 128;
  const int warp = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (warp >= rows * batch) return;
  const int row = warp % rows;
  const int b = warp / rows;
  if (skip && skip[b]) return;
  const int part0 = 0;
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
#pragma unroll
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
#pragma unroll
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
  int Su;         // leading digits used (<= S, 2..8): pairs s, t <= Su with s + t <= Su + 1
  const int* expA;  // [2][batch][n] (joint: equal for both parts)
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

// x 2^e as an FP64 number (round to nearest even), with integer operations
// only (the FP64 pipe of this GPU retires about two lanes per clock per SM,
// so FP64 conversions in an epilogue would idle the tensor core).  |x| < 2^63;
// results below the normal range flush to zero.  The FP32 value (truncated,
// for sums of squares) is returned in *f.
__device__ __forceinline__ double i64_ldexp(long long x, int e, float* f) {
  if (x == 0) {
    *f = 0.f;
    return 0.0;
  }
  const unsigned long long sign = x < 0 ? (1ull << 63) : 0ull;
  unsigned long long m = x < 0 ? (unsigned long long)(-x) : (unsigned long long)x;
  const int lz = __clzll((long long)m);
  m <<= lz;                                     // leading bit at 63
  int be = 63 - lz + e + 1023;                  // biased exponent of the leading bit
  const int fe = be - 1023 + 127;
  *f = fe <= 0 ? 0.f : (fe >= 255 ? __int_as_float(0x7F800000) : __int_as_float((fe << 23) | (int)((m >> 40) & 0x7FFFFF)));
  unsigned long long q = m >> 11;               // 53 bits
  const unsigned long long rem = m & 0x7FFull;
  if (rem > 0x400ull || (rem == 0x400ull && (q & 1ull))) q += 1;
  if (q >> 53) {
    q >>= 1;
    be += 1;
  }
  if (be <= 0) return __longlong_as_double((long long)sign);
  if (be >= 2047) return __longlong_as_double((long long)(sign | 0x7FF0000000000000ull));
  return __longlong_as_double((long long)(sign | ((unsigned long long)be << 52) | (q & 0xFFFFFFFFFFFFFull)));
}

// The pair schedule shared by the producer and the MMA issuer: for each term,
// band, digit s of A (with a non-empty run of B digits t in the band), K chunk
// ch, and t in the run.  Band b covers the weights w = s + t in
// [2 + W b, min(1 + W (b + 1), Su + 1)], W = BAND_W.  Group g = term Su + w - 2
// of the tile (one per weight and term) lives in TMEM slot g mod 4, so a
// group's first MMA waits until the epilogue has drained group g - 4.
constexpr int BAND_W = 4;
__device__ __forceinline__ int num_bands(int Su) { return (Su + BAND_W - 1) / BAND_W; }
__device__ __forceinline__ int band_lo(int band) { return 2 + BAND_W * band; }
__device__ __forceinline__ int band_hi(int band, int Su) {
  return 1 + BAND_W * (band + 1) < Su + 1 ? 1 + BAND_W * (band + 1) : Su + 1;
}

// Tiles of the launch: t -> (x tile, y tile, z = 2 b + part), x fastest.
struct TileIdx {
  int b, part, m0, n0;
};
__device__ __forceinline__ TileIdx tile_of(int t, int nx, int ny) {
  TileIdx r;
  const int xt = t % nx;
  const int rest = t / nx;
  const int yt = rest % ny;
  const int z = rest / ny;
  r.b = z >> 1;
  r.part = z & 1;
  r.m0 = yt * tc::BM;
  r.n0 = xt * BN;
  return r;
}

// Persistent: CTA c takes tiles c, c + gridDim.x, ...; tiles of converged or
// failed matrices are skipped by every role alike.  The pipelines (A chunks,
// B stages, TMEM slots) run on across tiles, so the epilogue's final stores of
// one tile overlap the MMAs of the next.
template <int MODE>
__global__ void __launch_bounds__(THREADS, 1)
    oz_cgemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, OzArgs args) {
  using namespace tc;
  extern __shared__ __align__(1024) unsigned char smraw[];
  const int n = args.n, S = args.S, batch = args.batch, Su = args.Su;
  const int nx = (n + BN - 1) / BN, ny = (n + BM - 1) / BM;
  const int ntiles = nx * ny * 2 * batch;

  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
  unsigned char* a_res = base;
  unsigned char* b_ring = base + A_RES_BYTES;
  uint64_t* bars = reinterpret_cast<uint64_t*>(b_ring + B_STAGES * B_STAGE_BYTES);
  uint64_t* b_full = bars;
  uint64_t* b_empty = bars + B_STAGES;
  uint64_t* a_full = bars + 2 * B_STAGES;  // [A_BUFS]
  uint64_t* a_empty = a_full + A_BUFS;     // [A_BUFS]
  uint64_t* slot_full = a_empty + A_BUFS;  // [SLOTS]: group complete (MMA -> epilogue)
  uint64_t* slot_empty = slot_full + SLOTS;  // [SLOTS]: group drained (epilogue -> MMA)
  uint64_t* mma_done = slot_empty + SLOTS;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mma_done + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nch = args.Kp / (KB * CHUNK_KB);

  if (threadIdx.x == 0) {
    for (int i = 0; i < B_STAGES; ++i) {
      mbar_init(&b_full[i], 1);
      mbar_init(&b_empty[i], 1);
    }
    for (int i = 0; i < A_BUFS; ++i) {
      mbar_init(&a_full[i], 1);
      mbar_init(&a_empty[i], 1);
    }
    for (int i = 0; i < SLOTS; ++i) {
      mbar_init(&slot_full[i], 1);
      mbar_init(&slot_empty[i], EPI_WARPS);
    }
    mbar_init(mma_done, 1);
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

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- producer: A chunks and B stages in schedule order
      int bi = 0, ai = 0;
      bool ok = true;
      for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const TileIdx T = tile_of(tile, nx, ny);
        if (args.skip && args.skip[T.b]) continue;
        for (int term = 0; term < 2 && ok; ++term) {
          const int ap = term, bp = term ? (T.part ^ 1) : T.part;
          for (int band = 0; band < num_bands(Su) && ok; ++band) {
            const int lo = band_lo(band), hi = band_hi(band, Su);
            const int sa = lo - Su > 1 ? lo - Su : 1, sb = hi - 1 < Su ? hi - 1 : Su;  // digits with a run
            for (int s1 = sa; s1 <= sb && ok; s1 += 2) {
              const int s2 = s1 + 1 <= sb ? s1 + 1 : 0;
              const int slead = s2 ? s2 : s1;
              const int tlo = lo - slead > 1 ? lo - slead : 1;
              const int thi = hi - s1 < Su ? hi - s1 : Su;
              for (int ch = 0; ch < nch && ok; ++ch) {
                for (int q2 = 0; q2 < (s2 ? 2 : 1) && ok; ++q2) {
                  const int s = q2 == 0 ? slead : s1;
                  const int slot = ai % A_BUFS;
                  if (ai >= A_BUFS && !mbar_wait(&a_empty[slot], ((ai / A_BUFS) - 1) & 1)) { ok = false; break; }
                  mbar_arrive_expect_tx(&a_full[slot], (uint32_t)A_CHUNK_BYTES);
#pragma unroll
                  for (int q = 0; q < CHUNK_KB; ++q)
                    tma_load_3d(a_res + slot * A_CHUNK_BYTES + q * A_BOX_BYTES, &mapA, &a_full[slot],
                                (ch * CHUNK_KB + q) * KB, T.m0, (ap * S + (s - 1)) * batch + T.b);
                  ++ai;
                }
                for (int t = tlo; t <= thi && ok; ++t) {
                  const int st = bi % B_STAGES;
                  if (bi >= B_STAGES && !mbar_wait(&b_empty[st], ((bi / B_STAGES) - 1) & 1)) { ok = false; break; }
                  mbar_arrive_expect_tx(&b_full[st], (uint32_t)B_STAGE_BYTES);
#pragma unroll
                  for (int q = 0; q < CHUNK_KB; ++q)
                    tma_load_3d(b_ring + st * B_STAGE_BYTES + q * B_BOX_BYTES, &mapB, &b_full[st],
                                (ch * CHUNK_KB + q) * KB, T.n0, (bp * S + (t - 1)) * batch + T.b);
                  ++bi;
                }
              }
            }
          }
        }
      }
      if (!ok) {
        atomicExch(args.err, FROB_ERR_TIMEOUT);
        // let the copies already issued land before the CTA can leave
        for (int j = (bi > B_STAGES ? bi - B_STAGES : 0); j < bi; ++j)
          mbar_wait(&b_full[j % B_STAGES], (j / B_STAGES) & 1);
        for (int j = (ai > A_BUFS ? ai - A_BUFS : 0); j < ai; ++j) mbar_wait(&a_full[j % A_BUFS], (j / A_BUFS) & 1);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer
      constexpr uint32_t IDESC = instr_desc<0, BN>();
      int bi = 0, ai = 0;
      int g0 = 0;  // groups of the earlier tiles of this CTA
      bool ok = true;
      const int nb = num_bands(Su);
      for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const TileIdx T = tile_of(tile, nx, ny);
        if (args.skip && args.skip[T.b]) continue;
        for (int term = 0; term < 2 && ok; ++term) {
          const int gt = g0 + term * Su;  // group of weight 2 of this term
          for (int band = 0; band < nb && ok; ++band) {
            const int lo = band_lo(band), hi = band_hi(band, Su);
            const int sa = lo - Su > 1 ? lo - Su : 1, sb = hi - 1 < Su ? hi - 1 : Su;
            uint32_t started = 0;  // weights of this band whose accumulator has been initialised
            for (int s1 = sa; s1 <= sb && ok; s1 += 2) {
              const int s2 = s1 + 1 <= sb ? s1 + 1 : 0;
              const int slead = s2 ? s2 : s1;
              const int tlo = lo - slead > 1 ? lo - slead : 1;
              const int thi = hi - s1 < Su ? hi - s1 : Su;
              // runs: s1 over [t1lo, thi], s2 over [tlo, t2hi]
              const int t1lo = lo - s1 > 1 ? lo - s1 : 1;
              const int t2hi = s2 ? (hi - s2 < Su ? hi - s2 : Su) : 0;
              for (int ch = 0; ch < nch && ok; ++ch) {
                int slot2 = 0;
                if (s2) {
                  slot2 = ai % A_BUFS;
                  if (!mbar_wait(&a_full[slot2], (ai / A_BUFS) & 1)) { ok = false; break; }
                  ++ai;
                }
                const int slot1 = ai % A_BUFS;
                if (!mbar_wait(&a_full[slot1], (ai / A_BUFS) & 1)) { ok = false; break; }
                ++ai;
                tc_fence_after();
                for (int t = tlo; t <= thi && ok; ++t) {
                  const int st = bi % B_STAGES;
                  if (!mbar_wait(&b_full[st], (bi / B_STAGES) & 1)) { ok = false; break; }
                  tc_fence_after();
                  const uint32_t sbs = smem_u32(b_ring + st * B_STAGE_BYTES);
                  for (int q2 = 0; q2 < 2; ++q2) {
                    const int s = q2 == 0 ? s1 : s2;
                    if (q2 == 0 ? (t < t1lo) : (s2 == 0 || t > t2hi)) continue;
                    const int w = s + t;
                    const int g = gt + (w - 2);
                    if (!((started >> w) & 1u) && g >= SLOTS) {
                      // first MMA of group g: slot g mod 4 must be drained of group g - 4
                      if (!mbar_wait(&slot_empty[g % SLOTS], ((g / SLOTS) - 1) & 1)) { ok = false; break; }
                      tc_fence_after();
                    }
                    const uint32_t sas = smem_u32(a_res + (q2 == 0 ? slot1 : slot2) * A_CHUNK_BYTES);
                    const uint32_t dt = tmem + (uint32_t)((g % SLOTS) * BN);
#pragma unroll
                    for (int q = 0; q < CHUNK_KB; ++q)
#pragma unroll
                      for (int kk = 0; kk < KB / 16; ++kk) {
                        const uint64_t ad = sw128_desc(sas + q * A_BOX_BYTES + kk * 32);
                        const uint64_t bd = sw128_desc(sbs + q * B_BOX_BYTES + kk * 32);
                        mma<0>(dt, ad, bd, IDESC, ((started >> w) & 1u));
                        started |= 1u << w;
                      }
                  }
                  mma_commit(&b_empty[st]);
                  ++bi;
                  if (s2 && t == t2hi) mma_commit(&a_empty[slot2]);  // s2's last pair of this chunk
                }
                mma_commit(&a_empty[slot1]);
              }
              // groups whose last pair has A digit s1 or s2 are complete
              if (ok)
                for (int w = lo; w <= hi; ++w) {
                  const int slast = w - 1 < Su ? w - 1 : Su;
                  if (slast == s1 || (s2 && slast == s2)) mma_commit(&slot_full[(gt + (w - 2)) % SLOTS]);
                }
            }
          }
        }
        g0 += 2 * Su;
      }
      if (!ok) atomicExch(args.err, FROB_ERR_TIMEOUT);
      mma_commit(mma_done);
      mbar_wait(mma_done, 0);  // every MMA of this CTA has finished with TMEM and shared memory
    }
  } else {
    // ---------------- epilogue: warps 2..9 -> TMEM lanes 32 (warp % 4) .., column half
    const int quarter = warp & 3;
    const int half = (warp - 2) >> 2;
    const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(half * 64);
    const int64_t nn = (int64_t)n * n;
    int g0 = 0;
    bool ok = true;
    for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
      const TileIdx T = tile_of(tile, nx, ny);
      if (args.skip && args.skip[T.b]) continue;
      const int b = T.b, part = T.part;
      const int row = T.m0 + quarter * 32 + lane;
      const float sg1 = part == 0 ? -1.f : 1.f;  // - Ai Bi (re), + Ai Br (im)
      long long acc[64];
#pragma unroll
      for (int c = 0; c < 64; ++c) acc[c] = 0;
      for (int gl = 0; gl < 2 * Su; ++gl) {  // groups complete in this order
        const int g = g0 + gl;
        const int slot = g % SLOTS;
        if (!mbar_wait(&slot_full[slot], (g / SLOTS) & 1)) { ok = false; break; }
        tc_fence_after();
        const int term = gl / Su;
        const int w = gl % Su + 2;
        const float sgn = term ? sg1 : 1.f;
        const int sh = 52 - 7 * w;
        const float pre = sh < 0 ? sgn * pow2f(sh) : sgn;
        const int lsh = sh < 0 ? 0 : sh;
#pragma unroll
        for (int c0 = 0; c0 < 64; c0 += 16) {
          float v[16];
          tmem_ld16(lane_base + (uint32_t)(slot * BN + c0), v);
#pragma unroll
          for (int i = 0; i < 16; ++i)
            acc[c0 + i] += (long long)((unsigned long long)(long long)__float2int_rn(v[i] * pre) << lsh);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&slot_empty[slot])) : "memory");
      }
      g0 += 2 * Su;
      if (!ok) break;
      // the two terms share the row and column exponents (joint splits)
      const int ea = row < n ? args.expA[(int64_t)b * n + row] : 0;
      const int* eB = args.expB + ((int64_t)part * batch + b) * n;
      const int c_base = T.n0 + half * 64;
      if constexpr (MODE == RESID) {
        // R = I - P: off the diagonal the sign bit of P flips; the diagonal
        // (one entry per row) takes an FP64 subtraction.  sum |R_ij|^2 is
        // accumulated in FP32 (a norm for the stopping test).
        float ssf = 0.f;
        double ssd = 0.0;
        if (row < n) {
          double* RT = args.outR + ((int64_t)part * batch + b) * nn;
#pragma unroll
          for (int c = 0; c < 64; ++c) {
            const int col = c_base + c;
            if (col < n) {
              float pf;
              const double pr = i64_ldexp(acc[c], ea + __ldg(eB + col) - 52, &pf);
              if (part == 0 && col == row) {
                const double r = 1.0 - pr;
                RT[(int64_t)col * n + row] = r;
                ssd += r * r;
              } else {
                RT[(int64_t)col * n + row] = __longlong_as_double(__double_as_longlong(pr) ^ (1ll << 63));
                ssf = fmaf(pf, pf, ssf);
              }
            }
          }
        }
        double ss = ssd + (double)ssf;  // every lane takes part in the reduction below
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
        if (lane == 0 && ss != 0.0) atomicAdd(args.rnorm2 + b, ss);
      } else if (row < n) {
        // The old value comes from X^T (equal to X entry for entry, and
        // coalesced across the warp's rows); each batch of CB loads is issued
        // before any store (more would spill at the 168-register cap of ten
        // warps).  X itself is written with 32-byte stores, one full sector
        // of four columns of a row per lane, when n allows.
        double* Xp = args.X + ((int64_t)part * batch + b) * nn;
        double* XTp = args.XT + ((int64_t)part * batch + b) * nn;
        const bool vec = (n & 3) == 0;
        constexpr int CB = 4;
#pragma unroll
        for (int c0 = 0; c0 < 64; c0 += CB) {
          double v[CB];
#pragma unroll
          for (int i = 0; i < CB; ++i) {
            const int col = c_base + c0 + i;
            v[i] = col < n ? XTp[(int64_t)col * n + row] : 0.0;
          }
#pragma unroll
          for (int i = 0; i < CB; ++i) {
            const int col = c_base + c0 + i;
            if (col < n) {
              float pf;
              v[i] += i64_ldexp(acc[c0 + i], ea + __ldg(eB + col) - 52, &pf);
              XTp[(int64_t)col * n + row] = v[i];
            }
          }
#pragma unroll
          for (int i = 0; i < CB; i += 4) {
            const int col = c_base + c0 + i;
            double* dst = Xp + (int64_t)row * n + col;
            if (vec && col < n) {
              asm volatile("st.global.v4.f64 [%0], {%1, %2, %3, %4};" ::"l"(dst), "d"(v[i]), "d"(v[i + 1]),
                           "d"(v[i + 2]), "d"(v[i + 3])
                           : "memory");
            } else {
#pragma unroll
              for (int q = 0; q < 4; ++q)
                if (col + q < n) dst[q] = v[i + q];
            }
          }
        }
      }
    }
    if (!ok && lane == 0) atomicExch(args.err, FROB_ERR_TIMEOUT);
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
