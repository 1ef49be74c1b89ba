// FP64-accurate real matrix products of any size on the BF16 tensor cores, by
// exact splitting of the operands (Ozaki, Ogita, Oishi and Rump, Numer.
// Algorithms 2012, scheme I) -- the real counterpart of ozaki.cuh's complex
// residual products, for the large products of Frobenius inversion in FP64
// (S = A + B X1 and X1 S^{-1}, Sec. 4.1, the updates of the recursive LU and
// triangular solves, and the LU panels' rank-32 updates), where this GPU's
// FP64 pipe (about 1.25 TFLOP/s) is the bound of the CUDA-core path.
//
//   D = epilogue(op(A) op(B)),  op(A): M x K,  op(B): K x N,  FP64.
//
// Splitting.  Row i of op(A) is scaled by 2^-ea_i and column j of op(B) by
// 2^-eb_j (2^e the smallest power of two above the largest magnitude of the
// row / column), and every scaled entry r in (-1, 1) is written with S signed
// base-128 digits (S = 8), r = sum_s d_s 2^(-7 s) + (remainder below 2^(-7 S - 1)),
// |d_1| <= 128, |d_s| <= 64 (s >= 2), exact in BF16 (the same integer
// construction as ozaki.cuh: one rounding of r 2^(7 S) to an integer, then
// balanced digits by shifts).  The digit planes are K-major: A's rows, and
// op(B)'s columns, with K contiguous, padded to a multiple of 128 with zeros.
//
// Products.  The pairs (s, t) with s + t <= S + 1 are accumulated per weight
// 2^(-7 (s + t)) in FP32 in TMEM ("groups", as in ozaki.cuh), over K
// chunks of at most 512: within a chunk every group sum with s + t <= 7 is an
// integer below 2^24 (exact), and the groups of weight 2^-56 and below lie
// under the result's FP64 unit.  Each group of each chunk is added into a
// 64-bit fixed-point accumulator per output element, in units of 2^-U of the
// scaled product (rounded to nearest where the group's weight is below the
// unit), and the accumulator is converted to FP64 once (integer operations)
// and handed to the element-wise epilogue.  The unit is as fine as overflow
// allows: with an integer q_k >= 2^12 sum_s |d_s| 2^(-7 s) per scaled entry
// (from its first two digits; at least 2^12 times its magnitude), every partial sum of digit products of row i and
// column j is at most sum_k q_k q'_k 2^-24 <= |q| |q'| 2^-24 (Cauchy-Schwarz),
// and the split kernels accumulate sum_k q_k^2 per row and column exactly as
// integers; U is the largest integer with |q| |q'| 2^-24 <= 2^(62 - U) for the
// row and the largest of an epilogue warp's 64 columns, which keeps every
// partial sum below 2^62 units.  For Gaussian rows |q| 2^-12 is about
// sqrt(K) / 4, so U is about 66 - log2 K.  Relative to the row and column
// scales the result is within about 2^-57 sqrt(K) of the exact product
// (digit truncation) plus half a unit per rounded chunk group, the rounding
// of the final FP64 value aside: on Gaussian operands a few times the error
// of the correctly rounded product, against ten or more for FP64 dot products.
//
// Kernel: as oz_cgemm_kernel (persistent CTAs, one per SM; a producer warp
// keeping two consecutive A digits resident per 128-wide K slice in four A
// chunk buffers while the B digit stages of the union of their runs stream
// once through a 3-stage TMA ring, an MMA warp, eight epilogue warps;
// 128 x 128 tiles; four 128-column TMEM slots, group g in slot g mod 4;
// weights in bands of four), with one real term per tile and an outer loop
// over the 512-wide K chunks.  Every mbarrier wait is
// bounded (tc::mbar_wait); a wait that gives up sets the caller's flag to
// FROB_ERR_TIMEOUT, the producer lets its copies land and the CTA returns.
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "common.cuh"
#include "ozaki.cuh"
#include "tc_gemm.cuh"

namespace frob {
namespace ozr {

// digits per operand: eight (56 bits relative to the row / column maximum;
// pairs s + t <= 9, 36 products per chunk), so that each product is at least
// as accurate as an FP64 product (seven digits, 49 bits, lost up to ~20x
// against FP64 in the cancelling updates of triangular solves)
constexpr int S_DIG = 8;
constexpr int KC = 512;           // K per exact chunk
constexpr int MIN_MNK = 256;      // products at least this large in every dimension take the digit path ...
// ... and so do smaller ones with M, N >= MIN_MN_THIN and M N K >= THIN_MIN_MNK
// (the rank-32 updates of LU panels and the diagonal blocks of the recursive
// triangular solves): a digit product costs about 70 us plus 14 us per 10^6
// M N and 128-wide K slice, the FP64 pipe about 105 us per 10^6 M N and 32 K
constexpr int MIN_MN_THIN = 128;
constexpr int64_t THIN_MIN_MNK = 24ll << 20;
constexpr int SUB = KC / (oz::KB * oz::CHUNK_KB);  // 128-wide sub-chunks per chunk (4)
constexpr int SMALL_KP = 128;     // K up to this: split in one pass (ozr_digits_small_kernel)
// shared memory of ozr_gemm_kernel: four resident A chunks (two digits in use,
// two loading) and three B stages of 32 KB each
constexpr int R_A_BUFS = 4;
constexpr int R_B_STAGES = 3;
constexpr int R_SMEM_BYTES = (R_A_BUFS + R_B_STAGES) * oz::A_CHUNK_BYTES + 1024 +
                             (2 * R_B_STAGES + 2 * R_A_BUFS + 2 * oz::SLOTS + 1) * 8 + 16;
static_assert(oz::A_CHUNK_BYTES == oz::B_STAGE_BYTES, "A chunks and B stages of one size");
static_assert(R_SMEM_BYTES <= 232448, "shared memory per CTA");
constexpr int EPI_W = 4;          // output columns per epilogue block
// exponent of a row / column that holds an infinity or a NaN: its digits are
// zero and every product entry it touches is NaN, as on the CUDA cores
constexpr int NONFINITE_EXP = 0x40000000;

struct RArgs {
  int M, N, Kp, batch;
  int S, Su;          // digits in the arrays / used
  const int* expA;    // [batch][M]
  const int* expB;    // [batch][N]
  const unsigned long long* sqA;  // [batch][M]: sum_k q_k^2 of each row's digits
  const unsigned long long* sqB;  // [batch][N]
  int* err;
};

// ---------------------------------------------------------------- split
// (The exponents, e_r = smallest integer with max_k |X_rk| < 2^e_r, come
// from ozr_exp_kernel in ozr.cu.)
// Digits: dst[s][b][r][Kp] (BF16) of X 2^-e_r, k in [K, Kp) zero; 32 x 32
// tiles through shared memory so that both sides are accessed along their
// contiguous dimension, DIG_KT tiles along k per block.  Each row's
// sum_k q_k^2 (q_k >= 2^12 sum_s |d_s| 2^(-7 s)) is added into sq[b][r]
// (zeroed by the caller) with one integer atomic per row and block.
// grid (ceil(Kp / (32 DIG_KT)), ceil(R / 32), batch), 256 threads.
constexpr int DIG_KT = 1;
template <int S>
__global__ void __launch_bounds__(256) ozr_digits_kernel(int R, int K, int Kp, int batch, const double* src,
                                                         int64_t ld, int64_t sb, int trans, const int* exps,
                                                         __nv_bfloat16* dst, unsigned long long* sq) {
  __shared__ double tile[32][33];
  const int b = blockIdx.z;
  const int r0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const double* sbp = src + (int64_t)b * sb;
  long long off = 0;  // 64 (1 + 128 + ... + 128^(S-2))
#pragma unroll
  for (int j = 0; j < S - 1; ++j) off = (off << 7) + 64;
  const int64_t plane = (int64_t)batch * R * Kp;
  unsigned int q2[4] = {0u, 0u, 0u, 0u};  // rows r0 + ty + 8 j
  for (int kt = 0; kt < DIG_KT; ++kt) {
    const int k0 = (blockIdx.x * DIG_KT + kt) * 32;
    if (k0 >= Kp) break;
    if (kt) __syncthreads();
    for (int i = ty; i < 32; i += 8) {
      if (trans) {
        const int k = k0 + i, r = r0 + tx;
        tile[i][tx] = (k < K && r < R) ? sbp[(int64_t)k * ld + r] : 0.0;
      } else {
        const int r = r0 + i, k = k0 + tx;
        tile[i][tx] = (k < K && r < R) ? sbp[(int64_t)r * ld + k] : 0.0;
      }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 4; ++j) {  // a warp: one row r, 32 consecutive k
      const int i = ty + 8 * j;
      const int r = r0 + i, k = k0 + tx;
      if (r >= R || k >= Kp) continue;
      const double x = trans ? tile[tx][i] : tile[i][tx];
      const int e = exps[(int64_t)b * R + r];
      const long long G = oz::scaled_fixed(x, 7 * S - e) + off;
      __nv_bfloat16* out = dst + ((int64_t)b * R + r) * Kp + k;
      int d1 = 0, d2 = 0;
#pragma unroll
      for (int sl = 0; sl < S; ++sl) {
        const int sh = 7 * (S - 1 - sl);
        const int d = sl == 0 ? (int)(G >> sh) : (int)((G >> sh) & 127) - 64;
        reinterpret_cast<uint16_t*>(out)[(int64_t)sl * plane] = (uint16_t)oz::bf16_bits_of_int(d);
        if (sl == 0) d1 = d < 0 ? -d : d;
        if (sl == 1) d2 = d < 0 ? -d : d;
      }
      // 2^12 sum_s |d_s| 2^(-7 s) <= 32 |d_1| + |d_2| / 4 + 2^-2.99 (the
      // digits after the second are at most 64): q = 32 |d_1| + ceil((|d_2| + 1) / 4)
      // <= 4113, q^2 < 2^24.02
      const unsigned int q = 32u * (unsigned)d1 + (((unsigned)d2 + 4u) >> 2);
      q2[j] += q * q;
    }
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int r = r0 + ty + 8 * j;
    unsigned long long t = q2[j];  // <= 2^26.1 per lane
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (tx == 0 && r < R && t != 0) atomicAdd(sq + (int64_t)b * R + r, t);
  }
}

// Thin operands (K <= SMALL_KP, so Kp = SMALL_KP): one block per 32 rows
// computes each row's exponent (as ozr_absmax / ozr_exp_final), its digits and
// its sum_k q_k^2 in one pass, writing exps and sq directly (no atomics).
// grid (ceil(R / 32), batch), 256 threads.
template <int S>
__global__ void __launch_bounds__(256) ozr_digits_small_kernel(int R, int K, int batch, const double* src, int64_t ld,
                                                               int64_t sb, int trans, int* exps, __nv_bfloat16* dst,
                                                               unsigned long long* sq) {
  constexpr int KP = SMALL_KP;
  __shared__ double tile[32][KP + 1];
  const int b = blockIdx.y;
  const int r0 = blockIdx.x * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const double* sbp = src + (int64_t)b * sb;
  if (trans) {
    for (int k = ty; k < KP; k += 8) {
      const int r = r0 + tx;
      tile[tx][k] = (k < K && r < R) ? sbp[(int64_t)k * ld + r] : 0.0;
    }
  } else {
    for (int i = ty; i < 32; i += 8) {
      const int r = r0 + i;
#pragma unroll
      for (int q = 0; q < KP / 32; ++q) {
        const int k = q * 32 + tx;
        tile[i][k] = (k < K && r < R) ? sbp[(int64_t)r * ld + k] : 0.0;
      }
    }
  }
  __syncthreads();
  long long off = 0;  // 64 (1 + 128 + ... + 128^(S-2))
#pragma unroll
  for (int j = 0; j < S - 1; ++j) off = (off << 7) + 64;
  const int64_t plane = (int64_t)batch * R * KP;
  for (int i = ty; i < 32; i += 8) {  // a warp: one row
    const int r = r0 + i;
    if (r >= R) break;                 // uniform in the warp
    unsigned long long m = 0;
#pragma unroll
    for (int q = 0; q < KP / 32; ++q) {
      const unsigned long long a = (unsigned long long)__double_as_longlong(tile[i][q * 32 + tx]) & 0x7FFFFFFFFFFFFFFFull;
      m = a > m ? a : m;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long t = __shfl_xor_sync(0xffffffffu, m, o);
      m = t > m ? t : m;
    }
    const int mex = (int)(m >> 52);
    int e = 0;
    if (mex == 0x7FF) e = NONFINITE_EXP;
    else if (m != 0) e = (mex == 0) ? -1022 : mex - 1022;
    unsigned int q2 = 0;
    __nv_bfloat16* out = dst + ((int64_t)b * R + r) * KP;
#pragma unroll
    for (int q = 0; q < KP / 32; ++q) {
      const int k = q * 32 + tx;
      const long long G = oz::scaled_fixed(tile[i][k], 7 * S - e) + off;
      int d1 = 0, d2 = 0;
#pragma unroll
      for (int sl = 0; sl < S; ++sl) {
        const int sh = 7 * (S - 1 - sl);
        const int d = sl == 0 ? (int)(G >> sh) : (int)((G >> sh) & 127) - 64;
        reinterpret_cast<uint16_t*>(out + k)[(int64_t)sl * plane] = (uint16_t)oz::bf16_bits_of_int(d);
        if (sl == 0) d1 = d < 0 ? -d : d;
        if (sl == 1) d2 = d < 0 ? -d : d;
      }
      const unsigned int qk = 32u * (unsigned)d1 + (((unsigned)d2 + 4u) >> 2);  // as ozr_digits_kernel
      q2 += qk * qk;
    }
    unsigned long long t = q2;  // <= 4 x 2^24.02 per lane
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (tx == 0) {
      exps[(int64_t)b * R + r] = e;
      sq[(int64_t)b * R + r] = t;
    }
  }
}

// Fixed-point unit exponent U for a row and column whose digits' sums of
// squares are sa and sb: the largest U with 2^(62 - U) >= (sa sb)^(1/2) 2^-24,
// i.e. U = 62 - (ceil(log2(sa sb) / 2) - 24), from the exact 128-bit product
// (62 when either is 0: every product is zero).
__device__ __forceinline__ int unit_exponent(unsigned long long sa, unsigned long long sb) {
  if (sa == 0 || sb == 0) return 62;
  unsigned long long lo = sa * sb, hi = __umul64hi(sa, sb);
  if (lo == 0) {  // P - 1
    hi -= 1;
    lo = ~0ull;
  } else {
    lo -= 1;
  }
  const int cl = hi ? 128 - __clzll((long long)hi) : (lo ? 64 - __clzll((long long)lo) : 0);  // ceil(log2 P)
  return 62 - ((cl + 1) / 2 - 24);
}

// ---------------------------------------------------------------- product
// Tiles t -> (x tile, y tile, matrix), x fastest.  Per tile: for each K chunk
// c, band, digit s of A (with a non-empty run of B digits t in the band),
// 128-wide sub-chunk of c, and t in the run.  Group g = (tile's first group)
// + c Su + (s + t - 2) lives in TMEM slot g mod 4.
template <class Epi>
__global__ void __launch_bounds__(oz::THREADS, 1)
    ozr_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, RArgs args,
                    Epi epi) {
  using namespace tc;
  using oz::A_BOX_BYTES; using oz::A_CHUNK_BYTES; using oz::B_BOX_BYTES; using oz::B_STAGE_BYTES;
  using oz::CHUNK_KB; using oz::EPI_WARPS; using oz::KB; using oz::SLOTS;
  constexpr int A_BUFS = R_A_BUFS, B_STAGES = R_B_STAGES, A_RES_BYTES = R_A_BUFS * A_CHUNK_BYTES;
  constexpr int BN = oz::BN;
  extern __shared__ __align__(1024) unsigned char smraw[];
  const int M = args.M, N = args.N, S = args.S, batch = args.batch, Su = args.Su;
  const int nx = (N + BN - 1) / BN, ny = (M + BM - 1) / BM;
  const int ntiles = nx * ny * batch;
  const int nsub = args.Kp / (KB * CHUNK_KB);   // 128-wide sub-chunks
  const int nch = (nsub + SUB - 1) / SUB;      // exact chunks of up to KC
  const int gpt = nch * Su;                    // groups per tile

  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
  unsigned char* a_res = base;
  unsigned char* b_ring = base + A_RES_BYTES;
  uint64_t* bars = reinterpret_cast<uint64_t*>(b_ring + B_STAGES * B_STAGE_BYTES);
  uint64_t* b_full = bars;
  uint64_t* b_empty = bars + B_STAGES;
  uint64_t* a_full = bars + 2 * B_STAGES;
  uint64_t* a_empty = a_full + A_BUFS;
  uint64_t* slot_full = a_empty + A_BUFS;
  uint64_t* slot_empty = slot_full + SLOTS;
  uint64_t* mma_done = slot_empty + SLOTS;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mma_done + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

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

  // Schedule, shared by the producer and the MMA issuer: per chunk, band and
  // pair of consecutive A digits (s1, s2 = s1 + 1; s1 alone at the end of an
  // odd range) and 128-wide sub-chunk ch, the A chunks of s2 and s1 (in that
  // order) are resident and the B digits t of the union of their runs stream
  // past once, each feeding the pairs (s1, t) and (s2, t) of the band.
  if (warp == 0) {
    if (lane == 0) {
      // ---------------- producer
      int bi = 0, ai = 0;
      bool ok = true;
      for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const int xt = tile % nx, yt = (tile / nx) % ny, b = tile / (nx * ny);
        const int m0 = yt * BM, n0 = xt * BN;
        for (int c = 0; c < nch && ok; ++c) {
          const int ch0 = c * SUB, ch1 = (ch0 + SUB < nsub) ? ch0 + SUB : nsub;
          for (int band = 0; band < oz::num_bands(Su) && ok; ++band) {
            const int lo = oz::band_lo(band), hi = oz::band_hi(band, Su);
            const int sa = lo - Su > 1 ? lo - Su : 1, sb = hi - 1 < Su ? hi - 1 : Su;  // digits with a run
            for (int s1 = sa; s1 <= sb && ok; s1 += 2) {
              const int s2 = s1 + 1 <= sb ? s1 + 1 : 0;
              const int slead = s2 ? s2 : s1;
              const int tlo = lo - slead > 1 ? lo - slead : 1;
              const int thi = hi - s1 < Su ? hi - s1 : Su;
              for (int ch = ch0; ch < ch1 && ok; ++ch) {
                for (int q2 = 0; q2 < (s2 ? 2 : 1) && ok; ++q2) {
                  const int s = q2 == 0 ? slead : s1;
                  const int slot = ai % A_BUFS;
                  if (ai >= A_BUFS && !mbar_wait(&a_empty[slot], ((ai / A_BUFS) - 1) & 1)) { ok = false; break; }
                  mbar_arrive_expect_tx(&a_full[slot], (uint32_t)A_CHUNK_BYTES);
#pragma unroll
                  for (int q = 0; q < CHUNK_KB; ++q)
                    tma_load_3d(a_res + slot * A_CHUNK_BYTES + q * A_BOX_BYTES, &mapA, &a_full[slot],
                                (ch * CHUNK_KB + q) * KB, m0, (s - 1) * batch + b);
                  ++ai;
                }
                for (int t = tlo; t <= thi && ok; ++t) {
                  const int st = bi % B_STAGES;
                  if (bi >= B_STAGES && !mbar_wait(&b_empty[st], ((bi / B_STAGES) - 1) & 1)) { ok = false; break; }
                  mbar_arrive_expect_tx(&b_full[st], (uint32_t)B_STAGE_BYTES);
#pragma unroll
                  for (int q = 0; q < CHUNK_KB; ++q)
                    tma_load_3d(b_ring + st * B_STAGE_BYTES + q * B_BOX_BYTES, &mapB, &b_full[st],
                                (ch * CHUNK_KB + q) * KB, n0, (t - 1) * batch + b);
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
      int g0 = 0;
      bool ok = true;
      const int nb = oz::num_bands(Su);
      for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        for (int c = 0; c < nch && ok; ++c) {
          const int ch0 = c * SUB, ch1 = (ch0 + SUB < nsub) ? ch0 + SUB : nsub;
          const int gc = g0 + c * Su;  // group of weight 2 in this chunk
          for (int band = 0; band < nb && ok; ++band) {
            const int lo = oz::band_lo(band), hi = oz::band_hi(band, Su);
            const int sa = lo - Su > 1 ? lo - Su : 1, sb = hi - 1 < Su ? hi - 1 : Su;
            uint32_t started = 0;
            for (int s1 = sa; s1 <= sb && ok; s1 += 2) {
              const int s2 = s1 + 1 <= sb ? s1 + 1 : 0;
              const int slead = s2 ? s2 : s1;
              const int tlo = lo - slead > 1 ? lo - slead : 1;
              const int thi = hi - s1 < Su ? hi - s1 : Su;
              // runs: s1 over [t1lo, thi], s2 over [tlo, t2hi]
              const int t1lo = lo - s1 > 1 ? lo - s1 : 1;
              const int t2hi = s2 ? (hi - s2 < Su ? hi - s2 : Su) : 0;
              for (int ch = ch0; ch < ch1 && ok; ++ch) {
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
                    const int g = gc + (w - 2);
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
                  if (s2 && t == t2hi) mma_commit(&a_empty[slot2]);  // s2's last pair of this sub-chunk
                }
                mma_commit(&a_empty[slot1]);
              }
              // groups whose last pair has A digit s1 or s2 are complete
              if (ok)
                for (int w = lo; w <= hi; ++w) {
                  const int slast = w - 1 < Su ? w - 1 : Su;
                  if (slast == s1 || (s2 && slast == s2)) mma_commit(&slot_full[(gc + (w - 2)) % SLOTS]);
                }
            }
          }
        }
        g0 += gpt;
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
    int g0 = 0;
    bool ok = true;
    for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
      const int xt = tile % nx, yt = (tile / nx) % ny, b = tile / (nx * ny);
      const int row = yt * BM + quarter * 32 + lane;
      const int c_base = xt * BN + half * 64;
      // fixed-point unit 2^-U of this thread's 64 accumulators, from the sums
      // of squares of its row and of the largest of its columns: every
      // partial sum stays below 2^62 units
      unsigned long long sb = 0;
      if (c_base + lane < N) sb = __ldg(args.sqB + (int64_t)b * N + c_base + lane);
      if (c_base + 32 + lane < N) {
        const unsigned long long t = __ldg(args.sqB + (int64_t)b * N + c_base + 32 + lane);
        sb = t > sb ? t : sb;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(0xffffffffu, sb, o);
        sb = t > sb ? t : sb;
      }
      const int U = unit_exponent(row < M ? __ldg(args.sqA + (int64_t)b * M + row) : 0ull, sb);
      long long acc[64];
#pragma unroll
      for (int c = 0; c < 64; ++c) acc[c] = 0;
      for (int gl = 0; gl < gpt; ++gl) {  // groups complete in this order
        const int g = g0 + gl;
        const int slot = g % SLOTS;
        if (!mbar_wait(&slot_full[slot], (g / SLOTS) & 1)) { ok = false; break; }
        tc_fence_after();
        const int w = gl % Su + 2;
        // the group's FP32 sums are integers below 2^31: rounded to nearest
        // where the weight is below the unit, else shifted up exactly
        const int sh = U - 7 * w;
        const float pre = sh < 0 ? oz::pow2f(sh) : 1.f;
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
      g0 += gpt;
      if (!ok) break;
      if (row < M) {
        const int ea = args.expA[(int64_t)b * M + row];
        const int* eB = args.expB + (int64_t)b * N;
        // EPI_W columns at a time, every load of a block before its stores
#pragma unroll
        for (int c0 = 0; c0 < 64; c0 += EPI_W) {
          int eb[EPI_W];
#pragma unroll
          for (int q = 0; q < EPI_W; ++q) eb[q] = c_base + c0 + q < N ? __ldg(eB + c_base + c0 + q) : 0;
          double v[EPI_W];
#pragma unroll
          for (int q = 0; q < EPI_W; ++q) {
            float pf;
            v[q] = (ea == NONFINITE_EXP || eb[q] == NONFINITE_EXP) ? __longlong_as_double(0x7FF8000000000000ll)
                                                                   : oz::i64_ldexp(acc[c0 + q], ea + eb[q] - U, &pf);
          }
          epi_row<EPI_W>(epi, b, row, c_base + c0, v, N);
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

// ---------------------------------------------------------------- host side (ozr.cu)
int64_t kp_of(int K);
// scratch for one product (digits of both operands, exponents, flag)
size_t scratch_bytes(int M, int N, int K, int batch);
// whether a product of this shape takes the digit path (when scratch allows)
inline bool digit_shape(int M, int N, int K) {
  if (M >= MIN_MNK && N >= MIN_MNK && K >= MIN_MNK) return true;
  return K >= 1 && M >= MIN_MN_THIN && N >= MIN_MN_THIN && (int64_t)M * N * K >= THIN_MIN_MNK;
}
// Splits op(A) (M x K: A[i][k], or A[k][i] with transA) and op(B) (its
// columns: B[k][j], or B[j][k] with transB_rows -- op(B)^T's rows stored
// contiguously) into the scratch and builds the TMA maps and kernel arguments;
// false if a map cannot be encoded.
bool prepare(int M, int N, int K, int batch, const double* A, int64_t lda, int64_t sa, bool transA,
             const double* B, int64_t ldb, int64_t sb, bool b_rows_are_k_major, void* scratch, int* err,
             CUtensorMap* ma, CUtensorMap* mb, RArgs* args, cudaStream_t st);

template <class Epi>
inline cudaError_t launch(const CUtensorMap& ma, const CUtensorMap& mb, const RArgs& a, Epi epi, cudaStream_t st) {
  set_smem_attr(ozr_gemm_kernel<Epi>, R_SMEM_BYTES);
  const int64_t tiles = (int64_t)((a.N + oz::BN - 1) / oz::BN) * ((a.M + tc::BM - 1) / tc::BM) * a.batch;
  if (tiles > INT32_MAX) return cudaErrorInvalidValue;
  const unsigned grid = persistent_grid(tiles);
  FROB_LAUNCH("ozr_gemm<f64 digits>", st,
              ozr_gemm_kernel<Epi><<<grid, oz::THREADS, R_SMEM_BYTES, st>>>(ma, mb, a, epi));
  return cudaGetLastError();
}

}  // namespace ozr
}  // namespace frob
