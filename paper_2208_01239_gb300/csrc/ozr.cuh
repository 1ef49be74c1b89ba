// FP64-accurate real matrix products of any size on the BF16 tensor cores, by
// exact splitting of the operands (Ozaki, Ogita, Oishi and Rump, Numer.
// Algorithms 2012, scheme I) -- the real counterpart of ozaki.cuh's complex
// residual products, for the large products of Frobenius inversion in FP64
// (S = A + B X1 and X1 S^{-1}, Sec. 4.1, and the updates of the recursive
// triangular solves), where this GPU's FP64 pipe (about 1.25 TFLOP/s) is the
// bound of the CUDA-core path.
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
// under the result's FP64 unit.  Each group of each chunk is added exactly
// into a 64-bit fixed-point accumulator per output element, in units of
// 2^-U of the scaled product with U = 62 - ceil(log2 Kp) (at most 52), so
// that no sum over K can overflow; the accumulator is converted to FP64 once
// (integer operations) and handed to the element-wise epilogue.  Relative to
// the row and column scales the result is within about 2^-57 sqrt(K) of the
// exact product (digit truncation) and 2^-U per chunk group (fixed-point
// rounding of the weights below 2^-U): at least the accuracy of an FP64
// product, whose rounding errors are about 2^-53 sqrt(K) of the same scales.
//
// Kernel: as oz_cgemm_kernel (persistent CTAs, one per SM; a producer warp
// with a TMA ring of B digit stages and three resident A digit chunks, an MMA
// warp, eight epilogue warps; 128 x 128 tiles; four 128-column TMEM slots,
// group g in slot g mod 4; weights in bands of four), with one real term per
// tile and an outer loop over the 512-wide K chunks.  Every mbarrier wait is
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
constexpr int MIN_MNK = 256;      // smaller products stay on the CUDA cores
constexpr int SUB = KC / (oz::KB * oz::CHUNK_KB);  // 128-wide sub-chunks per chunk (4)
// exponent of a row / column that holds an infinity or a NaN: its digits are
// zero and every product entry it touches is NaN, as on the CUDA cores
constexpr int NONFINITE_EXP = 0x40000000;

struct RArgs {
  int M, N, Kp, batch;
  int S, Su;          // digits in the arrays / used
  int U;              // fixed-point unit exponent
  const int* expA;    // [batch][M]
  const int* expB;    // [batch][N]
  int* err;
};

// ---------------------------------------------------------------- split
// (The exponents, e_r = smallest integer with max_k |X_rk| < 2^e_r, come
// from ozr_exp_kernel in ozr.cu.)
// Digits: dst[s][b][r][Kp] (BF16) of X 2^-e_r, k in [K, Kp) zero; 32 x 32
// tiles through shared memory so that both sides are accessed along their
// contiguous dimension.  grid (ceil(Kp / 32), ceil(R / 32), batch), 256 threads.
template <int S>
__global__ void __launch_bounds__(256) ozr_digits_kernel(int R, int K, int Kp, int batch, const double* src,
                                                         int64_t ld, int64_t sb, int trans, const int* exps,
                                                         __nv_bfloat16* dst) {
  __shared__ double tile[32][33];
  const int b = blockIdx.z;
  const int r0 = blockIdx.y * 32, k0 = blockIdx.x * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const double* sbp = src + (int64_t)b * sb;
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
  long long off = 0;  // 64 (1 + 128 + ... + 128^(S-2))
#pragma unroll
  for (int j = 0; j < S - 1; ++j) off = (off << 7) + 64;
  const int64_t plane = (int64_t)batch * R * Kp;
  for (int i = ty; i < 32; i += 8) {
    const int r = r0 + i, k = k0 + tx;
    if (r >= R || k >= Kp) continue;
    const double x = trans ? tile[tx][i] : tile[i][tx];
    const int e = exps[(int64_t)b * R + r];
    const long long G = oz::scaled_fixed(x, 7 * S - e) + off;
    __nv_bfloat16* out = dst + ((int64_t)b * R + r) * Kp + k;
#pragma unroll
    for (int sl = 0; sl < S; ++sl) {
      const int sh = 7 * (S - 1 - sl);
      const int d = sl == 0 ? (int)(G >> sh) : (int)((G >> sh) & 127) - 64;
      reinterpret_cast<uint16_t*>(out)[(int64_t)sl * plane] = (uint16_t)oz::bf16_bits_of_int(d);
    }
  }
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
  using oz::A_BOX_BYTES; using oz::A_BUFS; using oz::A_CHUNK_BYTES; using oz::A_RES_BYTES;
  using oz::B_BOX_BYTES; using oz::B_STAGES; using oz::B_STAGE_BYTES; using oz::CHUNK_KB; using oz::EPI_WARPS;
  using oz::KB; using oz::SLOTS;
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
            for (int s = 1; s <= Su && ok; ++s) {
              const int tlo = lo - s > 1 ? lo - s : 1;
              const int thi = hi - s < Su ? hi - s : Su;
              if (tlo > thi) continue;
              const int za = (s - 1) * batch + b;
              for (int ch = ch0; ch < ch1 && ok; ++ch) {
                const int slot = ai % A_BUFS;
                if (ai >= A_BUFS && !mbar_wait(&a_empty[slot], ((ai / A_BUFS) - 1) & 1)) { ok = false; break; }
                mbar_arrive_expect_tx(&a_full[slot], (uint32_t)A_CHUNK_BYTES);
#pragma unroll
                for (int q = 0; q < CHUNK_KB; ++q)
                  tma_load_3d(a_res + slot * A_CHUNK_BYTES + q * A_BOX_BYTES, &mapA, &a_full[slot],
                              (ch * CHUNK_KB + q) * KB, m0, za);
                ++ai;
                for (int t = tlo; t <= thi && ok; ++t) {
                  const int zb = (t - 1) * batch + b;
                  const int st = bi % B_STAGES;
                  if (bi >= B_STAGES && !mbar_wait(&b_empty[st], ((bi / B_STAGES) - 1) & 1)) { ok = false; break; }
                  mbar_arrive_expect_tx(&b_full[st], (uint32_t)B_STAGE_BYTES);
#pragma unroll
                  for (int q = 0; q < CHUNK_KB; ++q)
                    tma_load_3d(b_ring + st * B_STAGE_BYTES + q * B_BOX_BYTES, &mapB, &b_full[st],
                                (ch * CHUNK_KB + q) * KB, n0, zb);
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
            uint32_t started = 0;
            for (int s = 1; s <= Su && ok; ++s) {
              const int tlo = lo - s > 1 ? lo - s : 1;
              const int thi = hi - s < Su ? hi - s : Su;
              if (tlo > thi) continue;
              for (int ch = ch0; ch < ch1 && ok; ++ch) {
                const int aslot = ai % A_BUFS;
                if (!mbar_wait(&a_full[aslot], (ai / A_BUFS) & 1)) { ok = false; break; }
                ++ai;
                tc_fence_after();
                const uint32_t sa = smem_u32(a_res + aslot * A_CHUNK_BYTES);
                for (int t = tlo; t <= thi && ok; ++t) {
                  const int w = s + t;
                  const int g = gc + (w - 2);
                  if (!((started >> w) & 1u) && g >= SLOTS) {
                    // first MMA of group g: slot g mod 4 must be drained of group g - 4
                    if (!mbar_wait(&slot_empty[g % SLOTS], ((g / SLOTS) - 1) & 1)) { ok = false; break; }
                    tc_fence_after();
                  }
                  const int st = bi % B_STAGES;
                  if (!mbar_wait(&b_full[st], (bi / B_STAGES) & 1)) { ok = false; break; }
                  tc_fence_after();
                  const uint32_t sb = smem_u32(b_ring + st * B_STAGE_BYTES);
                  const uint32_t dt = tmem + (uint32_t)((g % SLOTS) * BN);
#pragma unroll
                  for (int q = 0; q < CHUNK_KB; ++q)
#pragma unroll
                    for (int kk = 0; kk < KB / 16; ++kk) {
                      const uint64_t ad = sw128_desc(sa + q * A_BOX_BYTES + kk * 32);
                      const uint64_t bd = sw128_desc(sb + q * B_BOX_BYTES + kk * 32);
                      mma<0>(dt, ad, bd, IDESC, ((started >> w) & 1u));
                      started |= 1u << w;
                    }
                  mma_commit(&b_empty[st]);
                  ++bi;
                }
                mma_commit(&a_empty[aslot]);
              }
              // groups whose last pair was digit s of A are complete
              if (ok)
                for (int t = tlo; t <= thi; ++t) {
                  const int w = s + t;
                  const int slast = w - 1 < Su ? w - 1 : Su;
                  if (s == slast) mma_commit(&slot_full[(gc + (w - 2)) % SLOTS]);
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
    const int U = args.U;
    int g0 = 0;
    bool ok = true;
    for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
      const int xt = tile % nx, yt = (tile / nx) % ny, b = tile / (nx * ny);
      const int row = yt * BM + quarter * 32 + lane;
      long long acc[64];
#pragma unroll
      for (int c = 0; c < 64; ++c) acc[c] = 0;
      for (int gl = 0; gl < gpt; ++gl) {  // groups complete in this order
        const int g = g0 + gl;
        const int slot = g % SLOTS;
        if (!mbar_wait(&slot_full[slot], (g / SLOTS) & 1)) { ok = false; break; }
        tc_fence_after();
        const int w = gl % Su + 2;
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
        const int c_base = xt * BN + half * 64;
#pragma unroll
        for (int c = 0; c < 64; ++c) {
          const int col = c_base + c;
          if (col < N) {
            float pf;
            const int eb = __ldg(eB + col);
            const double v = (ea == NONFINITE_EXP || eb == NONFINITE_EXP) ? __longlong_as_double(0x7FF8000000000000ll)
                                                                           : oz::i64_ldexp(acc[c], ea + eb - U, &pf);
            epi(b, row, col, v);
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

// ---------------------------------------------------------------- host side (ozr.cu)
// Fixed-point unit exponent for an inner dimension padded to Kp.
int unit_exponent(int Kp);
int64_t kp_of(int K);
// scratch for one product (digits of both operands, exponents, flag)
size_t scratch_bytes(int M, int N, int K, int batch);
// Splits op(A) (M x K: A[i][k], or A[k][i] with transA) and op(B) (its
// columns: B[k][j], or B[j][k] with transB_rows -- op(B)^T's rows stored
// contiguously) into the scratch and builds the TMA maps and kernel arguments;
// false if a map cannot be encoded.
bool prepare(int M, int N, int K, int batch, const double* A, int64_t lda, int64_t sa, bool transA,
             const double* B, int64_t ldb, int64_t sb, bool b_rows_are_k_major, void* scratch, int* err,
             CUtensorMap* ma, CUtensorMap* mb, RArgs* args, cudaStream_t st);

template <class Epi>
inline cudaError_t launch(const CUtensorMap& ma, const CUtensorMap& mb, const RArgs& a, Epi epi, cudaStream_t st) {
  set_smem_attr(ozr_gemm_kernel<Epi>, oz::SMEM_BYTES);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t tiles = (int64_t)((a.N + oz::BN - 1) / oz::BN) * ((a.M + tc::BM - 1) / tc::BM) * a.batch;
  if (tiles > INT32_MAX) return cudaErrorInvalidValue;
  const unsigned grid = (unsigned)(tiles < sms ? tiles : (sms > 0 ? sms : 1));
  FROB_LAUNCH("ozr_gemm<f64 digits>", st,
              ozr_gemm_kernel<Epi><<<grid, oz::THREADS, oz::SMEM_BYTES, st>>>(ma, mb, a, epi));
  return cudaGetLastError();
}

}  // namespace ozr
}  // namespace frob
