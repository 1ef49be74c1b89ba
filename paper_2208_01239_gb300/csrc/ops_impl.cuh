// Host-side drivers: the blocked factorisations and solves built from the
// kernels of dense_impl.cuh (with the one-CTA FP32 factorisations for
// n <= 512), the four inversion algorithms (Frobenius with LU, including the
// formula for invertible B and the automatic choice of the factored part;
// Frobenius with Cholesky; complex LU; complex Cholesky), the Frobenius
// linear solve, the complex-LU and 2n real augmented solves, and the
// adjoint.
#pragma once

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <string>
#include <type_traits>
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"
#include "dense_impl.cuh"
#include "ops.h"
#include "ozr.cuh"
#include "tc_gemm.cuh"

namespace frob {

// ------------------------------------------------------------------ small kernels
// SplitMix64 (Steele, Lea and Flood, OOPSLA 2014): state advanced by the
// golden-ratio increment, then the published finaliser.  mu for matrix b and
// draw `attempt` is the (b * 2^32 + attempt + 1)-th output for `seed`, mapped
// to the open interval (0, 1) as ((z >> 11) + 0.5) * 2^-53.
__host__ __device__ inline double draw_mu(uint64_t seed, int b, int attempt) {
  uint64_t ctr = ((uint64_t)(uint32_t)b << 32) + (uint64_t)(uint32_t)attempt + 1ull;
  uint64_t z = seed + ctr * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z = z ^ (z >> 31);
  return ((double)(z >> 11) + 0.5) * 0x1.0p-53;
}

__device__ __forceinline__ void init_info(frob_info* info, int b, double mu) {
  if (info == nullptr) return;
  frob_info f;
  f.status = FROB_OK;
  f.bad_index = 0;
  f.ns_iters = 0;
  f.fell_back = 0;
  f.mu = mu;
  f.residual = 0.0;
  info[b] = f;
}

// M = A + iB (interleaved) -> planes A (two copies: one is factorised, one
// becomes S) and B.  Almost sure variant (Sec. 4.2): A' = A - mu B,
// B' = mu A + B.  HPD variant (Sec. 4.3): only the lower triangle is read;
// A = Re (symmetric), B = Im (skew-symmetric, zero diagonal).  part = 1 (the
// formula for invertible B): the planes of -iM = B - iA, A' = B, B' = -A.
// LBc (FROB_PART_AUTO; p == NULL otherwise) receives a copy of B to factor.
template <typename R>
__global__ void split_kernel(int n, MatB<const typename cplx_of<R>::type> M, MatB<R> A1, MatB<R> A2, MatB<R> Bp,
                             frob_info* info, int hpd, int almost_sure, uint64_t seed, int attempt, int part = 0,
                             MatB<R> LBc = MatB<R>{nullptr, 0, 0}, int* partb = nullptr,
                             frob_info* infoB = nullptr) {
  const int b = blockIdx.z;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * n) return;
  const int i = (int)(e / n), j = (int)(e % n);
  const double mu = almost_sure ? draw_mu(seed, b, attempt) : 0.0;
  if (e == 0) {
    init_info(info, b, mu);
    if (infoB) init_info(infoB, b, 0.0);
    if (partb) partb[b] = part == 1 ? 1 : 0;
  }
  const auto* Mb = M.at(b);
  R a, bb;
  if (hpd) {
    if (i >= j) {
      auto v = Mb[(int64_t)i * M.ld + j];
      a = v.x;
      bb = (i == j) ? (R)0 : v.y;
    } else {
      auto v = Mb[(int64_t)j * M.ld + i];
      a = v.x;
      bb = -v.y;
    }
  } else {
    auto v = Mb[(int64_t)i * M.ld + j];
    a = v.x;
    bb = v.y;
    if (almost_sure) {
      R m = (R)mu;
      R a2 = a - m * bb;
      bb = m * a + bb;
      a = a2;
    } else if (part == 1) {
      const R a2 = bb;
      bb = -a;
      a = a2;
    }
    if (LBc.p) LBc.at(b)[(int64_t)i * LBc.ld + j] = bb;
  }
  A1.at(b)[(int64_t)i * A1.ld + j] = a;
  if (A2.p) A2.at(b)[(int64_t)i * A2.ld + j] = a;
  Bp.at(b)[(int64_t)i * Bp.ld + j] = bb;
}

// complex copy M -> W (baselines), with the info records initialised
template <typename C>
__global__ void copy_kernel(int n, MatB<const C> M, MatB<C> W, frob_info* info) {
  const int b = blockIdx.z;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * n) return;
  const int i = (int)(e / n), j = (int)(e % n);
  if (e == 0) init_info(info, b, 0.0);
  W.at(b)[(int64_t)i * W.ld + j] = M.at(b)[(int64_t)i * M.ld + j];
}

// rp = the permutation P of P A = L U as a row map: (P B)[r] = B[rp[r]].
// Built by applying the recorded exchanges in order to the identity.
static __global__ void rowperm_kernel(int n, const int* piv, int* rp, int use_smem) {
  const int b = blockIdx.x;
  extern __shared__ int sp[];
  int* p = use_smem ? sp : rp + (int64_t)b * n;
  const int* pv = piv + (int64_t)b * n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) p[i] = i;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 0; k < n; ++k) {
      int q = pv[k];
      int x = p[k];
      p[k] = p[q];
      p[q] = x;
    }
  }
  __syncthreads();
  if (use_smem)
    for (int i = threadIdx.x; i < n; i += blockDim.x) rp[(int64_t)b * n + i] = p[i];
}

// X[:, rp[c]] = Z[:, c]   (M^{-1} = (U^{-1} L^{-1}) P)
template <typename C>
__global__ void colperm_kernel(int n, MatB<const C> Z, MatB<C> X, const int* rp) {
  const int b = blockIdx.z;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * n) return;
  const int i = (int)(e / n), c = (int)(e % n);
  X.at(b)[(int64_t)i * X.ld + rp[(int64_t)b * n + c]] = Z.at(b)[(int64_t)i * Z.ld + c];
}

// ------------------------------------------------------------------ launch helpers
inline dim3 elem_grid(int n, int batch) {
  int64_t nn = (int64_t)n * n;
  return dim3((unsigned)((nn + 255) / 256), 1, (unsigned)batch);
}

constexpr size_t PANEL_SMEM_MAX = 200 * 1024;

template <typename T> inline int panel_width() { return PANEL_MAX; }

// real flops of one multiply-add of T
template <typename T> constexpr double madd_flops() { return is_cplx<T>::value ? 8.0 : 2.0; }

// The multiply-adds gemm_kernel computes for (M, N, K, tile_mode): its K
// range per 64 x 64 tile (see the tile modes), clipped to the matrix.
inline double gemm_madds(int M, int N, int K, int tile_mode) {
  if (tile_mode == 0) return (double)M * N * K;
  double total = 0.0;
  for (int i0 = 0; i0 < M; i0 += TB)
    for (int j0 = 0; j0 < N; j0 += TB) {
      if ((tile_mode & 1) && j0 > i0 + TB - 1) continue;
      int kbeg = (tile_mode & 2) ? std::max(i0, j0) : 0;
      if ((tile_mode & 4) && j0 > kbeg) kbeg = j0;
      const int kend = ((tile_mode & 8) && i0 + TB < K) ? i0 + TB : K;
      if (kend > kbeg) total += (double)std::min(TB, M - i0) * std::min(TB, N - j0) * (kend - kbeg);
    }
  return total;
}

// Tensor-core scratch of the FP32 drivers: while a TcScope is open on this
// host thread, FP32 products of at least TC3_MIN_MN x TC3_MIN_MN x TC3_MIN_K
// (full products, no tile skipping) run as split-TF32 tensor-core GEMMs
// (tc_gemm.cuh) in this scratch instead of on the CUDA cores.  The scratch is
// the caller's workspace; consecutive products reuse it in stream order.  Its
// first 256 bytes hold the kernels' timeout flag, reported into the info
// records when the scope closes.
struct TcScratch {
  unsigned char* p = nullptr;
  size_t bytes = 0;
  int* err = nullptr;
};
inline thread_local TcScratch t_tc;
// The same for the FP64 drivers: FP64 products of a digit shape
// (ozr::digit_shape: at least ozr::MIN_MNK in every dimension, or thinner
// ones large enough to beat the FP64 pipe) run as exact digit products on
// the BF16 tensor cores (ozr.cuh) while an OzScope is open.
inline thread_local TcScratch t_oz;
inline TcScratch& tc_slot() { return t_tc; }
inline TcScratch& oz_slot() { return t_oz; }


static __global__ void tc_err_report_kernel(const int* err, frob_info* info, int batch) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < batch && *err != 0) report(info, b, FROB_ERR_TIMEOUT, 0);
}

template <TcScratch& (*SLOT)()> class ScratchScope {
 public:
  ScratchScope(unsigned char* p, size_t bytes, frob_info* info, int batch, cudaStream_t st, bool on = true)
      : saved_(SLOT()), info_(info), batch_(batch), st_(st) {
    if (on && p && bytes > 256 && !t_tc_off) {
      SLOT() = TcScratch{p, bytes, reinterpret_cast<int*>(p)};
      cudaMemsetAsync(p, 0, 256, st);
    } else {
      SLOT() = TcScratch{};
    }
  }
  ~ScratchScope() {
    if (SLOT().err && info_)
      FROB_LAUNCH("tc_err_report", st_,
                  tc_err_report_kernel<<<(batch_ + 127) / 128, 128, 0, st_>>>(SLOT().err, info_, batch_));
    SLOT() = saved_;
  }
  ScratchScope(const ScratchScope&) = delete;
  ScratchScope& operator=(const ScratchScope&) = delete;

 private:
  TcScratch saved_;
  frob_info* info_;
  int batch_;
  cudaStream_t st_;
};
using TcScope = ScratchScope<tc_slot>;
using OzScope = ScratchScope<oz_slot>;

// bytes an FP64 driver reserves for its largest digit product (order n)
inline size_t oz_scratch_for(int n, int batch) {
  return n >= ozr::MIN_MNK ? ozr::scratch_bytes(n, n, n, batch) : 0;
}

template <typename T, int OPA, int OPB, class Epi>
inline void gemm_launch(int M, int N, int K, int batch, MatB<const T> A, MatB<const T> B, Epi epi, int tile_mode,
                        cudaStream_t st, int npairs = 1, int shift = 0) {
  if (M <= 0 || N <= 0) return;
  const double fl = madd_flops<T>() * gemm_madds(M, N, K, tile_mode) * batch * npairs;
  if constexpr (std::is_same<T, float>::value) {
    if (tile_mode == 0 && npairs == 1 && t_tc.p && M >= tc::TC3_MIN_MN && N >= tc::TC3_MIN_MN &&
        K >= tc::TC3_MIN_K && tc::tc3_scratch_bytes(M, N, K, batch) <= t_tc.bytes) {
      CUtensorMap ma, mb;
      // op(A) rows with k contiguous: A as stored (OP_N) or transposed; the B
      // operand holds op(B)^T, i.e. B transposed (OP_N) or as stored
      if (tc::tc3_prepare(M, N, K, batch, A.p, A.ld, A.bs, OPA != OP_N, B.p, B.ld, B.bs, OPB == OP_N, t_tc.p, &ma,
                          &mb, st)) {
        set_launch_flops(fl);
        tc::tc3_launch(ma, mb, M, N, K, batch, epi, t_tc.err, st);
        return;
      }
    }
  }
  if constexpr (std::is_same<T, double>::value) {
    if (tile_mode == 0 && npairs == 1 && t_oz.p && ozr::digit_shape(M, N, K) &&
        ozr::scratch_bytes(M, N, K, batch) <= t_oz.bytes) {
      CUtensorMap ma, mb;
      ozr::RArgs ra;
      // op(B)'s columns are the rows of B when OPB transposes it
      if (ozr::prepare(M, N, K, batch, A.p, A.ld, A.bs, OPA != OP_N, B.p, B.ld, B.bs, OPB != OP_N, t_oz.p, t_oz.err,
                       &ma, &mb, &ra, st)) {
        set_launch_flops(fl);
        ozr::launch(ma, mb, ra, epi, st);
        return;
      }
    }
  }
  set_launch_flops(fl);
  dim3 grid((N + TB - 1) / TB, (M + TB - 1) / TB, batch * npairs);
  static const std::string name = std::string("gemm<") + type_tag<T>() + ",op" + std::to_string(OPA) + ",op" +
                                  std::to_string(OPB) + "," + Epi::tag + ">";
  FROB_LAUNCH(name.c_str(), st,
              gemm_kernel<T, OPA, OPB, Epi><<<grid, NTH, 0, st>>>(M, N, K, A, B, epi, tile_mode, npairs, shift));
}

template <typename T>
inline EpiAxpby<T> axpby(MatB<T> D, T alpha, T beta, bool beta_zero) {
  return EpiAxpby<T>{D, MatB<const T>{D.p, D.ld, D.bs}, alpha, beta, beta_zero ? 1 : 0};
}

template <typename T, bool CONJ>
inline void mirror(int n, int batch, MatB<T> A, cudaStream_t st) {
  const dim3 g((unsigned)((n + 31) / 32), (unsigned)((n + 31) / 32), (unsigned)batch);
  FROB_LAUNCH(CONJ ? "mirror<herm>" : "mirror<sym>", st, mirror_kernel<T, CONJ><<<g, 256, 0, st>>>(n, A));
}

template <typename T, int OPT, bool LOWER, bool UNIT, bool RHS_I>
inline void trsm_smem_attr() {
  set_smem_attr(trsm_step_kernel<T, OPT, LOWER, UNIT, RHS_I>, (int)sizeof(SmemTrsm<T>));
}

// op(T) X = B over all block rows (in order of the substitution)
template <typename T, int OPT, bool LOWER, bool UNIT, bool RHS_I>
inline void trsm(int n, int nrhs, int batch, MatB<const T> Tm, MatB<const T> Bm, MatB<T> X, const int* rowperm,
                 cudaStream_t st) {
  trsm_smem_attr<T, OPT, LOWER, UNIT, RHS_I>();
  const int nblk = (n + TB - 1) / TB;
  dim3 grid((nrhs + TB - 1) / TB, 1, batch);
  for (int s = 0; s < nblk; ++s) {
    int kb = LOWER ? s : nblk - 1 - s;
    {
      // the product over the finished block rows and the substitution
      const int r0 = kb * TB, rows = std::min(TB, n - r0);
      const int kfin = LOWER ? r0 : n - r0 - rows;
      set_launch_flops(madd_flops<T>() * ((double)rows * nrhs * kfin + 0.5 * rows * rows * nrhs) * batch);
    }
    static const std::string name = std::string("trsm<") + type_tag<T>() + ",op" + std::to_string(OPT) +
                                    (LOWER ? ",lower" : ",upper") + (UNIT ? ",unit" : "") + (RHS_I ? ",rhs=I" : "") +
                                    ">";
    FROB_LAUNCH(name.c_str(), st, trsm_step_kernel<T, OPT, LOWER, UNIT, RHS_I><<<grid, NTH, sizeof(SmemTrsm<T>), st>>>(n, nrhs, kb, Tm, Bm, X,
                                                                                       rowperm));
  }
}

// X[r] = B[rp[r]] (rp NULL: a plain copy), n rows of ncols entries
template <typename T>
__global__ void rowgather_kernel(int n, int ncols, MatB<const T> B, MatB<T> X, const int* rp) {
  const int b = blockIdx.z;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * ncols) return;
  const int r = (int)(e / ncols), c = (int)(e % ncols);
  const int sr = rp ? rp[(int64_t)b * n + r] : r;
  X.at(b)[(int64_t)r * X.ld + c] = B.at(b)[(int64_t)sr * B.ld + c];
}

template <typename T>
__global__ void copy2d_kernel(int rows, int cols, MatB<const T> S, MatB<T> D) {
  const int b = blockIdx.z;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)rows * cols) return;
  const int r = (int)(e / cols), c = (int)(e % cols);
  D.at(b)[(int64_t)r * D.ld + c] = S.at(b)[(int64_t)r * S.ld + c];
}

template <typename T, bool UNIT>
inline void trtri(int n, int batch, MatB<const T> Lm, MatB<T> X, MatB<T> Tmp, cudaStream_t st);

// Explicit inverses of the diagonal blocks of a recursive triangular solve
// (all blocks of at most TRSM_REC_BASE rows, padded to TRSM_REC_BASE with the
// identity): inverse q of matrix b at G + (q batch + b) RB^2, row-major with
// ld RB.  `off[q]` is block q's first row.
constexpr int REC_INV_MAX = 64;
struct RecInv {
  const double* G;
  int nb;
  int off[REC_INV_MAX];
};

struct RecBlocks {
  int nb;
  int off[REC_INV_MAX];
  int sz[REC_INV_MAX];
};

// Padded copies of the diagonal blocks: D[q][b] = [B 0; 0 I] with B the
// block of T (transposed when `trans`), grid (RB^2 / 256, nb, batch).
template <int RB>
__global__ void gather_diag_kernel(RecBlocks blk, int trans, MatB<const double> Tm, double* D, int batch) {
  const int q = blockIdx.y, b = blockIdx.z;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= RB * RB) return;
  const int r = e / RB, c = e % RB;
  const int o = blk.off[q], sz = blk.sz[q];
  double v = r == c ? 1.0 : 0.0;
  if (r < sz && c < sz) {
    const double* Tb = Tm.at(b);
    v = trans ? Tb[(int64_t)(o + c) * Tm.ld + (o + r)] : Tb[(int64_t)(o + r) * Tm.ld + (o + c)];
  }
  D[((int64_t)q * batch + b) * RB * RB + e] = v;
}

// Recursive triangular solve op(T) X = X in place (Elmroth, Gustavson,
// Jonsson and Kagstrom's recursive blocking): split at h, solve the first
// half, remove its contribution from the second half with one product,
// solve the second half.  Almost all of the n^2 nrhs flops land in large
// products that spread over the whole GPU, where the block-row steps of
// trsm() have only ceil(nrhs / 64) x batch CTAs each; blocks of at most
// TRSM_REC_BASE rows are one digit product with their explicit inverse
// (computed for all blocks at once by rec_inverses) when the FP64 digit
// products are on, else trsm().
constexpr int TRSM_REC_BASE = 256;
constexpr int TRSM_REC_MIN = 1024;   // smallest order that takes the recursive form
constexpr int TRSM_REC_TILES = 512;  // ... when ceil(nrhs / 64) x batch is at most this

template <typename T, int OPT, bool LOWER, bool UNIT>
inline void trsm_rec(int n, int nrhs, int batch, MatB<const T> Tm, MatB<T> X, cudaStream_t st,
                     const RecInv* inv = nullptr, int r0 = 0) {
  if (n <= TRSM_REC_BASE) {
    if constexpr (std::is_same<T, double>::value) {
      if (inv) {
        // X = G X with G = op(T)^{-1} (LOWER) or its transpose (upper op(T)),
        // formed out of place behind the inverses, then copied back
        int q = 0;
        while (q < inv->nb && inv->off[q] != r0) ++q;
        const int64_t rr = (int64_t)TRSM_REC_BASE * TRSM_REC_BASE;
        MatB<const double> Gq{inv->G + (int64_t)q * batch * rr, TRSM_REC_BASE, rr};
        MatB<double> Y{const_cast<double*>(inv->G) + (int64_t)inv->nb * batch * rr, nrhs, (int64_t)n * nrhs};
        MatB<const double> Xc{X.p, X.ld, X.bs};
        if (LOWER)
          gemm_launch<double, OP_N, OP_N>(n, nrhs, n, batch, Gq, Xc, axpby<double>(Y, 1.0, 0.0, true), 0, st);
        else
          gemm_launch<double, OP_T, OP_N>(n, nrhs, n, batch, Gq, Xc, axpby<double>(Y, 1.0, 0.0, true), 0, st);
        const int64_t ne = (int64_t)n * nrhs;
        FROB_LAUNCH("copy2d", st,
                    copy2d_kernel<double><<<dim3((unsigned)((ne + 255) / 256), 1, (unsigned)batch), 256, 0, st>>>(
                        n, nrhs, MatB<const double>{Y.p, Y.ld, Y.bs}, X));
        return;
      }
    }
    trsm<T, OPT, LOWER, UNIT, false>(n, nrhs, batch, Tm, MatB<const T>{X.p, X.ld, X.bs}, X, nullptr, st);
    return;
  }
  const int h = ((n / 2 + TB - 1) / TB) * TB;
  // block (i0, j0) of op(T) as a GEMM operand of mode OPT
  auto blk = [&](int i0, int j0) { return OPT == OP_N ? Tm.sub(i0, j0) : Tm.sub(j0, i0); };
  auto cst = [](MatB<T> m) { return MatB<const T>{m.p, m.ld, m.bs}; };
  if (LOWER) {
    trsm_rec<T, OPT, LOWER, UNIT>(h, nrhs, batch, Tm, X, st, inv, r0);
    gemm_launch<T, OPT, OP_N>(n - h, nrhs, h, batch, blk(h, 0), cst(X), axpby<T>(X.sub(h, 0), neg_(one_v<T>()),
                                                                                 one_v<T>(), false), 0, st);
    trsm_rec<T, OPT, LOWER, UNIT>(n - h, nrhs, batch, Tm.sub(h, h), X.sub(h, 0), st, inv, r0 + h);
  } else {
    trsm_rec<T, OPT, LOWER, UNIT>(n - h, nrhs, batch, Tm.sub(h, h), X.sub(h, 0), st, inv, r0 + h);
    gemm_launch<T, OPT, OP_N>(h, nrhs, n - h, batch, blk(0, h), cst(X.sub(h, 0)),
                              axpby<T>(X, neg_(one_v<T>()), one_v<T>(), false), 0, st);
    trsm_rec<T, OPT, LOWER, UNIT>(h, nrhs, batch, Tm, X, st, inv, r0);
  }
}

// The diagonal blocks trsm_rec reaches for order n (first row, rows).
inline void rec_blocks(int n, int r0, RecBlocks& out) {
  if (n <= TRSM_REC_BASE) {
    if (out.nb < REC_INV_MAX) {
      out.off[out.nb] = r0;
      out.sz[out.nb] = n;
    }
    ++out.nb;
    return;
  }
  const int h = ((n / 2 + TB - 1) / TB) * TB;
  rec_blocks(h, r0, out);
  rec_blocks(n - h, r0 + h, out);
}

// With the FP64 digit products on: the inverses of all diagonal blocks of
// the recursion in one batched triangular inverse, at the end of the digit
// scratch (behind the largest product's digits), so that each block of the
// solve is one digit product.  False (nothing done) when the blocks are too
// many or the scratch is short.
template <typename T, int OPT, bool LOWER, bool UNIT>
inline bool rec_inverses(int n, int nrhs, int batch, MatB<const T> Tm, RecInv& inv, cudaStream_t st) {
  if constexpr (!std::is_same<T, double>::value) {
    return false;
  } else {
    if (!t_oz.p || nrhs < ozr::MIN_MN_THIN) return false;
    RecBlocks blk{};
    rec_blocks(n, 0, blk);
    if (blk.nb > REC_INV_MAX) return false;
    for (int q = 0; q < blk.nb; ++q)
      if (!ozr::digit_shape(blk.sz[q], nrhs, blk.sz[q])) return false;
    constexpr int RB = TRSM_REC_BASE;
    const size_t plane = (size_t)blk.nb * batch * RB * RB * sizeof(double);
    const size_t ybytes = (size_t)RB * nrhs * batch * sizeof(double);
    const size_t tail = (3 * plane + ybytes + 511) & ~(size_t)255;
    const int h = ((n / 2 + TB - 1) / TB) * TB;
    const size_t head = std::max(ozr::scratch_bytes(n - h, nrhs, h, batch), ozr::scratch_bytes(RB, nrhs, RB, batch));
    if (head + 256 + tail > t_oz.bytes) return false;
    // [G: inverses][Y: products of one block][D: padded blocks][J: join scratch]
    double* G = reinterpret_cast<double*>(t_oz.p + ((t_oz.bytes - tail) & ~(size_t)255));
    double* D = G + plane / sizeof(double) + ybytes / sizeof(double);
    double* J = D + plane / sizeof(double);
    constexpr bool transpose = (LOWER && OPT != OP_N) || (!LOWER && OPT == OP_N);
    FROB_LAUNCH("gather_diag", st,
                (gather_diag_kernel<RB><<<dim3(RB * RB / 256, (unsigned)blk.nb, (unsigned)batch), 256, 0, st>>>(
                    blk, transpose ? 1 : 0, Tm, D, batch)));
    const int64_t rr = (int64_t)RB * RB;
    trtri<double, UNIT>(RB, blk.nb * batch, MatB<const double>{D, RB, rr}, MatB<double>{G, RB, rr},
                        MatB<double>{J, RB, rr}, st);
    inv.G = G;
    inv.nb = blk.nb;
    for (int q = 0; q < blk.nb; ++q) inv.off[q] = blk.off[q];
    return true;
  }
}

// op(T) X = P B (rowperm) or = B: the recursive form for large orders with
// few right-hand-side tiles, else the block-row steps.  X may alias B when
// rowperm is NULL.
template <typename T, int OPT, bool LOWER, bool UNIT>
inline void trsm_any(int n, int nrhs, int batch, MatB<const T> Tm, MatB<const T> Bm, MatB<T> X, const int* rowperm,
                     cudaStream_t st) {
  const int64_t tiles = (int64_t)((nrhs + TB - 1) / TB) * batch;
  if (n < TRSM_REC_MIN || tiles > TRSM_REC_TILES) {
    trsm<T, OPT, LOWER, UNIT, false>(n, nrhs, batch, Tm, Bm, X, rowperm, st);
    return;
  }
  if (rowperm || Bm.p != X.p) {
    const int64_t ne = (int64_t)n * nrhs;
    FROB_LAUNCH("rowgather", st,
                rowgather_kernel<T><<<dim3((unsigned)((ne + 255) / 256), 1, (unsigned)batch), 256, 0, st>>>(
                    n, nrhs, Bm, X, rowperm));
  }
  RecInv inv;
  const bool have_inv = rec_inverses<T, OPT, LOWER, UNIT>(n, nrhs, batch, Tm, inv, st);
  trsm_rec<T, OPT, LOWER, UNIT>(n, nrhs, batch, Tm, X, st, have_inv ? &inv : nullptr, 0);
}

// X = L^{-1} for lower triangular L (unit diagonal if UNIT), recursively:
// the 64 x 64 diagonal blocks are inverted in one launch, then neighbouring
// blocks of size s = 64, 128, ... are joined,
//   [A 0; B C]^{-1} = [A^{-1} 0; -C^{-1} B A^{-1}  C^{-1}],
// by two batched products per pair that skip the zero triangles (B A^{-1}
// from k = j0, C^{-1} (B A^{-1}) up to k = i0 + 64).  Tmp: n x n scratch of
// the same layout (its lower blocks are overwritten).
template <typename T, bool UNIT>
inline void trtri(int n, int batch, MatB<const T> Lm, MatB<T> X, MatB<T> Tmp, cudaStream_t st) {
  set_smem_attr(trtri_diag_kernel<T, UNIT>, (int)sizeof(SmemTrsm<T>));
  static const std::string name = std::string("trtri_diag<") + type_tag<T>() + ">";
  const int nblk = (n + TB - 1) / TB;
  FROB_LAUNCH(name.c_str(), st,
              trtri_diag_kernel<T, UNIT><<<dim3(nblk, 1, batch), NTH, sizeof(SmemTrsm<T>), st>>>(n, Lm, X));
  auto cst = [](MatB<T> m) { return MatB<const T>{m.p, m.ld, m.bs}; };
  // the pairs of one level with full-size C in one launch (pair p is pair 0
  // moved 2 s p down the diagonal), a short last pair on its own
  auto join = [&](int r, int s, int sc, int npairs) {
    if constexpr (std::is_same<T, double>::value) {
      // with the FP64 digit products on: each pair as two full products on
      // the tensor cores (the zero triangles included), one pair per launch
      if (t_oz.p && s >= ozr::MIN_MNK && sc >= ozr::MIN_MNK) {
        if (batch == 1 && npairs > 1) {
          // the pairs of this level are equal blocks spaced 2 s down the
          // diagonal: one batched product each, batch stride 2 s (ld + 1)
          auto step = [&](auto m) {
            auto v = m;
            v.bs = 2 * (int64_t)s * (m.ld + 1);
            return v;
          };
          MatB<T> Tq = step(Tmp.sub(r + s, r));
          gemm_launch<T, OP_N, OP_N>(sc, s, s, npairs, step(Lm.sub(r + s, r)), step(cst(X.sub(r, r))),
                                     axpby<T>(Tq, one_v<T>(), zero_v<T>(), true), 0, st);     // B A^{-1}
          gemm_launch<T, OP_N, OP_N>(sc, s, sc, npairs, step(cst(X.sub(r + s, r + s))), cst(Tq),
                                     axpby<T>(step(X.sub(r + s, r)), neg_(one_v<T>()), zero_v<T>(), true), 0,
                                     st);                                                       // -C^{-1} (B A^{-1})
          return;
        }
        for (int q = 0; q < npairs; ++q) {
          const int rq = r + 2 * s * q;
          MatB<T> Tq = Tmp.sub(rq + s, rq);
          gemm_launch<T, OP_N, OP_N>(sc, s, s, batch, Lm.sub(rq + s, rq), cst(X.sub(rq, rq)),
                                     axpby<T>(Tq, one_v<T>(), zero_v<T>(), true), 0, st);       // B A^{-1}
          gemm_launch<T, OP_N, OP_N>(sc, s, sc, batch, cst(X.sub(rq + s, rq + s)), cst(Tq),
                                     axpby<T>(X.sub(rq + s, rq), neg_(one_v<T>()), zero_v<T>(), true), 0,
                                     st);                                                         // -C^{-1} (B A^{-1})
        }
        return;
      }
    }
    MatB<const T> B = Lm.sub(r + s, r);
    MatB<T> Tp = Tmp.sub(r + s, r);
    gemm_launch<T, OP_N, OP_N>(sc, s, s, batch, B, cst(X.sub(r, r)), axpby<T>(Tp, one_v<T>(), zero_v<T>(), true), 4,
                               st, npairs, 2 * s);                                        // B A^{-1}
    gemm_launch<T, OP_N, OP_N>(sc, s, sc, batch, cst(X.sub(r + s, r + s)), cst(Tp),
                               axpby<T>(X.sub(r + s, r), neg_(one_v<T>()), zero_v<T>(), true), 8, st, npairs,
                               2 * s);                                                    // -C^{-1} (B A^{-1})
  };
  for (int s = TB; s < n; s *= 2) {
    const int full = n / (2 * s);              // pairs [2 s p, 2 s p + 2 s) inside the matrix
    if (full > 0) join(0, s, s, full);
    const int r = full * 2 * s;                // a last pair with a short C
    if (r + s < n) join(r, s, n - r - s, 1);
  }
}

template <typename T> inline void panel_smem_attr() {
  set_smem_attr(getrf_panel_kernel<T>, (int)PANEL_SMEM_MAX);
  set_smem_attr(laswp_trsm_kernel<T>, (int)laswp_trsm_smem<T>());
}

template <typename T> inline const char* getrf_panel_name() {
  static const std::string s = std::string("getrf_panel<") + type_tag<T>() + ">";
  return s.c_str();
}
template <typename T> inline const char* laswp_name() {
  static const std::string s = std::string("laswp_trsm<") + type_tag<T>() + ">";
  return s.c_str();
}
// Scratch of the multi-CTA panel factorization (getrf_panel_mc_kernel), carved
// from the caller's workspace by the routines that factor with getrf: used for
// matrices of order above PANEL_THREADS in calls of at most MC_BATCH_MAX
// matrices, 0 bytes otherwise.
template <typename T> inline size_t mc_scratch_bytes(int n, int batch) {
  return (n > PANEL_THREADS && batch <= MC_BATCH_MAX) ? mc_scratch_per_matrix<T>() * (size_t)batch : 0;
}

inline int num_sms() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

template <typename T> inline const char* getrf_cl_name() {
  static const std::string s = std::string("getrf_panel_cl<") + type_tag<T>() + ">";
  return s.c_str();
}

// Whether a cluster of G CTAs with `smem` bytes of dynamic shared memory each
// can be scheduled for getrf_panel_cl_kernel<T> (asked once per shape and
// device; cluster sizes above 8 need the non-portable opt-in).
template <typename T> inline bool cluster_panel_ok(int G, size_t smem) {
  static std::mutex mu;
  static std::map<std::tuple<int, int, size_t>, bool> seen;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  auto key = std::make_tuple(dev, G, smem);
  auto it = seen.find(key);
  if (it != seen.end()) return it->second;
  // the largest size any shape uses, so that a later launch of a cached
  // shape is never refused for a smaller limit set in between
  bool ok = cudaFuncSetAttribute(getrf_panel_cl_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)MC_SMEM_MAX) == cudaSuccess;
  if (ok && G > 8)
    ok = cudaFuncSetAttribute(getrf_panel_cl_kernel<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
         cudaSuccess;
  if (ok) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)G, 1, 1);
    cfg.blockDim = dim3(MC_THREADS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)G;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    ok = cudaOccupancyMaxActiveClusters(&clusters, getrf_panel_cl_kernel<T>, &cfg) == cudaSuccess && clusters >= 1;
  }
  cudaGetLastError();  // a refused attribute or query leaves no error behind
  seen[key] = ok;
  return ok;
}

template <typename T> inline const char* getrf_mc_name() {
  static const std::string s = std::string("getrf_panel_mc<") + type_tag<T>() + ">";
  return s.c_str();
}

// The second stream of the LU's look-ahead (highest priority, so that a
// panel waiting beside a product gets its SMs first) and its two events, per
// host thread and created on first use; nullptr when the stream cannot be
// made, the device changed, or `st` is being captured into a graph.
struct PanelStream {
  cudaStream_t s = nullptr;
  cudaEvent_t ready = nullptr;  // the next panel's columns are updated
  cudaEvent_t done = nullptr;   // the next panel is factored
  int dev = -1;
  bool failed = false;
  ~PanelStream() {
    if (ready) cudaEventDestroy(ready);
    if (done) cudaEventDestroy(done);
    if (s) cudaStreamDestroy(s);
  }
};
inline thread_local PanelStream t_panel_stream;

inline PanelStream* panel_stream(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return nullptr;
  }
  PanelStream& p = t_panel_stream;
  int dev = 0;
  cudaGetDevice(&dev);
  if (p.failed || (p.s && p.dev != dev)) return nullptr;
  if (!p.s) {
    int least = 0, greatest = 0;
    cudaDeviceGetStreamPriorityRange(&least, &greatest);
    if (cudaStreamCreateWithPriority(&p.s, cudaStreamNonBlocking, greatest) != cudaSuccess ||
        cudaEventCreateWithFlags(&p.ready, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p.done, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      p.failed = true;
      return nullptr;
    }
    p.dev = dev;
  }
  return &p;
}

// Panels [kbeg, kend) of a right-looking LU with partial pivoting, in place:
// each 32-wide panel is factored (by cooperating CTAs when `mc`), its row
// exchanges are applied to every other column of the matrix, and U12 and the
// trailing update reach the columns up to u_end (n: the whole matrix; a
// recursive LU's block passes its right edge).
//   Look-ahead (when the next panel takes the multi-CTA forms): the trailing
// update first reaches the next panel's columns only; that panel is then
// factored on the second stream while the rest of the update runs on `st`
// with the panel's CL_MAX SMs left free by the persistent product kernels,
// and the next exchange-and-U12 step waits for both (single matrices only).  Neither waits on the other, so a panel that finds no room runs
// after the product.  The two touch disjoint columns; the panel's row exchanges reach
// the other columns only in that later step.
template <typename T>
inline void getrf_panels(int n, int batch, MatB<T> A, int* piv, frob_info* info, int info_off, cudaStream_t st,
                         unsigned char* mcs, bool mc, int gcap, int kbeg, int kend, int u_end) {
  const int nb = panel_width<T>();
  auto panel = [&](int k0, int kb, cudaStream_t ps) {
    const int m = n - k0;
    const size_t bytes = (size_t)m * (kb + 1) * sizeof(T);
    const int staged = bytes <= PANEL_SMEM_MAX;
    int R = 0, G = 0;
    // a thread-block cluster holding the whole panel (exchange through
    // distributed shared memory), when its rows fit 16 CTAs' shared memory
    int Rc = 0, Gc = 0;
    if (mc && m > PANEL_THREADS && batch * CL_MAX <= num_sms()) {
      Gc = std::min(CL_MAX, (m + MC_MIN_ROWS - 1) / MC_MIN_ROWS);
      Rc = (m + Gc - 1) / Gc;
      const size_t smem_c = (size_t)Rc * (PANEL_MAX + 1) * sizeof(T);
      if (smem_c > MC_SMEM_MAX || !cluster_panel_ok<T>(Gc, smem_c)) Gc = 0;
    }
    if (Gc == 0 && mc && m > PANEL_THREADS) {
      R = std::max(MC_MIN_ROWS, (m + gcap - 1) / gcap);
      G = (m + R - 1) / R;
      if (mc_smem<T>(R) > MC_SMEM_MAX) G = 0;
    }
    if (Gc > 0) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3((unsigned)Gc, (unsigned)batch, 1);
      cfg.blockDim = dim3(MC_THREADS, 1, 1);
      cfg.dynamicSmemBytes = (size_t)Rc * (PANEL_MAX + 1) * sizeof(T);
      cfg.stream = ps;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = (unsigned)Gc;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      cudaError_t le = cudaSuccess;
      FROB_LAUNCH(getrf_cl_name<T>(), ps,
                  le = cudaLaunchKernelEx(&cfg, getrf_panel_cl_kernel<T>, n, k0, kb, A, piv, info, info_off, Rc));
      if (le != cudaSuccess) {
        // refused (e.g. no room for the cluster): the cooperative-grid panel
        cudaGetLastError();
        R = std::max(MC_MIN_ROWS, (m + gcap - 1) / gcap);
        G = (m + R - 1) / R;
        if (mc_smem<T>(R) > MC_SMEM_MAX) G = 0;
        Gc = 0;
      }
    }
    if (Gc > 0) {
      // launched on the cluster
    } else if (G > 0) {
      const size_t smem = mc_smem<T>(R);
      int64_t bs = (int64_t)mc_scratch_per_matrix<T>();
      long long limit = 1ll << 31;  // about a second of SM clock
      int k0v = k0, kbv = kb;
      void* args[] = {(void*)&n, (void*)&k0v, (void*)&kbv, (void*)&A, (void*)&piv, (void*)&info, (void*)&info_off,
                      (void*)&mcs, (void*)&bs, (void*)&R, (void*)&limit};
      FROB_LAUNCH(getrf_mc_name<T>(), ps,
                  cudaLaunchCooperativeKernel((const void*)getrf_panel_mc_kernel<T>, dim3((unsigned)G, (unsigned)batch),
                                              dim3(MC_THREADS), args, smem, ps));
    } else if (m <= PANEL_THREADS && sizeof(T) <= 8) {
      FROB_LAUNCH(getrf_panel_name<T>(), ps,
                  getrf_panel_reg_kernel<T><<<batch, PANEL_THREADS, 0, ps>>>(n, k0, kb, A, piv, info, info_off));
    } else {
      FROB_LAUNCH(getrf_panel_name<T>(), ps,
                  getrf_panel_kernel<T><<<batch, PANEL_THREADS, staged ? bytes : 0, ps>>>(n, k0, kb, A, piv, info,
                                                                                         info_off, staged));
    }
  };
  // look-ahead only for a single matrix, whose multi-CTA panels leave most of
  // the GPU idle (a batch's panels already spread over the SMs), and while the
  // stream is free to fork
  PanelStream* la = (mc && batch == 1 && kend - kbeg > nb) ? panel_stream(st) : nullptr;
  bool pending = false;  // panel k0 was factored on la->s
  for (int k0 = kbeg; k0 < kend; k0 += nb) {
    const int kb = std::min(nb, kend - k0);
    if (pending) {
      cudaStreamWaitEvent(st, la->done, 0);
      pending = false;
    } else {
      panel(k0, kb, st);
    }
    FROB_LAUNCH(laswp_name<T>(), st,
                laswp_trsm_kernel<T><<<dim3((n + TB - 1) / TB, 1, batch), NTH, laswp_trsm_smem<T>(), st>>>(n, k0, kb, A,
                                                                                                       piv, u_end));
    const int r = k0 + kb;
    if (r < u_end) {
      MatB<const T> L21{A.p + (int64_t)r * A.ld + k0, A.ld, A.bs};
      MatB<const T> U12{A.p + (int64_t)k0 * A.ld + r, A.ld, A.bs};
      MatB<T> A22 = A.sub(r, r);
      const int nkb = std::min(nb, kend - r);  // the next panel's width (when r < kend)
      if (la && r < kend && n - r > PANEL_THREADS && u_end - r > nkb) {
        // the next panel's columns (nkb, kb <= PANEL_MAX)
        static_assert(PANEL_MAX <= 32, "update_narrow_kernel covers 32 columns and 32 of K");
        static const std::string nname = std::string("update_narrow<") + type_tag<T>() + ">";
        set_launch_flops(madd_flops<T>() * gemm_madds(n - r, nkb, kb, 0) * batch);
        FROB_LAUNCH(nname.c_str(), st,
                    update_narrow_kernel<T><<<dim3((unsigned)((n - r + 31) / 32), 1, (unsigned)batch), 256, 0, st>>>(
                        n - r, nkb, kb, L21, U12, A22));
        cudaEventRecord(la->ready, st);
        cudaStreamWaitEvent(la->s, la->ready, 0);
        panel(r, nkb, la->s);
        cudaEventRecord(la->done, la->s);
        pending = true;
        SmReserve keep(CL_MAX);
        gemm_launch<T, OP_N, OP_N>(n - r, u_end - r - nkb, kb, batch, L21,
                                   MatB<const T>{U12.p + nkb, U12.ld, U12.bs},
                                   axpby<T>(A22.sub(0, nkb), neg_(one_v<T>()), one_v<T>(), false), 0, st);
      } else {
        gemm_launch<T, OP_N, OP_N>(n - r, u_end - r, kb, batch, L21, U12,
                                   axpby<T>(A22, neg_(one_v<T>()), one_v<T>(), false), 0, st);
      }
    }
  }
}

// Recursive LU of the column block [c0, c0 + w) (rows c0 .. n - 1; Toledo's
// recursion, as LAPACK's getrf2): factor the left half, U12 = L11^{-1} A12,
// A22 -= L21 U12 (one product with K = the left half's width), factor the
// right half.  The row exchanges are applied to every column as each panel
// is factored, so the halves need no separate exchange passes.  Blocks of at
// most `nb` columns take the panel loop.
//   With an n x n scratch plane `tmp`: U12 = (L11^{-1}) A12, the inverse by the
//   recursive triangular inverse into tmp (its joins are large products),
//   the product into tmp and copied back; every product of the recursion then
//   has K >= 256 and nb = GETRF_REC_NB_INV (512) keeps the panel loop's
//   rank-32 updates on the CUDA cores small.
//   Without it: U12 by a triangular solve, which for narrow blocks is a few
//   CTAs of FP64-pipe work per launch, so nb = GETRF_REC_NB (2048) keeps every
//   solve at 1024 rows or more (recursive); measured with 512-wide blocks:
//   112 ms of a 521 ms inversion of order 8192 in those solves.
// The left half has round_down(w / 2, 256) columns (at least 256), so the
// inverse (w1 x w1) and its join scratch (w1 x w1, beside it) fit in tmp.
constexpr int GETRF_REC_NB = 2048;
constexpr int GETRF_REC_NB_INV = 512;

template <typename T>
inline void getrf_rec(int n, int batch, MatB<T> A, int* piv, frob_info* info, int info_off, cudaStream_t st,
                      unsigned char* mcs, bool mc, int gcap, int c0, int w, MatB<T> tmp, int nb) {
  if (w <= nb) {
    getrf_panels<T>(n, batch, A, piv, info, info_off, st, mcs, mc, gcap, c0, c0 + w, c0 + w);
    return;
  }
  const int w1 = tmp.p ? std::max(256, (w / 2) / 256 * 256) : ((w / 2 + 255) / 256) * 256;
  getrf_rec<T>(n, batch, A, piv, info, info_off, st, mcs, mc, gcap, c0, w1, tmp, nb);
  auto cst = [](MatB<T> m) { return MatB<const T>{m.p, m.ld, m.bs}; };
  MatB<T> A12 = A.sub(c0, c0 + w1);
  if (tmp.p) {
    MatB<T> Li = tmp, J = tmp.sub(0, w1), D = tmp.sub(0, w1);
    trtri<T, true>(w1, batch, cst(A.sub(c0, c0)), Li, J, st);                          // L11^{-1}
    gemm_launch<T, OP_N, OP_N>(w1, w - w1, w1, batch, cst(Li), cst(A12), axpby<T>(D, one_v<T>(), zero_v<T>(), true),
                               0, st);                                                  // U12 = L11^{-1} A12
    const int64_t ne = (int64_t)w1 * (w - w1);
    FROB_LAUNCH("copy2d", st,
                copy2d_kernel<T><<<dim3((unsigned)((ne + 255) / 256), 1, (unsigned)batch), 256, 0, st>>>(
                    w1, w - w1, cst(D), A12));
  } else {
    trsm_any<T, OP_N, true, true>(w1, w - w1, batch, cst(A.sub(c0, c0)), cst(A12), A12, nullptr, st);
  }
  gemm_launch<T, OP_N, OP_N>(n - c0 - w1, w - w1, w1, batch, cst(A.sub(c0 + w1, c0)), cst(A12),
                             axpby<T>(A.sub(c0 + w1, c0 + w1), neg_(one_v<T>()), one_v<T>(), false), 0, st);
  getrf_rec<T>(n, batch, A, piv, info, info_off, st, mcs, mc, gcap, c0 + w1, w - w1, tmp, nb);
}

// LU with partial pivoting (P A = L U, in place).  Panels of more than
// PANEL_THREADS rows are factored by several cooperating CTAs per matrix when
// `mcs` (mc_scratch_bytes of scratch) is given: one cooperative launch of
// G x batch CTAs, G x batch at most one per SM, so a single large matrix keeps
// the panel off its critical path's single SM.  While tensor-core products are
// on (FP64 digit products or FP32 split TF32), orders above the recursion's
// block width take the recursive form (with `tmp`, an n x n scratch plane:
// U12 by triangular inverses, 512-wide blocks); the right-looking panel loop
// otherwise.
template <typename T>
inline void getrf(int n, int batch, MatB<T> A, int* piv, frob_info* info, int info_off, cudaStream_t st,
                  unsigned char* mcs = nullptr, MatB<T> tmp = MatB<T>{nullptr, 0, 0}) {
  if constexpr (std::is_same<T, float>::value) {
    if (n <= SLU_MAX) {
      // one CTA per matrix (panels, U12 solves and trailing updates between CTA barriers)
      set_smem_attr(getrf_small_kernel<float>, SLU_SMEM);
      FROB_LAUNCH("getrf_small<f32>", st,
                  getrf_small_kernel<float><<<batch, SLU_THREADS, SLU_SMEM, st>>>(n, A, piv, info, info_off));
      return;
    }
  }
  panel_smem_attr<T>();
  const bool mc = mcs != nullptr && mc_scratch_bytes<T>(n, batch) > 0;
  const int gcap = mc ? std::max(1, std::min(MC_GMAX, num_sms() / batch)) : 0;
  if (mc) {
    set_smem_attr(getrf_panel_mc_kernel<T>, (int)MC_SMEM_MAX);
    cudaMemsetAsync(mcs, 0, mc_scratch_bytes<T>(n, batch), st);  // barrier counters and flags
  }
  bool rec = false;
  if constexpr (std::is_same<T, double>::value) rec = t_oz.p != nullptr;
  if constexpr (std::is_same<T, float>::value) rec = t_tc.p != nullptr;
  const int nb = tmp.p ? GETRF_REC_NB_INV : GETRF_REC_NB;
  if (rec && n > nb)
    getrf_rec<T>(n, batch, A, piv, info, info_off, st, mcs, mc, gcap, 0, n, tmp, nb);
  else
    getrf_panels<T>(n, batch, A, piv, info, info_off, st, mcs, mc, gcap, 0, n, n);
}

// Blocked right-looking Cholesky (A = L L^H, lower triangle, in place): per
// 32-wide panel, one launch for the diagonal block and the rows below it (the
// block factored by one warp of every CTA, the rows one thread each), then
// the trailing update of the lower tiles.  Real FP32 matrices with n <= 512
// take one launch instead, one CTA per matrix (potrf_small_kernel).
template <typename T> inline const char* potrf_panel_name() {
  static const std::string s = std::string("potrf_panel<") + type_tag<T>() + ">";
  return s.c_str();
}

template <typename T>
inline void potrf(int n, int batch, MatB<T> A, frob_info* info, int info_off, cudaStream_t st) {
  if constexpr (std::is_same<T, float>::value) {
    if (n <= SCHOL_MAX) {
      // one CTA per matrix (its panels, row solves and trailing updates between CTA barriers)
      set_smem_attr(potrf_small_kernel<float>, SCHOL_SMEM);
      FROB_LAUNCH("potrf_small<f32>", st,
                  potrf_small_kernel<float><<<batch, SCHOL_THREADS, SCHOL_SMEM, st>>>(n, A, info, info_off));
      return;
    }
  }
  const int nb = panel_width<T>();
  for (int k0 = 0; k0 < n; k0 += nb) {
    const int kb = std::min(nb, n - k0);
    const int r = k0 + kb;
    const int rb = r < n ? (n - r + 127) / 128 : 1;
    FROB_LAUNCH(potrf_panel_name<T>(), st,
                potrf_panel_kernel<T><<<dim3(rb, batch), 128, 0, st>>>(n, k0, kb, A, info, info_off));
    if (r < n) {
      MatB<const T> L21{A.p + (int64_t)r * A.ld + k0, A.ld, A.bs};
      MatB<T> A22 = A.sub(r, r);
      gemm_launch<T, OP_N, OP_C>(n - r, n - r, kb, batch, L21, L21, axpby<T>(A22, neg_(one_v<T>()), one_v<T>(), false),
                                 1, st);
    }
  }
}

inline void rowperm(int n, int batch, const int* piv, int* rp, cudaStream_t st) {
  const int use_smem = (size_t)n * sizeof(int) <= 48 * 1024;
  FROB_LAUNCH("rowperm", st, rowperm_kernel<<<batch, 256, use_smem ? n * sizeof(int) : 0, st>>>(n, piv, rp, use_smem));
}

// ------------------------------------------------------------------ workspace
inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Carve {
  unsigned char* base;
  size_t off = 0;
  template <typename T> T* take(size_t count) {
    T* p = reinterpret_cast<T*>(base ? base + off : nullptr);
    off += align256(count * sizeof(T));
    return p;
  }
};

template <typename T> inline MatB<T> plane(Carve& c, int n, int batch) {
  T* p = c.take<T>((size_t)n * n * batch);
  return MatB<T>{p, n, (int64_t)n * n};
}

// ------------------------------------------------------------------ algorithms
// Frobenius inversion with LU (Sec. 4.1).  R = double or float.
template <typename R>
size_t frob_lu_ws(int n, int batch, void* ws, Planes<R>* out) {
  Carve c{static_cast<unsigned char*>(ws)};
  Planes<R> p;
  p.LA = plane<R>(c, n, batch);
  p.S = plane<R>(c, n, batch);
  p.Bp = plane<R>(c, n, batch);
  p.X1 = plane<R>(c, n, batch);
  p.Y = plane<R>(c, n, batch);
  p.piv1 = c.take<int>((size_t)n * batch);
  p.piv2 = c.take<int>((size_t)n * batch);
  p.rp1 = c.take<int>((size_t)n * batch);
  p.rp2 = c.take<int>((size_t)n * batch);
  p.partb = c.take<int>((size_t)batch);
  p.infoB = c.take<frob_info>((size_t)batch);
  p.mcs = c.take<unsigned char>(mc_scratch_bytes<R>(n, batch));
  // FP32: split-TF32 tensor-core products; FP64: digit products on the BF16
  // tensor cores (the same slot; only one applies per precision)
  p.tcs_bytes = std::is_same<R, float>::value ? tc_scratch_for(n, batch) : oz_scratch_for(n, batch);
  p.tcs = c.take<unsigned char>(p.tcs_bytes);
  if (out) *out = p;
  return c.off;
}

// FROB_PART_AUTO: per matrix, the pivot ratios min |u_kk| / max |u_kk| of
// the LU factors of A (LA) and B (LB) (0 for a factorization that reported a
// zero or non-finite pivot); B is chosen when its ratio is larger.  One CTA
// per matrix.
template <typename R>
__global__ void choose_part_kernel(int n, MatB<const R> LA, MatB<const R> LB, const frob_info* info,
                                   const frob_info* infoB, int* partb) {
  const int b = blockIdx.x;
  __shared__ double red[4][32];
  double mina = INFINITY, maxa = 0.0, minb = INFINITY, maxb = 0.0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const double ua = fabs((double)LA.at(b)[(int64_t)k * LA.ld + k]);
    const double ub = fabs((double)LB.at(b)[(int64_t)k * LB.ld + k]);
    mina = fmin(mina, ua);
    maxa = fmax(maxa, ua);
    minb = fmin(minb, ub);
    maxb = fmax(maxb, ub);
  }
  for (int o = 16; o > 0; o >>= 1) {
    mina = fmin(mina, __shfl_xor_sync(0xffffffffu, mina, o));
    maxa = fmax(maxa, __shfl_xor_sync(0xffffffffu, maxa, o));
    minb = fmin(minb, __shfl_xor_sync(0xffffffffu, minb, o));
    maxb = fmax(maxb, __shfl_xor_sync(0xffffffffu, maxb, o));
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    red[0][w] = mina;
    red[1][w] = maxa;
    red[2][w] = minb;
    red[3][w] = maxb;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < (int)(blockDim.x >> 5); ++k) {
      mina = fmin(mina, red[0][k]);
      maxa = fmax(maxa, red[1][k]);
      minb = fmin(minb, red[2][k]);
      maxb = fmax(maxb, red[3][k]);
    }
    const double ra = (info[b].status == FROB_OK && maxa > 0.0 && maxa < INFINITY) ? mina / maxa : 0.0;
    const double rb = (infoB[b].status == FROB_OK && maxb > 0.0 && maxb < INFINITY) ? minb / maxb : 0.0;
    partb[b] = rb > ra ? 1 : 0;
  }
}

// For the matrices that take B: LA <- LU of B, piv1 <- its pivots, and the
// planes of -iM = B - iA: S <- B, Bp <- -A (S and Bp held A and B); the LU
// of A's report, if any, is withdrawn.
template <typename R>
__global__ void swap_part_kernel(int n, const int* partb, MatB<R> LA, MatB<const R> LB, MatB<R> S, MatB<R> Bp,
                                 int* piv1, const int* pivB, frob_info* info) {
  const int b = blockIdx.z;
  if (!partb[b]) return;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * n) return;
  const int i = (int)(e / n), j = (int)(e % n);
  LA.at(b)[(int64_t)i * LA.ld + j] = LB.at(b)[(int64_t)i * LB.ld + j];
  R* ps = S.at(b) + (int64_t)i * S.ld + j;
  R* pb = Bp.at(b) + (int64_t)i * Bp.ld + j;
  const R a = *ps, bb = *pb;
  *ps = bb;
  *pb = -a;
  if (j == 0) piv1[(int64_t)b * n + i] = pivB[(int64_t)b * n + i];
  if (e == 0) init_info(info, b, 0.0);
}

template <typename R>
void frob_lu_run(int n, int batch, MatB<const typename cplx_of<R>::type> M, MatB<typename cplx_of<R>::type> X,
                 const frob_opts& o, void* ws, frob_info* info, cudaStream_t st) {
  Planes<R> p;
  frob_lu_ws<R>(n, batch, ws, &p);
  // large products on the tensor cores: split TF32 (FP32), exact BF16 digit
  // products (FP64, unless opts ask for the FP64 pipe)
  TcScope tc_scope(p.tcs, p.tcs_bytes, info, batch, st, std::is_same<R, float>::value);
  OzScope oz_scope(p.tcs, p.tcs_bytes, info, batch, st,
                   std::is_same<R, double>::value && o.fp64_gemm == FROB_GEMM_AUTO);
  auto cst = [](MatB<R> m) { return MatB<const R>{m.p, m.ld, m.bs}; };
  const bool autop = o.part == FROB_PART_AUTO;
  FROB_LAUNCH("split", st, split_kernel<R><<<elem_grid(n, batch), 256, 0, st>>>(n, M, p.LA, p.S, p.Bp, info, 0, o.almost_sure, o.seed,
                                                       o.attempt, o.part == FROB_PART_B ? 1 : 0,
                                                       autop ? p.X1 : MatB<R>{nullptr, 0, 0}, p.partb,
                                                       autop ? p.infoB : nullptr));
  getrf<R>(n, batch, p.LA, p.piv1, info, 0, st, p.mcs, p.Y);                          // A = P1^T L1 U1
  if (autop) {
    // the LU of B in the X1 plane (free until the first solve), its pivots
    // in rp1 (free until the row map is built); keep the better-conditioned
    getrf<R>(n, batch, p.X1, p.rp1, p.infoB, 0, st, p.mcs, p.Y);
    FROB_LAUNCH("choose_part", st,
                choose_part_kernel<R><<<batch, 256, 0, st>>>(n, cst(p.LA), cst(p.X1), info, p.infoB, p.partb));
    FROB_LAUNCH("swap_part", st, swap_part_kernel<R><<<elem_grid(n, batch), 256, 0, st>>>(
                                     n, p.partb, p.LA, cst(p.X1), p.S, p.Bp, p.piv1, p.rp1, info));
  }
  rowperm(n, batch, p.piv1, p.rp1, st);
  trsm_any<R, OP_N, true, true>(n, n, batch, cst(p.LA), cst(p.Bp), p.X1, p.rp1, st);   // L1 Y = P1 B
  trsm_any<R, OP_N, false, false>(n, n, batch, cst(p.LA), cst(p.X1), p.X1, nullptr, st); // U1 X1 = Y
  gemm_launch<R, OP_N, OP_N>(n, n, n, batch, cst(p.Bp), cst(p.X1), axpby<R>(p.S, (R)1, (R)1, false), 0,
                             st);                                                       // S = A + B X1
  getrf<R>(n, batch, p.S, p.piv2, info, n, st, p.mcs, p.LA);  // S = P2^T L2 U2 (L1 U1 no longer needed)
  rowperm(n, batch, p.piv2, p.rp2, st);
  trtri<R, true>(n, batch, cst(p.S), p.Y, p.LA, st);                                     // Y = L2^{-1}
  trsm_any<R, OP_N, false, false>(n, n, batch, cst(p.S), cst(p.Y), p.Y, nullptr, st); // Z = U2^{-1} Y
  EpiFrobOut<R> epi{X, cst(p.Y), p.rp2, n, o.almost_sure ? info : nullptr,
                    o.part != FROB_PART_A ? p.partb : nullptr};
  gemm_launch<R, OP_N, OP_N>(n, n, n, batch, cst(p.X1), cst(p.Y), epi, 0, st);          // X = Z P2 - i X1 Z P2
}

// Frobenius inversion with Cholesky (Sec. 4.3).
template <typename R>
size_t frob_chol_ws(int n, int batch, void* ws, Planes<R>* out) {
  Carve c{static_cast<unsigned char*>(ws)};
  Planes<R> p{};
  p.LA = plane<R>(c, n, batch);
  p.S = plane<R>(c, n, batch);
  p.Bp = plane<R>(c, n, batch);
  p.Y = plane<R>(c, n, batch);
  p.tcs_bytes = std::is_same<R, float>::value ? tc_scratch_for(n, batch) : oz_scratch_for(n, batch);
  p.tcs = c.take<unsigned char>(p.tcs_bytes);
  if (out) *out = p;
  return c.off;
}

template <typename R>
void frob_chol_run(int n, int batch, MatB<const typename cplx_of<R>::type> M, MatB<typename cplx_of<R>::type> X,
                   void* ws, frob_info* info, cudaStream_t st, int fp64_gemm) {
  Planes<R> p;
  frob_chol_ws<R>(n, batch, ws, &p);
  // large products on the tensor cores: split TF32 (FP32), exact BF16 digit
  // products (FP64, unless the caller asks for the FP64 pipe)
  TcScope tc_scope(p.tcs, p.tcs_bytes, info, batch, st, std::is_same<R, float>::value);
  OzScope oz_scope(p.tcs, p.tcs_bytes, info, batch, st,
                   std::is_same<R, double>::value && fp64_gemm == FROB_GEMM_AUTO);
  auto cst = [](MatB<R> m) { return MatB<const R>{m.p, m.ld, m.bs}; };
  FROB_LAUNCH("split", st, split_kernel<R><<<elem_grid(n, batch), 256, 0, st>>>(n, M, p.LA, p.S, p.Bp, info, 1, 0, 0, 0));
  potrf<R>(n, batch, p.LA, info, 0, st);                                                 // A = R1^T R1, L1 = R1^T
  trsm_any<R, OP_N, true, false>(n, n, batch, cst(p.LA), cst(p.Bp), p.Bp, nullptr, st); // X1 = L1^{-1} B
  gemm_launch<R, OP_T, OP_N>(n, n, n, batch, cst(p.Bp), cst(p.Bp), axpby<R>(p.S, (R)-1, (R)1, false), 1,
                             st);                                                         // S = A - X1^T X1
  trsm_any<R, OP_T, false, false>(n, n, batch, cst(p.LA), cst(p.Bp), p.Bp, nullptr, st); // X2 = L1^{-T} X1
  potrf<R>(n, batch, p.S, info, n, st);                                                  // S = R2^T R2
  trtri<R, false>(n, batch, cst(p.S), p.Y, p.LA, st);                                    // X5 = L2^{-1}
  // X6 = L2^{-T} X5 = X5^T X5 (S^{-1} = L2^{-T} L2^{-1}): a product of the
  // triangular inverse with itself, summed over k >= max(i, j), into the
  // plane of S (its factor is no longer needed); the product of a matrix
  // with its own transpose is symmetric in floating point too, so the tiles on
  // and below the diagonal are computed and the rest mirrored
  gemm_launch<R, OP_T, OP_N>(n, n, n, batch, cst(p.Y), cst(p.Y), axpby<R>(p.S, (R)1, (R)0, true), 3, st);
  mirror<R, false>(n, batch, p.S, st);
  // X = X6 - i X2 X6, all tiles: X2 X6 is antisymmetric only up to rounding,
  // and the two computed halves carry the correlated errors that keep the
  // residual at the FP64 level; completing one half from the other raises it
  // to about kappa u
  EpiFrobOut<R> epi{X, cst(p.S), nullptr, n, nullptr};
  gemm_launch<R, OP_N, OP_N>(n, n, n, batch, cst(p.Bp), cst(p.S), epi, 0, st);
}

// Complex LU inversion (Algorithm "Inversion with LU decomposition").
template <typename C>
size_t cplx_lu_ws(int n, int batch, void* ws, CPlanes<C>* out) {
  Carve c{static_cast<unsigned char*>(ws)};
  CPlanes<C> p{};
  p.W = plane<C>(c, n, batch);
  p.Y = plane<C>(c, n, batch);
  p.piv = c.take<int>((size_t)n * batch);
  p.rp = c.take<int>((size_t)n * batch);
  p.mcs = c.take<unsigned char>(mc_scratch_bytes<C>(n, batch));
  if (out) *out = p;
  return c.off;
}

template <typename C>
void cplx_lu_run(int n, int batch, MatB<const C> M, MatB<C> X, void* ws, frob_info* info, cudaStream_t st) {
  CPlanes<C> p;
  cplx_lu_ws<C>(n, batch, ws, &p);
  auto cst = [](MatB<C> m) { return MatB<const C>{m.p, m.ld, m.bs}; };
  FROB_LAUNCH("copy", st, copy_kernel<C><<<elem_grid(n, batch), 256, 0, st>>>(n, M, p.W, info));
  getrf<C>(n, batch, p.W, p.piv, info, 0, st, p.mcs);                                    // M = P^T L U
  rowperm(n, batch, p.piv, p.rp, st);
  trtri<C, true>(n, batch, cst(p.W), p.Y, X, st);                                         // Y = L^{-1}
  trsm_any<C, OP_N, false, false>(n, n, batch, cst(p.W), cst(p.Y), p.Y, nullptr, st);  // Z = U^{-1} Y
  FROB_LAUNCH("colperm", st, colperm_kernel<C><<<elem_grid(n, batch), 256, 0, st>>>(n, cst(p.Y), X, p.rp));          // X = Z P
}

// Complex Cholesky inversion (Algorithm "Inversion with Cholesky decomposition").
template <typename C>
size_t cplx_chol_ws(int n, int batch, void* ws, CPlanes<C>* out) {
  Carve c{static_cast<unsigned char*>(ws)};
  CPlanes<C> p{};
  p.W = plane<C>(c, n, batch);
  p.Y = plane<C>(c, n, batch);
  if (out) *out = p;
  return c.off;
}

template <typename C>
void cplx_chol_run(int n, int batch, MatB<const C> M, MatB<C> X, void* ws, frob_info* info, cudaStream_t st) {
  CPlanes<C> p;
  cplx_chol_ws<C>(n, batch, ws, &p);
  auto cst = [](MatB<C> m) { return MatB<const C>{m.p, m.ld, m.bs}; };
  FROB_LAUNCH("copy", st, copy_kernel<C><<<elem_grid(n, batch), 256, 0, st>>>(n, M, p.W, info));
  potrf<C>(n, batch, p.W, info, 0, st);                                                  // M = R^H R, L = R^H
  trtri<C, false>(n, batch, cst(p.W), p.Y, X, st);                                        // X1 = L^{-1}
  // X2 = L^{-H} X1 = X1^H X1: the triangular inverse times itself, summed
  // over k >= max(i, j); Hermitian in floating point too (a matrix times its
  // own conjugate transpose), so the tiles on and below the diagonal are
  // computed and the rest mirrored
  gemm_launch<C, OP_C, OP_N>(n, n, n, batch, cst(p.Y), cst(p.Y), axpby<C>(X, one_v<C>(), zero_v<C>(), true), 3, st);
  mirror<C, true>(n, batch, X, st);
}

// ------------------------------------------------------------------ linear solve
// Algorithm "Linear system with Frobenius inversion" (Sec. 3) for nrhs
// right-hand sides C + iD:  A = P1^T L1 U1; X1 = A^{-1} B; S = A + B X1;
// S = P2^T L2 U2; [x1, y1] = S^{-1} [C, D]; [x2, y2] = A^{-1} B [y1, x1];
// x = x1 + x2, y = y1 - y2 (the printed last step has y2 - y1; eq. (1.1)
// gives y1 - y2).
template <typename R>
__global__ void rhs_split_kernel(int n, int nrhs, MatB<const typename cplx_of<R>::type> Bc, MatB<R> CD) {
  const int b = blockIdx.z;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * nrhs) return;
  const int i = (int)(e / nrhs), j = (int)(e % nrhs);
  const auto v = Bc.at(b)[(int64_t)i * Bc.ld + j];
  CD.at(b)[(int64_t)i * CD.ld + j] = v.x;
  CD.at(b)[(int64_t)i * CD.ld + nrhs + j] = v.y;
}

template <typename R>
__global__ void solve_out_kernel(int n, int nrhs, MatB<const R> T, MatB<const R> U,
                                 MatB<typename cplx_of<R>::type> X) {
  const int b = blockIdx.z;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * nrhs) return;
  const int i = (int)(e / nrhs), j = (int)(e % nrhs);
  const R* t = T.at(b) + (int64_t)i * T.ld;
  const R* u = U.at(b) + (int64_t)i * U.ld;
  typename cplx_of<R>::type v;
  v.x = t[j] + u[j];               // x = x1 + x2
  v.y = t[nrhs + j] - u[nrhs + j];  // y = y1 - y2
  X.at(b)[(int64_t)i * X.ld + j] = v;
}

inline dim3 rect_grid(int n, int m, int batch) {
  int64_t nn = (int64_t)n * m;
  return dim3((unsigned)((nn + 255) / 256), 1, (unsigned)batch);
}

template <typename R> struct SolvePlanes {
  MatB<R> LA, S, Bp, X1, CD, T, U;
  int *piv1, *piv2, *rp1, *rp2;
  unsigned char* mcs;
  unsigned char* tcs;  // tensor-core products' scratch (split TF32 / FP64 digits)
  size_t tcs_bytes;
};

template <typename R> size_t frob_solve_ws(int n, int nrhs, int batch, SolvePlanes<R>* out, void* ws) {
  Carve c{static_cast<unsigned char*>(ws)};
  SolvePlanes<R> p;
  p.LA = plane<R>(c, n, batch);
  p.S = plane<R>(c, n, batch);
  p.Bp = plane<R>(c, n, batch);
  p.X1 = plane<R>(c, n, batch);
  auto rect = [&]() {
    R* q = c.take<R>((size_t)n * 2 * nrhs * batch);
    return MatB<R>{q, 2 * (int64_t)nrhs, (int64_t)n * 2 * nrhs};
  };
  p.CD = rect();
  p.T = rect();
  p.U = rect();
  p.piv1 = c.take<int>((size_t)n * batch);
  p.piv2 = c.take<int>((size_t)n * batch);
  p.rp1 = c.take<int>((size_t)n * batch);
  p.rp2 = c.take<int>((size_t)n * batch);
  p.mcs = c.take<unsigned char>(mc_scratch_bytes<R>(n, batch));
  p.tcs_bytes = std::is_same<R, float>::value ? tc_scratch_for(n, batch) : oz_scratch_for(n, batch);
  p.tcs = c.take<unsigned char>(p.tcs_bytes);
  if (out) *out = p;
  return c.off;
}

template <typename R>
void frob_solve_run(int n, int nrhs, int batch, MatB<const typename cplx_of<R>::type> M,
                    MatB<const typename cplx_of<R>::type> Bc, MatB<typename cplx_of<R>::type> X, void* ws,
                    frob_info* info, cudaStream_t st) {
  SolvePlanes<R> p;
  frob_solve_ws<R>(n, nrhs, batch, &p, ws);
  // the large products (S = A + B X1, the B [y1 | x1] products) on the tensor cores
  TcScope tc_scope(p.tcs, p.tcs_bytes, info, batch, st, std::is_same<R, float>::value);
  OzScope oz_scope(p.tcs, p.tcs_bytes, info, batch, st, std::is_same<R, double>::value);
  auto cst = [](MatB<R> m) { return MatB<const R>{m.p, m.ld, m.bs}; };
  const int m2 = 2 * nrhs;
  FROB_LAUNCH("split", st, split_kernel<R><<<elem_grid(n, batch), 256, 0, st>>>(n, M, p.LA, p.S, p.Bp, info, 0, 0, 0, 0));
  getrf<R>(n, batch, p.LA, p.piv1, info, 0, st, p.mcs);                                       // step 1
  rowperm(n, batch, p.piv1, p.rp1, st);
  trsm_any<R, OP_N, true, true>(n, n, batch, cst(p.LA), cst(p.Bp), p.X1, p.rp1, st);          // step 2
  trsm_any<R, OP_N, false, false>(n, n, batch, cst(p.LA), cst(p.X1), p.X1, nullptr, st);
  gemm_launch<R, OP_N, OP_N>(n, n, n, batch, cst(p.Bp), cst(p.X1), axpby<R>(p.S, (R)1, (R)1, false), 0, st);  // 3
  getrf<R>(n, batch, p.S, p.piv2, info, n, st, p.mcs);                                        // step 4
  rowperm(n, batch, p.piv2, p.rp2, st);
  FROB_LAUNCH("rhs_split", st, rhs_split_kernel<R><<<rect_grid(n, nrhs, batch), 256, 0, st>>>(n, nrhs, Bc, p.CD));
  trsm_any<R, OP_N, true, true>(n, m2, batch, cst(p.S), cst(p.CD), p.T, p.rp2, st);          // step 5
  trsm_any<R, OP_N, false, false>(n, m2, batch, cst(p.S), cst(p.T), p.T, nullptr, st);     // T = [x1 | y1]
  // step 6: CD = B [y1 | x1], then U = A^{-1} CD = [x2 | y2]
  MatB<const R> Ty{p.T.p + nrhs, p.T.ld, p.T.bs}, Tx{p.T.p, p.T.ld, p.T.bs};
  gemm_launch<R, OP_N, OP_N>(n, nrhs, n, batch, cst(p.Bp), Ty, axpby<R>(p.CD, (R)1, (R)0, true), 0, st);
  gemm_launch<R, OP_N, OP_N>(n, nrhs, n, batch, cst(p.Bp), Tx,
                             axpby<R>(MatB<R>{p.CD.p + nrhs, p.CD.ld, p.CD.bs}, (R)1, (R)0, true), 0, st);
  trsm_any<R, OP_N, true, true>(n, m2, batch, cst(p.LA), cst(p.CD), p.U, p.rp1, st);
  trsm_any<R, OP_N, false, false>(n, m2, batch, cst(p.LA), cst(p.U), p.U, nullptr, st);
  FROB_LAUNCH("solve_out", st,
              solve_out_kernel<R><<<rect_grid(n, nrhs, batch), 256, 0, st>>>(n, nrhs, cst(p.T), cst(p.U), X));  // 7
}

// Complex LU solve (the baseline): M = P^T L U, L Y = P C, U X = Y.
template <typename C> size_t cplx_solve_ws(int n, int nrhs, int batch) {
  Carve c{nullptr};
  plane<C>(c, n, batch);
  c.take<C>((size_t)n * nrhs * batch);
  c.take<int>((size_t)n * batch);
  c.take<int>((size_t)n * batch);
  c.take<unsigned char>(mc_scratch_bytes<C>(n, batch));
  return c.off;
}

template <typename C>
void cplx_solve_run(int n, int nrhs, int batch, MatB<const C> M, MatB<const C> Bc, MatB<C> X, void* ws,
                    frob_info* info, cudaStream_t st) {
  Carve c{static_cast<unsigned char*>(ws)};
  MatB<C> W = plane<C>(c, n, batch);
  C* yp = c.take<C>((size_t)n * nrhs * batch);
  int* piv = c.take<int>((size_t)n * batch);
  int* rp = c.take<int>((size_t)n * batch);
  unsigned char* mcs = c.take<unsigned char>(mc_scratch_bytes<C>(n, batch));
  MatB<C> Y{yp, nrhs, (int64_t)n * nrhs};
  auto cst = [](MatB<C> m) { return MatB<const C>{m.p, m.ld, m.bs}; };
  FROB_LAUNCH("copy", st, copy_kernel<C><<<elem_grid(n, batch), 256, 0, st>>>(n, M, W, info));
  getrf<C>(n, batch, W, piv, info, 0, st, mcs);
  rowperm(n, batch, piv, rp, st);
  trsm_any<C, OP_N, true, true>(n, nrhs, batch, cst(W), Bc, Y, rp, st);
  trsm_any<C, OP_N, false, false>(n, nrhs, batch, cst(W), cst(Y), X, nullptr, st);
}

// The 2n real augmented system (the third linear-solve method of Sec. 5.2):
// [[A, -B], [B, A]] [x; y] = [c; d] for M (x + iy) = c + id, by real LU with
// partial pivoting of the 2n x 2n matrix.  A failed pivot k (1-based, up to
// 2n) is reported as FROB_ERR_SINGULAR with bad_index = k.
template <typename R>
__global__ void aug_build_kernel(int n, MatB<const typename cplx_of<R>::type> M, MatB<R> W) {
  const int b = blockIdx.z;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * n) return;
  const int i = (int)(e / n), j = (int)(e % n);
  const auto v = M.at(b)[(int64_t)i * M.ld + j];
  R* w = W.at(b);
  w[(int64_t)i * W.ld + j] = v.x;              // A
  w[(int64_t)i * W.ld + n + j] = -v.y;         // -B
  w[(int64_t)(n + i) * W.ld + j] = v.y;        // B
  w[(int64_t)(n + i) * W.ld + n + j] = v.x;    // A
}

template <typename R>
__global__ void aug_rhs_kernel(int n, int nrhs, MatB<const typename cplx_of<R>::type> Bc, MatB<R> CD,
                               frob_info* info) {
  const int b = blockIdx.z;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e == 0) init_info(info, b, 0.0);
  if (e >= (int64_t)n * nrhs) return;
  const int i = (int)(e / nrhs), j = (int)(e % nrhs);
  const auto v = Bc.at(b)[(int64_t)i * Bc.ld + j];
  CD.at(b)[(int64_t)i * CD.ld + j] = v.x;
  CD.at(b)[(int64_t)(n + i) * CD.ld + j] = v.y;
}

template <typename R>
__global__ void aug_out_kernel(int n, int nrhs, MatB<const R> XY, MatB<typename cplx_of<R>::type> X) {
  const int b = blockIdx.z;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * nrhs) return;
  const int i = (int)(e / nrhs), j = (int)(e % nrhs);
  typename cplx_of<R>::type v;
  v.x = XY.at(b)[(int64_t)i * XY.ld + j];
  v.y = XY.at(b)[(int64_t)(n + i) * XY.ld + j];
  X.at(b)[(int64_t)i * X.ld + j] = v;
}

template <typename R> size_t aug_solve_ws(int n, int nrhs, int batch) {
  Carve c{nullptr};
  plane<R>(c, 2 * n, batch);
  c.take<R>((size_t)2 * n * nrhs * batch);
  c.take<R>((size_t)2 * n * nrhs * batch);
  c.take<int>((size_t)2 * n * batch);
  c.take<int>((size_t)2 * n * batch);
  c.take<unsigned char>(mc_scratch_bytes<R>(2 * n, batch));
  return c.off;
}

template <typename R>
void aug_solve_run(int n, int nrhs, int batch, MatB<const typename cplx_of<R>::type> M,
                   MatB<const typename cplx_of<R>::type> Bc, MatB<typename cplx_of<R>::type> X, void* ws,
                   frob_info* info, cudaStream_t st) {
  Carve c{static_cast<unsigned char*>(ws)};
  const int n2 = 2 * n;
  MatB<R> W = plane<R>(c, n2, batch);
  R* cdp = c.take<R>((size_t)n2 * nrhs * batch);
  R* xyp = c.take<R>((size_t)n2 * nrhs * batch);
  int* piv = c.take<int>((size_t)n2 * batch);
  int* rp = c.take<int>((size_t)n2 * batch);
  unsigned char* mcs = c.take<unsigned char>(mc_scratch_bytes<R>(n2, batch));
  MatB<R> CD{cdp, nrhs, (int64_t)n2 * nrhs}, XY{xyp, nrhs, (int64_t)n2 * nrhs};
  auto cst = [](MatB<R> m) { return MatB<const R>{m.p, m.ld, m.bs}; };
  FROB_LAUNCH("aug_build", st, aug_build_kernel<R><<<elem_grid(n, batch), 256, 0, st>>>(n, M, W));
  FROB_LAUNCH("aug_rhs", st, aug_rhs_kernel<R><<<rect_grid(n, nrhs, batch), 256, 0, st>>>(n, nrhs, Bc, CD, info));
  getrf<R>(n2, batch, W, piv, info, 0, st, mcs);
  rowperm(n2, batch, piv, rp, st);
  trsm_any<R, OP_N, true, true>(n2, nrhs, batch, cst(W), cst(CD), XY, rp, st);
  trsm_any<R, OP_N, false, false>(n2, nrhs, batch, cst(W), cst(XY), XY, nullptr, st);
  FROB_LAUNCH("aug_out", st, aug_out_kernel<R><<<rect_grid(n, nrhs, batch), 256, 0, st>>>(n, nrhs, cst(XY), X));
}

// ------------------------------------------------------------------ adjoint
// grad M = -X^H G X^H for X = M^{-1} (d(M^{-1}) = -M^{-1} dM M^{-1}), as two
// complex products, each by Gauss's three real multiplications (Sec. 2,
// Proposition "matrix mult"):
//   P = X^H G:  T1 = Xr^T Gr, T2 = Xi^T Gi, T3 = (Xr - Xi)^T (Gr + Gi)
//               Re P = T1 + T2, Im P = T3 - T1 + T2
//   Q = P X^H:  U1 = Pr Xr^T, U2 = Pi Xi^T, U3 = (Pr + Pi)(Xr - Xi)^T
//               Re Q = U1 + U2, Im Q = U3 - U1 + U2
//   grad = -Q
template <typename R>
__global__ void adj_split_kernel(int n, MatB<const typename cplx_of<R>::type> X,
                                 MatB<const typename cplx_of<R>::type> G, MatB<R> Xr, MatB<R> Xi, MatB<R> Xd,
                                 MatB<R> Gr, MatB<R> Gi, MatB<R> Gs) {
  const int b = blockIdx.z;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * n) return;
  const int i = (int)(e / n), j = (int)(e % n);
  auto x = X.at(b)[(int64_t)i * X.ld + j];
  auto g = G.at(b)[(int64_t)i * G.ld + j];
  const int64_t o = (int64_t)i * Xr.ld + j;
  Xr.at(b)[o] = x.x;
  Xi.at(b)[o] = x.y;
  Xd.at(b)[o] = x.x - x.y;
  Gr.at(b)[o] = g.x;
  Gi.at(b)[o] = g.y;
  Gs.at(b)[o] = g.x + g.y;
}

// in place: (T1, T2, T3) -> (Re P, Im P, Re P + Im P)
template <typename R>
__global__ void adj_combine_kernel(int n, MatB<R> T1, MatB<R> T2, MatB<R> T3) {
  const int b = blockIdx.z;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * n) return;
  const int64_t o = (e / n) * T1.ld + (e % n);
  const R t1 = T1.at(b)[o], t2 = T2.at(b)[o], t3 = T3.at(b)[o];
  const R pr = t1 + t2, pi = t3 - t1 + t2;
  T1.at(b)[o] = pr;
  T2.at(b)[o] = pi;
  T3.at(b)[o] = pr + pi;
}

template <typename R>
__global__ void adj_out_kernel(int n, MatB<const R> U1, MatB<const R> U2, MatB<const R> U3,
                               MatB<typename cplx_of<R>::type> out) {
  const int b = blockIdx.z;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * n) return;
  const int i = (int)(e / n), j = (int)(e % n);
  const int64_t o = (int64_t)i * U1.ld + j;
  const R u1 = U1.at(b)[o], u2 = U2.at(b)[o], u3 = U3.at(b)[o];
  typename cplx_of<R>::type v;
  v.x = -(u1 + u2);
  v.y = -(u3 - u1 + u2);
  out.at(b)[(int64_t)i * out.ld + j] = v;
}

template <typename R> size_t adjoint_ws(int n, int batch) {
  Carve c{nullptr};
  for (int k = 0; k < 9; ++k) plane<R>(c, n, batch);
  c.take<unsigned char>(std::is_same<R, float>::value ? tc_scratch_for(n, batch) : 0);
  return c.off;
}

// the adjoint has no info records: a tensor-core product whose bounded wait
// gave up turns the whole result into NaN
template <typename C> __global__ void adj_nan_on_err_kernel(int n, const int* err, MatB<C> out) {
  if (*err == 0) return;
  const int b = blockIdx.z;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * n) return;
  const int i = (int)(e / n), j = (int)(e % n);
  out.at(b)[(int64_t)i * out.ld + j] = C{NAN, NAN};
}

template <typename R>
void adjoint_run(int n, int batch, MatB<const typename cplx_of<R>::type> X, MatB<const typename cplx_of<R>::type> G,
                 MatB<typename cplx_of<R>::type> out, void* ws, cudaStream_t st) {
  Carve c{static_cast<unsigned char*>(ws)};
  MatB<R> P[9];
  for (int k = 0; k < 9; ++k) P[k] = plane<R>(c, n, batch);
  const size_t tcb = std::is_same<R, float>::value ? tc_scratch_for(n, batch) : 0;
  unsigned char* tcs = c.take<unsigned char>(tcb);
  TcScope tc_scope(tcs, tcb, nullptr, batch, st);  // FP32: the six products on the tensor cores
  MatB<R>&Xr = P[0], &Xi = P[1], &Xd = P[2], &Gr = P[3], &Gi = P[4], &Gs = P[5], &T1 = P[6], &T2 = P[7], &T3 = P[8];
  auto cst = [](MatB<R> m) { return MatB<const R>{m.p, m.ld, m.bs}; };
  const R one = (R)1, zero = (R)0;
  FROB_LAUNCH("adj_split", st, adj_split_kernel<R><<<elem_grid(n, batch), 256, 0, st>>>(n, X, G, Xr, Xi, Xd, Gr, Gi, Gs));
  gemm_launch<R, OP_T, OP_N>(n, n, n, batch, cst(Xr), cst(Gr), axpby<R>(T1, one, zero, true), 0, st);
  gemm_launch<R, OP_T, OP_N>(n, n, n, batch, cst(Xi), cst(Gi), axpby<R>(T2, one, zero, true), 0, st);
  gemm_launch<R, OP_T, OP_N>(n, n, n, batch, cst(Xd), cst(Gs), axpby<R>(T3, one, zero, true), 0, st);
  FROB_LAUNCH("adj_combine", st, adj_combine_kernel<R><<<elem_grid(n, batch), 256, 0, st>>>(n, T1, T2, T3));
  // U1 -> Gr, U2 -> Gi, U3 -> Gs (the G planes are free now)
  gemm_launch<R, OP_N, OP_T>(n, n, n, batch, cst(T1), cst(Xr), axpby<R>(Gr, one, zero, true), 0, st);
  gemm_launch<R, OP_N, OP_T>(n, n, n, batch, cst(T2), cst(Xi), axpby<R>(Gi, one, zero, true), 0, st);
  gemm_launch<R, OP_N, OP_T>(n, n, n, batch, cst(T3), cst(Xd), axpby<R>(Gs, one, zero, true), 0, st);
  FROB_LAUNCH("adj_out", st, adj_out_kernel<R><<<elem_grid(n, batch), 256, 0, st>>>(n, cst(Gr), cst(Gi), cst(Gs), out));
  if (t_tc.err)
    FROB_LAUNCH("adj_nan_on_err", st,
                adj_nan_on_err_kernel<typename cplx_of<R>::type><<<elem_grid(n, batch), 256, 0, st>>>(n, t_tc.err, out));
}

}  // namespace frob
