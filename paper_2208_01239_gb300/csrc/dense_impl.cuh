// Dense building blocks of Frobenius inversion on the CUDA cores (FP64 DFMA /
// FP32 FFMA), templated over the scalar type:
//   T = double, float  -> the real planes of Frobenius inversion (Sec. 4.1,
//                         4.3 of Dai, Lim and Ye)
//   T = zd, zf         -> complex arithmetic for the baselines
//                         (Algorithms "Inversion with LU / Cholesky
//                         decomposition")
//
// On GB300 the FP64 pipe retires about 2 DFMA per clock per SM, so every FP64
// kernel here is bound by that pipe, not by memory: the design goal is to keep
// all 152 SMs issuing FMAs (batched grids over tiles x matrices), not to
// minimise bytes.
//
// Kernels:
//   gemm_kernel        D = alpha op(A) op(B) + beta C, 64x64 tiles, with a
//                      pluggable epilogue (plain, or the Frobenius output
//                      writer that interleaves Re/Im, permutes columns and
//                      applies the almost-sure un-rotation).
//   trsm_step_kernel   one block row of a blocked triangular solve
//                      op(T) X = B: a GEMM over the finished block rows, then
//                      substitution with the 64x64 diagonal block in shared
//                      memory.  Optionally B = I with the zero blocks of the
//                      triangular result skipped.
//   getrf_panel_kernel LU with partial pivoting of one column panel; pivot
//                      search by warp-shuffle argmax.
//   laswp_trsm_kernel  applies a panel's row swaps to the other columns and
//                      forms U12 = L11^{-1} A12.
//   trtri_diag_kernel  inverses of the 64x64 diagonal blocks of a lower
//                      triangular matrix (the first step of trtri).
//   potrf_panel_kernel one 32-wide panel of a blocked Cholesky (lower,
//                      A = L L^H): the diagonal block by one warp in
//                      registers (redone by every CTA), then the rows below
//                      it, L21 = A21 L11^{-H}, one thread per row.
//   potrf_small_kernel the whole Cholesky of a real FP32 matrix with n <= 512
//                      by one CTA (panels, row solves and trailing updates
//                      between CTA barriers).
//   getrf_small_kernel the whole LU with partial pivoting of a real FP32
//                      matrix with n <= 512 by one CTA (rows addressed
//                      through a permutation, gathered at the end).
//   mirror_kernel      completes a symmetric / Hermitian matrix from its
//                      lower tiles.
#pragma once

#include <cooperative_groups.h>
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"
#include "ops.h"

namespace frob {

constexpr int TB = 64;   // tile rows / cols (also the block size of the blocked solvers)
constexpr int TK = 16;   // k step of the GEMM mainloop
constexpr int NTH = 256; // threads per GEMM / TRSM CTA

// ------------------------------------------------------------------ mainloop
// acc[r][c] += sum_{k in [kbeg, kend)} opA(i0 + 4 ty + r, k) * opB(k, j0 + 4 tx + c)
// where opA(i, k) = A[i][k] (OP_N), A[k][i] (OP_T) or conj(A[k][i]) (OP_C),
// and opB(k, j) = B[k][j] (OP_N), B[j][k] (OP_T) or conj(B[j][k]) (OP_C).
// Out-of-range rows (>= M), columns (>= N) and k (>= kend) read as zero.
// Each thread owns 4 consecutive rows and columns, so that its operands come
// from shared memory as 16-byte vectors (2 vector loads per 16 FMAs: the
// FP32 path would otherwise be bound by shared-memory loads); rows are padded
// to keep 16-byte alignment.
template <typename T> struct SmemAB {
  static constexpr int LD = TB + (16 / (int)sizeof(T) > 1 ? 16 / (int)sizeof(T) : 1);
  T a[TK][LD];
  T b[TK][LD];
};

// 4 consecutive elements from a 16-byte aligned shared-memory address
__device__ __forceinline__ void ld4(const float* p, float (&v)[4]) {
  const float4 q = *reinterpret_cast<const float4*>(p);
  v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ __forceinline__ void ld4(const double* p, double (&v)[4]) {
  const double2 q0 = reinterpret_cast<const double2*>(p)[0], q1 = reinterpret_cast<const double2*>(p)[1];
  v[0] = q0.x; v[1] = q0.y; v[2] = q1.x; v[3] = q1.y;
}
__device__ __forceinline__ void ld4(const zf* p, zf (&v)[4]) {
  const float4 q0 = reinterpret_cast<const float4*>(p)[0], q1 = reinterpret_cast<const float4*>(p)[1];
  v[0] = zf{q0.x, q0.y}; v[1] = zf{q0.z, q0.w}; v[2] = zf{q1.x, q1.y}; v[3] = zf{q1.z, q1.w};
}
__device__ __forceinline__ void ld4(const zd* p, zd (&v)[4]) {
#pragma unroll
  for (int i = 0; i < 4; ++i) v[i] = p[i];
}

template <typename T, int OPA>
__device__ __forceinline__ T load_opA(const T* A, int64_t lda, int i, int k, int M, int kend) {
  if (i >= M || k >= kend) return zero_v<T>();
  if (OPA == OP_N) return A[(int64_t)i * lda + k];
  T v = A[(int64_t)k * lda + i];
  return OPA == OP_C ? conj_(v) : v;
}
template <typename T, int OPB>
__device__ __forceinline__ T load_opB(const T* B, int64_t ldb, int k, int j, int N, int kend) {
  if (j >= N || k >= kend) return zero_v<T>();
  if (OPB == OP_N) return B[(int64_t)k * ldb + j];
  T v = B[(int64_t)j * ldb + k];
  return OPB == OP_C ? conj_(v) : v;
}

template <typename T, int OPA, int OPB>
__device__ __forceinline__ void mainloop(T (&acc)[4][4], SmemAB<T>& sm, const T* A, int64_t lda, const T* B,
                                         int64_t ldb, int M, int N, int i0, int j0, int kbeg, int kend) {
  const int t = threadIdx.x;
  const int tx = t & 15, ty = t >> 4;
  T ra[4], rb[4];
  // element e = t + 256 q of the 64x16 A tile / 16x64 B tile; the mapping
  // keeps consecutive threads on consecutive addresses of the source.
  auto fetch = [&](int k0) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int e = t + NTH * q;
      int il, kl;
      if (OPA == OP_N) { il = e >> 4; kl = e & 15; } else { il = e & 63; kl = e >> 6; }
      ra[q] = load_opA<T, OPA>(A, lda, i0 + il, k0 + kl, M, kend);
      int jl, kl2;
      if (OPB == OP_N) { jl = e & 63; kl2 = e >> 6; } else { jl = e >> 4; kl2 = e & 15; }
      rb[q] = load_opB<T, OPB>(B, ldb, k0 + kl2, j0 + jl, N, kend);
    }
  };
  auto stash = [&]() {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int e = t + NTH * q;
      int il, kl;
      if (OPA == OP_N) { il = e >> 4; kl = e & 15; } else { il = e & 63; kl = e >> 6; }
      sm.a[kl][il] = ra[q];
      int jl, kl2;
      if (OPB == OP_N) { jl = e & 63; kl2 = e >> 6; } else { jl = e >> 4; kl2 = e & 15; }
      sm.b[kl2][jl] = rb[q];
    }
  };
  if (kbeg >= kend) return;
  fetch(kbeg);
  for (int k0 = kbeg; k0 < kend; k0 += TK) {
    __syncthreads();
    stash();
    __syncthreads();
    if (k0 + TK < kend) fetch(k0 + TK);
#pragma unroll 4
    for (int kk = 0; kk < TK; ++kk) {
      T av[4], bv[4];
      ld4(&sm.a[kk][4 * ty], av);
      ld4(&sm.b[kk][4 * tx], bv);
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) mac(acc[r][c], av[r], bv[c]);
    }
  }
}

// ------------------------------------------------------------------ GEMM
// Epilogue: D = alpha * acc + beta * C (C may alias D; C is not read when
// beta_is_zero).
template <typename T> struct EpiAxpby {
  static constexpr const char* tag = "axpby";
  MatB<T> D;
  MatB<const T> C;
  T alpha, beta;
  int beta_is_zero;
  __device__ __forceinline__ void operator()(int b, int i, int j, T v) const {
    T out = mul_(alpha, v);
    if (!beta_is_zero) out = add_(out, mul_(beta, C.at(b)[(int64_t)i * C.ld + j]));
    D.at(b)[(int64_t)i * D.ld + j] = out;
  }
  static constexpr bool kRow = true;
  template <int W>
  __device__ __forceinline__ void row(int b, int i, int j0, const T (&v)[W], int ncols) const {
    T* d = D.at(b) + (int64_t)i * D.ld + j0;
    if (!beta_is_zero) {
      const T* c = C.at(b) + (int64_t)i * C.ld + j0;
      T cv[W];
#pragma unroll
      for (int q = 0; q < W; ++q) cv[q] = (j0 + q < ncols) ? c[q] : zero_v<T>();
#pragma unroll
      for (int q = 0; q < W; ++q)
        if (j0 + q < ncols) d[q] = add_(mul_(alpha, v[q]), mul_(beta, cv[q]));
    } else {
#pragma unroll
      for (int q = 0; q < W; ++q)
        if (j0 + q < ncols) d[q] = mul_(alpha, v[q]);
    }
  }
};

// The last product of Frobenius inversion, W = X1 Z with Z = S^{-1} (up to
// the column permutation P2), written straight into the interleaved complex
// result (Sec. 4.1, Algorithm "Frobenius inversion with LU decomposition",
// output X3 - i X4 with X3 = S^{-1}, X4 = X1 S^{-1}):
//   X[i][dst(j)] = (Z[i][j], -W[i][j])                         (mu = 0)
//   X[i][dst(j)] = (X3 - mu X4, mu X3 + X4), X3 = Z, X4 = -W   (almost sure,
//                                                  Sec. 4.2, Algorithm "Almost
//                                                  sure Frobenius inversion")
// dst = rowperm of P2 (S^{-1} = Z P2 moves column j of Z to column rp[j]);
// NULL for no permutation (Cholesky variant).
template <typename R> struct EpiFrobOut {
  static constexpr const char* tag = "frob_out";
  using C = typename cplx_of<R>::type;
  MatB<C> X;
  MatB<const R> Z;
  const int* rp;     // per-matrix permutation, batch stride n, or NULL
  int n;
  const frob_info* info; // info[b].mu, or NULL for mu = 0
  const int* partb = nullptr;  // partb[b] = 1: the inverse of -iM was formed, M^{-1} = -i (X3 + i X4)
  __device__ __forceinline__ void operator()(int b, int i, int j, R w) const {
    R x3 = Z.at(b)[(int64_t)i * Z.ld + j];
    R x4 = -w;
    int jd = rp ? rp[(int64_t)b * n + j] : j;
    C out;
    if (info) {
      R mu = (R)info[b].mu;
      out.x = x3 - mu * x4;
      out.y = mu * x3 + x4;
    } else if (partb && partb[b]) {
      out.x = x4;
      out.y = -x3;
    } else {
      out.x = x3;
      out.y = x4;
    }
    X.at(b)[(int64_t)i * X.ld + jd] = out;
  }
  static constexpr bool kRow = true;
  template <int W>
  __device__ __forceinline__ void row(int b, int i, int j0, const R (&w)[W], int ncols) const {
    const R* z = Z.at(b) + (int64_t)i * Z.ld + j0;
    R x3[W];
    int jd[W];
#pragma unroll
    for (int q = 0; q < W; ++q) {
      const bool in = j0 + q < ncols;
      x3[q] = in ? z[q] : R(0);
      jd[q] = (in && rp) ? rp[(int64_t)b * n + j0 + q] : j0 + q;
    }
    const R mu = info ? (R)info[b].mu : R(0);
    const bool swap = !info && partb && partb[b];
    C* x = X.at(b) + (int64_t)i * X.ld;
#pragma unroll
    for (int q = 0; q < W; ++q) {
      if (j0 + q >= ncols) continue;
      const R x4 = -w[q];
      C out;
      if (info) {
        out.x = x3[q] - mu * x4;
        out.y = mu * x3[q] + x4;
      } else if (swap) {
        out.x = x4;
        out.y = -x3[q];
      } else {
        out.x = x3[q];
        out.y = x4;
      }
      x[jd[q]] = out;
    }
  }
};

// tile_mode: 0 = all tiles; 1 = only tiles that touch the lower triangle
// (j0 <= i0 + 63), for products known to be symmetric / Hermitian; 2 = the
// sum starts at k = max(i0, j0), for op(A) op(B) = L^T L or L^H L with L lower
// triangular (opA(i, k) = 0 for k < i, opB(k, j) = 0 for k < j); 3 = both;
// bit 4: the sum starts at k = j0 (opB lower triangular: opB(k, j) = 0 for
// k < j); bit 8: it ends at k = i0 + 64 (opA lower triangular: opA(i, k) = 0
// for k > i).
template <typename T, int OPA, int OPB, class Epi>
__global__ void __launch_bounds__(NTH) gemm_kernel(int M, int N, int K, MatB<const T> A, MatB<const T> B, Epi epi,
                                                   int tile_mode, int npairs, int shift) {
  // blockIdx.z = matrix * npairs + pair: pair p moves every operand and the
  // output p * shift rows and columns down the diagonal (several equal
  // diagonal-block problems of one matrix in one launch)
  const int b = blockIdx.z / npairs;
  const int64_t dsh = (int64_t)(blockIdx.z % npairs) * shift;
  const int i0 = blockIdx.y * TB, j0 = blockIdx.x * TB;
  if ((tile_mode & 1) && j0 > i0 + TB - 1) return;
  __shared__ SmemAB<T> sm;
  T acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = zero_v<T>();
  int kbeg = (tile_mode & 2) ? (i0 > j0 ? i0 : j0) : 0;
  if ((tile_mode & 4) && j0 > kbeg) kbeg = j0;
  const int kend = ((tile_mode & 8) && i0 + TB < K) ? i0 + TB : K;
  mainloop<T, OPA, OPB>(acc, sm, A.at(b) + dsh * (A.ld + 1), A.ld, B.at(b) + dsh * (B.ld + 1), B.ld, M, N, i0, j0,
                        kbeg, kend);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      int i = i0 + 4 * ty + r, j = j0 + 4 * tx + c;
      if (i < M && j < N) epi(b, (int)(i + dsh), (int)(j + dsh), acc[r][c]);
    }
}

// ------------------------------------------------------------------ narrow update
// D[i][j] -= sum_k L[i][k] U[k][j] for N, K <= 32 (the next panel's columns in
// the LU's look-ahead): 32 rows x N columns per CTA, 256 threads, each thread
// 4 outputs of one column; L's rows and U staged in shared memory.  No
// masked work (the 64 x 64 tiles of gemm_kernel would spend half their FMAs
// on absent columns), and twice the CTAs.  grid (ceil(M / 32), 1, batch).
template <typename T>
__global__ void __launch_bounds__(256) update_narrow_kernel(int M, int N, int K, MatB<const T> L, MatB<const T> U,
                                                            MatB<T> D) {
  __shared__ T sl[32][33];
  __shared__ T su[32][33];
  const int b = blockIdx.z;
  const int i0 = blockIdx.x * 32;
  const int t = threadIdx.x;
  const T* Lb = L.at(b);
  const T* Ub = U.at(b);
  for (int e = t; e < 32 * 32; e += 256) {
    const int r = e >> 5, q = e & 31;
    sl[r][q] = (i0 + r < M && q < K) ? Lb[(int64_t)(i0 + r) * L.ld + q] : zero_v<T>();
    su[r][q] = (r < K && q < N) ? Ub[(int64_t)r * U.ld + q] : zero_v<T>();
  }
  __syncthreads();
  const int j = t & 31, r0 = (t >> 5) * 4;  // column j, rows r0 .. r0 + 3
  if (j >= N) return;
  T acc[4] = {zero_v<T>(), zero_v<T>(), zero_v<T>(), zero_v<T>()};
  for (int k = 0; k < K; ++k) {
    const T u = su[k][j];
#pragma unroll
    for (int q = 0; q < 4; ++q) mac(acc[q], sl[r0 + q][k], u);
  }
  T* Db = D.at(b);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = i0 + r0 + q;
    if (i < M) {
      T* d = Db + (int64_t)i * D.ld + j;
      *d = add_(*d, neg_(acc[q]));
    }
  }
}

// ------------------------------------------------------------------ mirror
// Completes a symmetric (CONJ = false) or Hermitian (CONJ = true) matrix whose
// 64 x 64 tiles on and below the diagonal are computed: A[i][j] = op(A[j][i])
// for every (i, j) whose 64-tile column is right of its 64-tile row, through
// a 32 x 32 shared-memory transpose (grid: 32-tiles x 32-tiles x batch, 32 x 8
// threads).
template <typename T, bool CONJ>
__global__ void __launch_bounds__(256) mirror_kernel(int n, MatB<T> A) {
  __shared__ T tile[32][33];
  const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
  if ((j0 >> 6) <= (i0 >> 6)) return;  // on or below the diagonal tiles: computed
  T* a = A.at(blockIdx.z);
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  // source rows j0.., columns i0.. (coalesced along i)
  for (int r = ty; r < 32; r += 8) {
    const int j = j0 + r, i = i0 + tx;
    if (j < n && i < n) tile[r][tx] = a[(int64_t)j * A.ld + i];
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int i = i0 + r, j = j0 + tx;
    if (i < n && j < n) a[(int64_t)i * A.ld + j] = CONJ ? conj_(tile[tx][r]) : tile[tx][r];
  }
}

// ------------------------------------------------------------------ TRSM step
// Block row kb (rows [kb*64, kb*64+64)) of op(T) X = B for one 64-column tile
// of X per CTA (grid: column tiles x batch).
//   LOWER: op(T) is lower triangular -> uses the finished block rows j < kb
//          (forward substitution); else upper -> j > kb (backward).
//   UNIT:  unit diagonal (the L of an LU factorisation).
//   RHS_I: B = I restricted to the tile; tiles right of the diagonal block
//          are zero and are written as such (the inverse of a lower
//          triangular matrix is lower triangular), and the sum skips the
//          block rows j < column tile where X is zero.
//   rowperm (optional): B row r is read from row rowperm[r] (B := P B).
// X may alias B when rowperm is NULL.
template <typename T> struct SmemTrsm {
  union {
    SmemAB<T> ab;
    T d[TB][TB + 1];
  } u;
  T w[TB][TB + 1];
  T dinv[TB];
};

// Substitution with the 64 x 64 triangular block sm.u.d (its reciprocal
// diagonal in sm.dinv) on the 64 right-hand sides in sm.w, in place,
// column-oriented: the 4 lanes of a column (consecutive lanes of one warp)
// hold its rows l = part + 4 i in registers; step rr finishes x_rr (its owner
// lane scales by 1 / d_rr), passes it to the other three by a shuffle, and
// every lane removes d[l][rr] x_rr from its unfinished rows with independent
// FMAs.  Ends with a __syncthreads.
template <typename T, bool LOWER>
__device__ __forceinline__ void subst64(SmemTrsm<T>& sm, int t) {
  {
    const int col = t >> 2, part = t & 3;
    const unsigned mask = 0xffffffffu;
    const int src = (threadIdx.x & 31) & ~3;
    T wr[TB / 4];
#pragma unroll
    for (int i = 0; i < TB / 4; ++i) wr[i] = sm.w[part + 4 * i][col];
#pragma unroll
    for (int s = 0; s < TB; ++s) {
      const int rr = LOWER ? s : (TB - 1 - s);
      T x = zero_v<T>();
      if (part == (rr & 3)) {
        wr[rr >> 2] = mul_(wr[rr >> 2], sm.dinv[rr]);
        x = wr[rr >> 2];
      }
      x = shfl_(mask, x, src | (rr & 3));
      const T nx = neg_(x);
#pragma unroll
      for (int i = 0; i < TB / 4; ++i) {
        const int l = part + 4 * i;
        if (LOWER ? (l > rr) : (l < rr)) mac(wr[i], sm.u.d[l][rr], nx);
      }
    }
#pragma unroll
    for (int i = 0; i < TB / 4; ++i) sm.w[part + 4 * i][col] = wr[i];
  }
  __syncthreads();
}

template <typename T, int OPT, bool LOWER, bool UNIT, bool RHS_I>
__global__ void __launch_bounds__(NTH) trsm_step_kernel(int n, int nrhs, int kb, MatB<const T> Tm, MatB<const T> Bm,
                                                        MatB<T> X, const int* rowperm) {
  const int b = blockIdx.z;
  const int ct = blockIdx.x;
  const int c0 = ct * TB;
  const int r0 = kb * TB;
  const int t = threadIdx.x;
  const int tx = t & 15, ty = t >> 4;
  extern __shared__ __align__(16) unsigned char smraw[];
  SmemTrsm<T>& sm = *reinterpret_cast<SmemTrsm<T>*>(smraw);
  T* Xb = X.at(b);
  const T* Tb = Tm.at(b);

  if (RHS_I && LOWER && ct > kb) {
    for (int e = t; e < TB * TB; e += NTH) {
      int r = r0 + e / TB, c = c0 + e % TB;
      if (r < n && c < nrhs) Xb[(int64_t)r * X.ld + c] = zero_v<T>();
    }
    return;
  }

  T acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = zero_v<T>();

  // acc = sum_j op(T)[r0.., j] X[j, c0..]  over the finished rows
  {
    int kbeg, kend;
    if (LOWER) { kbeg = RHS_I ? c0 : 0; kend = r0; }
    else { kbeg = r0 + TB; kend = n; }
    if (kbeg < kend) {
      // op(T) restricted to rows [r0, r0+64): pass the row offset through the pointer
      const T* Tp;
      if (OPT == OP_N) Tp = Tb + (int64_t)r0 * Tm.ld; else Tp = Tb + r0;
      mainloop<T, OPT, OP_N>(acc, sm.u.ab, Tp, Tm.ld, Xb, X.ld, n - r0, nrhs, 0, c0, kbeg, kend);
    }
  }
  __syncthreads();
  // w = B_tile - acc
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      int rl = 4 * ty + r, cl = 4 * tx + c;
      int gr = r0 + rl, gc = c0 + cl;
      T bv = zero_v<T>();
      if (gr < n && gc < nrhs) {
        if (RHS_I) bv = (gr == gc) ? one_v<T>() : zero_v<T>();
        else {
          int sr = rowperm ? rowperm[(int64_t)b * n + gr] : gr;
          bv = Bm.at(b)[(int64_t)sr * Bm.ld + gc];
        }
      }
      sm.w[rl][cl] = sub_(bv, acc[r][c]);
    }
  // diagonal block op(T)[r0.., r0..], masked to its triangle; padding rows
  // beyond n act as identity rows
  for (int e = t; e < TB * TB; e += NTH) {
    int rl = e / TB, cl = e % TB;
    int gr = r0 + rl, gc = r0 + cl;
    T v = zero_v<T>();
    bool in_tri = LOWER ? (cl <= rl) : (cl >= rl);
    if (gr < n && gc < n && in_tri) {
      if (OPT == OP_N) v = Tb[(int64_t)gr * Tm.ld + gc];
      else {
        v = Tb[(int64_t)gc * Tm.ld + gr];
        if (OPT == OP_C) v = conj_(v);
      }
    }
    if (rl == cl && (UNIT || gr >= n)) v = one_v<T>();
    sm.u.d[rl][cl] = v;
  }
  __syncthreads();
  if (t < TB) sm.dinv[t] = UNIT ? one_v<T>() : recip_(sm.u.d[t][t]);
  __syncthreads();
  subst64<T, LOWER>(sm, t);
  for (int e = t; e < TB * TB; e += NTH) {
    int rl = e / TB, cl = e % TB;
    int gr = r0 + rl, gc = c0 + cl;
    if (gr < n && gc < nrhs) Xb[(int64_t)gr * X.ld + gc] = sm.w[rl][cl];
  }
}

// Diagonal blocks of the inverse of a lower triangular L (unit diagonal if
// UNIT): X[kb][kb] = L[kb][kb]^{-1} for block row kb = blockIdx.x, and the
// tiles right of it in block row kb set to zero (grid: blocks x batch).
template <typename T, bool UNIT>
__global__ void __launch_bounds__(NTH) trtri_diag_kernel(int n, MatB<const T> Lm, MatB<T> X) {
  const int b = blockIdx.z;
  const int kb = blockIdx.x;
  const int r0 = kb * TB;
  const int t = threadIdx.x;
  extern __shared__ __align__(16) unsigned char smraw[];
  SmemTrsm<T>& sm = *reinterpret_cast<SmemTrsm<T>*>(smraw);
  T* Xb = X.at(b);
  const T* Lb = Lm.at(b);
  for (int e = t; e < TB * TB; e += NTH) {
    const int rl = e / TB, cl = e % TB;
    const int gr = r0 + rl, gc = r0 + cl;
    T v = zero_v<T>();
    if (gr < n && gc < n && cl <= rl) v = Lb[(int64_t)gr * Lm.ld + gc];
    if (rl == cl && (UNIT || gr >= n)) v = one_v<T>();
    sm.u.d[rl][cl] = v;
    sm.w[rl][cl] = rl == cl ? one_v<T>() : zero_v<T>();
  }
  __syncthreads();
  if (t < TB) sm.dinv[t] = UNIT ? one_v<T>() : recip_(sm.u.d[t][t]);
  __syncthreads();
  subst64<T, true>(sm, t);
  for (int e = t; e < TB * TB; e += NTH) {
    const int rl = e / TB, cl = e % TB;
    const int gr = r0 + rl, gc = r0 + cl;
    if (gr < n && gc < n) Xb[(int64_t)gr * X.ld + gc] = sm.w[rl][cl];
  }
  for (int e = t; e < TB * (n - r0 - TB); e += NTH) {  // right of the diagonal block
    const int rl = e / (n - r0 - TB), c = r0 + TB + e % (n - r0 - TB);
    if (r0 + rl < n) Xb[(int64_t)(r0 + rl) * X.ld + c] = zero_v<T>();
  }
}

// ------------------------------------------------------------------ panels
// Pivot key: |x| for reals, |re|^2 + |im|^2 for complex numbers (both give
// the entry of largest modulus).
__device__ __forceinline__ double pkey(double a) { return fabs(a); }
__device__ __forceinline__ float pkey(float a) { return fabsf(a); }
__device__ __forceinline__ double pkey(zd a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ float pkey(zf a) { return a.x * a.x + a.y * a.y; }

template <typename K> struct KeyIdx {
  K key;
  int idx;
};

// larger key wins; equal keys -> lower index; NaN keys never win
template <typename K> __device__ __forceinline__ KeyIdx<K> kmax(KeyIdx<K> a, KeyIdx<K> b) {
  if (b.key > a.key || (b.key == a.key && b.idx < a.idx)) return b;
  return a;
}

constexpr int PANEL_THREADS = 512;

// LU with partial pivoting of the column panel [k0, k0+kb) over rows [k0, n)
// of each matrix (grid: batch).  The panel is staged in shared memory when
// `staged` (rows * (kb + 1) * sizeof(T) fits), else factored in place in
// global memory.  piv[k] (absolute row, batch stride n) receives the row exchanged
// with row k.  A zero or non-finite pivot reports FROB_ERR_SINGULAR with
// bad_index = k + 1 + info_off and leaves that column unscaled.
template <typename T>
__global__ void __launch_bounds__(PANEL_THREADS) getrf_panel_kernel(int n, int k0, int kb, MatB<T> A, int* piv,
                                                                     frob_info* info, int info_off, int staged) {
  using K = typename real_of<T>::type;
  const int b = blockIdx.x;
  const int t = threadIdx.x;
  const int m = n - k0;
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ KeyIdx<K> red[PANEL_THREADS / 32];
  __shared__ int s_p;
  __shared__ T s_rinv;
  __shared__ int s_ok;
  T* g = A.at(b) + (int64_t)k0 * A.ld + k0;
  T* P;
  int64_t ps;
  if (staged) {
    // row stride kb + 1: a warp reading one column touches 32 different banks
    P = reinterpret_cast<T*>(smraw);
    ps = kb + 1;
    for (int e = t; e < m * kb; e += PANEL_THREADS) P[(e / kb) * ps + (e % kb)] = g[(int64_t)(e / kb) * A.ld + (e % kb)];
    __syncthreads();
  } else {
    P = g;
    ps = A.ld;
  }
  for (int j = 0; j < kb; ++j) {
    // argmax over rows [j, m) of column j
    KeyIdx<K> best{(K)-1, 0x7fffffff};
    bool bad = false;
    for (int r = j + t; r < m; r += PANEL_THREADS) {
      K kv = pkey(P[(int64_t)r * ps + j]);
      if (!(kv == kv) || kv == (K)INFINITY) bad = true;
      best = kmax(best, KeyIdx<K>{kv, r});
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      KeyIdx<K> other{__shfl_xor_sync(0xffffffffu, best.key, o), __shfl_xor_sync(0xffffffffu, best.idx, o)};
      best = kmax(best, other);
    }
    bad = __syncthreads_or(bad);
    if ((t & 31) == 0) red[t >> 5] = best;
    __syncthreads();
    if (t == 0) {
      KeyIdx<K> bb = red[0];
      for (int w = 1; w < PANEL_THREADS / 32; ++w) bb = kmax(bb, red[w]);
      int p = (bb.idx == 0x7fffffff) ? j : bb.idx;
      s_p = p;
      piv[(int64_t)b * n + k0 + j] = k0 + p;
      T pv = P[(int64_t)p * ps + j];
      bool ok = !bad && bb.key > (K)0;
      s_ok = ok;
      if (!ok) report(info, b, FROB_ERR_SINGULAR, info_off + k0 + j + 1);
      s_rinv = ok ? recip_(pv) : one_v<T>();
    }
    __syncthreads();
    const int p = s_p;
    if (p != j)
      for (int c = t; c < kb; c += PANEL_THREADS) {
        T x = P[(int64_t)j * ps + c];
        P[(int64_t)j * ps + c] = P[(int64_t)p * ps + c];
        P[(int64_t)p * ps + c] = x;
      }
    __syncthreads();
    if (s_ok) {
      const T rinv = s_rinv;
      for (int r = j + 1 + t; r < m; r += PANEL_THREADS) P[(int64_t)r * ps + j] = mul_(P[(int64_t)r * ps + j], rinv);
    }
    __syncthreads();
    // rank-1 update of the rest of the panel
    for (int r = j + 1 + t; r < m; r += PANEL_THREADS) {
      T l = neg_(P[(int64_t)r * ps + j]);
      T* row = P + (int64_t)r * ps;
      const T* prow = P + (int64_t)j * ps;
      for (int c = j + 1; c < kb; ++c) mac(row[c], l, prow[c]);
    }
    __syncthreads();
  }
  if (staged) {
    for (int e = t; e < m * kb; e += PANEL_THREADS) g[(int64_t)(e / kb) * A.ld + (e % kb)] = P[(e / kb) * ps + (e % kb)];
  }
}

// Row swaps of the panel [k0, k0+kb) applied to the columns outside it, and
// U12 = L11^{-1} A12 for the columns right of it (grid: column strips of 64
// x batch).  Strip s covers columns [64 s, 64 s + 64) of the matrix; columns
// inside the panel are skipped.
constexpr int PANEL_MAX = 32;  // widest column panel of the blocked LU / Cholesky

// As getrf_panel_kernel for panels of at most PANEL_THREADS rows (n - k0 <=
// 512) and scalars of at most 8 bytes: thread r keeps row r of the panel in
// registers; the pivot search reads column j from registers, the two rows of
// a swap pass through shared memory, and the rank-1 update of the panel is
// independent FMAs with the pivot row broadcast from shared memory.
// Same results and reports as getrf_panel_kernel.
template <typename T>
__global__ void __launch_bounds__(PANEL_THREADS) getrf_panel_reg_kernel(int n, int k0, int kb, MatB<T> A, int* piv,
                                                                         frob_info* info, int info_off) {
  using K = typename real_of<T>::type;
  const int b = blockIdx.x;
  const int t = threadIdx.x;
  const int m = n - k0;
  __shared__ KeyIdx<K> red[PANEL_THREADS / 32];
  __shared__ T prow[PANEL_MAX];
  __shared__ T jrow[PANEL_MAX];
  __shared__ int s_p;
  __shared__ T s_rinv;
  __shared__ int s_ok;
  T* g = A.at(b) + (int64_t)k0 * A.ld + k0;
  const bool mine = t < m;
  T r[PANEL_MAX];
#pragma unroll
  for (int c = 0; c < PANEL_MAX; ++c) r[c] = (mine && c < kb) ? g[(int64_t)t * A.ld + c] : zero_v<T>();
#pragma unroll
  for (int j = 0; j < PANEL_MAX; ++j) {
    if (j < kb) {
      // argmax over rows [j, m) of column j
      const bool cand = mine && t >= j;
      const K kv = cand ? pkey(r[j]) : (K)-1;
      bool bad = cand && (!(kv == kv) || kv == (K)INFINITY);
      KeyIdx<K> best{kv, cand ? t : 0x7fffffff};
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        KeyIdx<K> other{__shfl_xor_sync(0xffffffffu, best.key, o), __shfl_xor_sync(0xffffffffu, best.idx, o)};
        best = kmax(best, other);
      }
      bad = __syncthreads_or(bad);
      if ((t & 31) == 0) red[t >> 5] = best;
      __syncthreads();
      KeyIdx<K> bb = red[0];
      if (t == 0) {
        for (int w = 1; w < PANEL_THREADS / 32; ++w) bb = kmax(bb, red[w]);
        const int p = (bb.idx == 0x7fffffff) ? j : bb.idx;
        s_p = p;
        piv[(int64_t)b * n + k0 + j] = k0 + p;
      }
      __syncthreads();
      const int p = s_p;
      // swap rows j and p through shared memory
      if (t == p)
#pragma unroll
        for (int c = 0; c < PANEL_MAX; ++c) prow[c] = r[c];
      if (t == j && p != j)
#pragma unroll
        for (int c = 0; c < PANEL_MAX; ++c) jrow[c] = r[c];
      __syncthreads();
      if (t == j && p != j)
#pragma unroll
        for (int c = 0; c < PANEL_MAX; ++c) r[c] = prow[c];
      if (t == p && p != j)
#pragma unroll
        for (int c = 0; c < PANEL_MAX; ++c) r[c] = jrow[c];
      if (t == 0) {
        const T pv = prow[j];
        const bool ok = !bad && bb.key > (K)0;
        s_ok = ok;
        if (!ok) report(info, b, FROB_ERR_SINGULAR, info_off + k0 + j + 1);
        s_rinv = ok ? recip_(pv) : one_v<T>();
      }
      __syncthreads();
      if (mine && t > j) {
        if (s_ok) r[j] = mul_(r[j], s_rinv);
        const T l = neg_(r[j]);
#pragma unroll
        for (int c = j + 1; c < PANEL_MAX; ++c)
          if (c < kb) mac(r[c], l, prow[c]);
      }
      __syncthreads();  // prow / jrow are rewritten by the next column
    }
  }
  if (mine)
#pragma unroll
    for (int c = 0; c < PANEL_MAX; ++c)
      if (c < kb) g[(int64_t)t * A.ld + c] = r[c];
}


template <typename T> constexpr size_t laswp_trsm_smem() {
  return sizeof(T) * (size_t)(PANEL_MAX * (PANEL_MAX + 1) + PANEL_MAX * (TB + 1));
}

// u_end: U12 is formed for the columns [k0 + kb, u_end) only (n for the
// whole row; a recursive LU's block passes its right edge); the swaps reach
// every column outside the panel.
template <typename T>
__global__ void __launch_bounds__(NTH) laswp_trsm_kernel(int n, int k0, int kb, MatB<T> A, const int* piv,
                                                         int u_end) {
  const int b = blockIdx.z;
  const int t = threadIdx.x;
  const int c0 = blockIdx.x * TB;
  T* Ab = A.at(b);
  extern __shared__ __align__(16) unsigned char smraw[];
  T* l11 = reinterpret_cast<T*>(smraw);              // [kb][PANEL_MAX + 1]
  T* u = l11 + PANEL_MAX * (PANEL_MAX + 1);          // [kb][TB + 1]
  constexpr int LS = PANEL_MAX + 1, US = TB + 1;
  const int c = c0 + (t & 63);
  const bool col_ok = c < n && (c < k0 || c >= k0 + kb);
  // swaps, in order
  if (t < TB && col_ok) {
    for (int j = 0; j < kb; ++j) {
      int p = piv[(int64_t)b * n + k0 + j];
      if (p != k0 + j) {
        T x = Ab[(int64_t)(k0 + j) * A.ld + c];
        Ab[(int64_t)(k0 + j) * A.ld + c] = Ab[(int64_t)p * A.ld + c];
        Ab[(int64_t)p * A.ld + c] = x;
      }
    }
  }
  if (c0 + TB <= k0 + kb || c0 >= u_end) return;  // strip left of / inside the panel, or right of the block
  __syncthreads();
  for (int e = t; e < kb * kb; e += NTH) {
    int r = e / kb, q = e % kb;
    l11[r * LS + q] = Ab[(int64_t)(k0 + r) * A.ld + k0 + q];
  }
  for (int e = t; e < kb * TB; e += NTH) {
    int r = e / TB, q = e % TB;
    int cc = c0 + q;
    u[r * US + q] = (cc < u_end && cc >= k0 + kb) ? Ab[(int64_t)(k0 + r) * A.ld + cc] : zero_v<T>();
  }
  __syncthreads();
  // forward substitution with the unit lower triangle L11, one column per thread
  if (t < TB) {
    for (int r = 1; r < kb; ++r) {
      T s = u[r * US + t];
      for (int q = 0; q < r; ++q) mac(s, neg_(l11[r * LS + q]), u[q * US + t]);
      u[r * US + t] = s;
    }
  }
  __syncthreads();
  for (int e = t; e < kb * TB; e += NTH) {
    int r = e / TB, q = e % TB;
    int cc = c0 + q;
    if (cc < u_end && cc >= k0 + kb) Ab[(int64_t)(k0 + r) * A.ld + cc] = u[r * US + q];
  }
}

// Cholesky of the kb x kb diagonal block at g (lower, A11 = L11 L11^H) by one
// warp: lane r keeps row r in registers; step j broadcasts column j through
// colj (shared memory) and every lane applies its rank-1 update with
// independent FMAs.  Lane r returns row r of L11 in r[] (zeros above the
// diagonal); the first non-positive or non-finite pivot is returned in *fail
// (-1 if none; that pivot is replaced by 1).
template <typename T>
__device__ __forceinline__ void chol32_warp(const T* g, int64_t ld, int kb, T* colj, T (&r)[PANEL_MAX], int* fail) {
  using K = typename real_of<T>::type;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int c = 0; c < PANEL_MAX; ++c) r[c] = (lane < kb && c <= lane) ? g[(int64_t)lane * ld + c] : zero_v<T>();
  int f = -1;
#pragma unroll
  for (int j = 0; j < PANEL_MAX; ++j) {
    if (j < kb) {
      colj[lane] = r[j];
      __syncwarp();
      const K d = real_(colj[j]);
      const bool ok = d > (K)0 && d < (K)INFINITY;
      if (!ok && f < 0) f = j;
      const K l = ok ? sqrt(d) : (K)1;
      __syncwarp();
      if (lane == j) r[j] = from_real<T>(l);
      if (lane > j) r[j] = mul_(r[j], from_real<T>((K)1 / l));  // L[lane][j]
      colj[lane] = r[j];
      __syncwarp();
      const T lij = neg_(r[j]);
#pragma unroll
      for (int c = j + 1; c < PANEL_MAX; ++c)
        if (c <= lane) mac(r[c], lij, conj_(colj[c]));
      __syncwarp();
    }
  }
  *fail = f;
}

// One step of the blocked Cholesky: the panel [k0, k0 + kb).  Every CTA
// factors the diagonal block itself (warp 0, in registers; CTA 0 writes it
// back and reports a non-positive or non-finite pivot as FROB_ERR_NOT_HPD with
// bad_index = k + 1 + info_off, continuing with a unit pivot), then solves
// its rows below it, L21 = A21 L11^{-H}, one thread per row: x L11^H = a.
// Grid: row blocks of 128 (at least one) x batch.
template <typename T>
__global__ void __launch_bounds__(128) potrf_panel_kernel(int n, int k0, int kb, MatB<T> A, frob_info* info,
                                                          int info_off) {
  using K = typename real_of<T>::type;
  const int b = blockIdx.y;
  __shared__ T L[PANEL_MAX][PANEL_MAX + 1];
  __shared__ K dinv[PANEL_MAX];
  __shared__ T colj[PANEL_MAX];
  T* Ab = A.at(b);
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    T r[PANEL_MAX];
    int fail;
    T* g = Ab + (int64_t)k0 * A.ld + k0;
    chol32_warp<T>(g, A.ld, kb, colj, r, &fail);
#pragma unroll
    for (int c = 0; c < PANEL_MAX; ++c) L[lane][c] = r[c];
    if (lane < kb) dinv[lane] = (K)1 / real_(r[lane]);
    if (blockIdx.x == 0) {
      if (fail >= 0 && lane == 0) report(info, b, FROB_ERR_NOT_HPD, info_off + k0 + fail + 1);
      if (lane < kb)
#pragma unroll
        for (int c = 0; c < PANEL_MAX; ++c)
          if (c <= lane) g[(int64_t)lane * A.ld + c] = r[c];
    }
  }
  __syncthreads();
  const int row = k0 + kb + blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= n) return;
  T* a = Ab + (int64_t)row * A.ld + k0;
  T x[PANEL_MAX];
#pragma unroll
  for (int j = 0; j < PANEL_MAX; ++j) x[j] = j < kb ? a[j] : zero_v<T>();
#pragma unroll
  for (int j = 0; j < PANEL_MAX; ++j) {
    if (j < kb) {
      T s = x[j];
#pragma unroll
      for (int i = 0; i < j; ++i) mac(s, neg_(x[i]), conj_(L[j][i]));
      x[j] = mul_(s, from_real<T>(dinv[j]));
    }
  }
#pragma unroll
  for (int j = 0; j < PANEL_MAX; ++j)
    if (j < kb) a[j] = x[j];
}

// Whole-matrix Cholesky (lower, A = L L^T, in place) of a real FP32 matrix
// with n <= SCHOL_MAX by one CTA of SCHOL_THREADS threads, for the batched
// sizes where one CTA per matrix is enough work: it replaces the 2 n / 32
// launches of the blocked form.  Per 32-wide panel [k0, k0 + 32):
//   1. the panel's rows k0 .. n - 1 are copied into shared memory (P, row
//      pitch 33; 16-byte loads, eight lanes per 128-byte row, when the rows
//      are 16-byte aligned);
//   2. warp 0 factors the diagonal block from P in registers (chol32_warp);
//      a non-positive or non-finite pivot is reported as in
//      potrf_panel_kernel, with a unit pivot in its place;
//   3. thread t solves row 32 + t of P, x L11^T = a, column by column
//      (independent FMAs), and also keeps it transposed in Lt;
//   4. P goes back to global memory (the diagonal block's lower triangle
//      and the rows below it), and the 16 warps update the lower 32 x 32
//      tiles of the trailing matrix, A22 -= L21 L21^T: lane (ty, tx) of a
//      warp holds rows 4 ty .. 4 ty + 3 and columns 4 tx .. 4 tx + 3 and
//      16 + 4 tx .. 16 + 4 tx + 3 of its tile in registers, read from Lt as
//      broadcast float4s, so that each row's 8 entries are two 16-byte
//      chunks contiguous across the lanes in global memory.
// Entries above the diagonal are not written.  Grid: batch.
constexpr int SCHOL_MAX = 512;
constexpr int SCHOL_THREADS = 512;
constexpr int SCHOL_PP = PANEL_MAX + 1;        // row pitch of P
constexpr int SCHOL_LTP = SCHOL_MAX - 32 + 4;  // row pitch of Lt (rows below the first panel)
constexpr int SCHOL_SMEM = (PANEL_MAX * SCHOL_LTP + SCHOL_MAX * SCHOL_PP + 2 * PANEL_MAX) * 4;

template <typename T>  // float
__global__ void __launch_bounds__(SCHOL_THREADS, 1) potrf_small_kernel(int n, MatB<T> A, frob_info* info,
                                                                       int info_off) {
  static_assert(sizeof(T) == 4 && T(0.5f) == 0.5f, "real FP32 only");
  extern __shared__ float4 schol_raw[];
  float* Lt = reinterpret_cast<float*>(schol_raw);  // Lt[c * SCHOL_LTP + r] = L[k0 + 32 + r][k0 + c]
  float* P = Lt + PANEL_MAX * SCHOL_LTP;            // P[r * SCHOL_PP + c] = A[k0 + r][k0 + c]
  float* dinv = P + SCHOL_MAX * SCHOL_PP;
  float* colj = dinv + PANEL_MAX;
  const int b = blockIdx.x;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  float* Ab = A.at(b);
  const int64_t ld = A.ld;
  const bool vec = (ld & 3) == 0 && (reinterpret_cast<uintptr_t>(Ab) & 15) == 0;
  for (int k0 = 0; k0 < n; k0 += PANEL_MAX) {
    const int kb = n - k0 < PANEL_MAX ? n - k0 : PANEL_MAX;
    const int r0 = k0 + kb;
    const int m = n - r0;  // rows below the panel (kb = 32 whenever m > 0)
    const int pr = n - k0;  // rows of P
    // 1. panel -> P
    if (vec && kb == PANEL_MAX) {
      for (int e = t; e < pr * 8; e += SCHOL_THREADS) {
        const int r = e >> 3, q = e & 7;
        const float4 v = *reinterpret_cast<const float4*>(Ab + (int64_t)(k0 + r) * ld + k0 + 4 * q);
        float* d = P + r * SCHOL_PP + 4 * q;
        d[0] = v.x;
        d[1] = v.y;
        d[2] = v.z;
        d[3] = v.w;
      }
    } else {
      for (int e = t; e < pr * PANEL_MAX; e += SCHOL_THREADS) {
        const int r = e >> 5, c = e & 31;
        P[r * SCHOL_PP + c] = c < kb ? Ab[(int64_t)(k0 + r) * ld + k0 + c] : 0.f;
      }
    }
    __syncthreads();
    // 2. diagonal block
    if (warp == 0) {
      float rr[PANEL_MAX];
      int fail;
      chol32_warp<float>(P, SCHOL_PP, kb, colj, rr, &fail);
      if (fail >= 0 && lane == 0) report(info, b, FROB_ERR_NOT_HPD, info_off + k0 + fail + 1);
#pragma unroll
      for (int c = 0; c < PANEL_MAX; ++c) P[lane * SCHOL_PP + c] = rr[c];
      if (lane < kb) dinv[lane] = 1.f / rr[lane];
    }
    __syncthreads();
    // 3. rows below it
    if (t < m) {
      float x[PANEL_MAX];
      float* pr_t = P + (PANEL_MAX + t) * SCHOL_PP;
#pragma unroll
      for (int j = 0; j < PANEL_MAX; ++j) x[j] = pr_t[j];
#pragma unroll
      for (int j = 0; j < PANEL_MAX; ++j) {
        x[j] *= dinv[j];
#pragma unroll
        for (int i = j + 1; i < PANEL_MAX; ++i) x[i] = fmaf(-x[j], P[i * SCHOL_PP + j], x[i]);
      }
#pragma unroll
      for (int j = 0; j < PANEL_MAX; ++j) {
        pr_t[j] = x[j];
        Lt[j * SCHOL_LTP + t] = x[j];
      }
    }
    __syncthreads();
    // 4. P -> panel (lower triangle of the diagonal block, full rows below)
    if (vec && kb == PANEL_MAX) {
      for (int e = t; e < pr * 8; e += SCHOL_THREADS) {
        const int r = e >> 3, q = e & 7;
        const float* sp = P + r * SCHOL_PP + 4 * q;
        float* g = Ab + (int64_t)(k0 + r) * ld + k0 + 4 * q;
        if (r >= PANEL_MAX || 4 * q + 3 <= r) {
          *reinterpret_cast<float4*>(g) = make_float4(sp[0], sp[1], sp[2], sp[3]);
        } else {
#pragma unroll
          for (int c = 0; c < 4; ++c)
            if (4 * q + c <= r) g[c] = sp[c];
        }
      }
    } else {
      for (int e = t; e < pr * PANEL_MAX; e += SCHOL_THREADS) {
        const int r = e >> 5, c = e & 31;
        if (c < kb && (r >= PANEL_MAX || c <= r)) Ab[(int64_t)(k0 + r) * ld + k0 + c] = P[r * SCHOL_PP + c];
      }
    }
    if (m <= 0) break;
    const int mt = (m + 31) >> 5;
    const int ntile = mt * (mt + 1) / 2;
    const int ty = lane >> 2, tx = lane & 3;
    for (int tile = warp; tile < ntile; tile += SCHOL_THREADS / 32) {
      int I = 0;
      while ((I + 1) * (I + 2) / 2 <= tile) ++I;  // tile = I (I + 1) / 2 + J, J <= I
      const int J = tile - I * (I + 1) / 2;
      const int rb = 32 * I + 4 * ty, cb = 32 * J + 4 * tx;  // columns cb .. cb + 3, cb + 16 .. cb + 19
      float acc[4][8];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
#pragma unroll 8
      for (int c = 0; c < PANEL_MAX; ++c) {
        const float4 rv = *reinterpret_cast<const float4*>(Lt + c * SCHOL_LTP + rb);
        const float4 c0 = *reinterpret_cast<const float4*>(Lt + c * SCHOL_LTP + cb);
        const float4 c1 = *reinterpret_cast<const float4*>(Lt + c * SCHOL_LTP + cb + 16);
        const float ra[4] = {rv.x, rv.y, rv.z, rv.w};
        const float ca[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(ra[i], ca[j], acc[i][j]);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int row = rb + i;
        if (row >= m) continue;
        float* dst = Ab + (int64_t)(r0 + row) * ld + r0;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int col = cb + 16 * h;
          if (vec && col + 3 <= row) {  // all four in range and on or below the diagonal
            float4 v = *reinterpret_cast<const float4*>(dst + col);
            v.x -= acc[i][4 * h];
            v.y -= acc[i][4 * h + 1];
            v.z -= acc[i][4 * h + 2];
            v.w -= acc[i][4 * h + 3];
            *reinterpret_cast<float4*>(dst + col) = v;
          } else {
#pragma unroll
            for (int j = 0; j < 4; ++j)
              if (col + j <= row) dst[col + j] -= acc[i][4 * h + j];
          }
        }
      }
    }
    __syncthreads();
  }
}

// Whole-matrix LU with partial pivoting (A = P^T L U, in place, L unit lower,
// LAPACK-style swap list piv) of a real FP32 matrix with n <= SLU_MAX by one
// CTA of SLU_THREADS threads.  Rows are not moved in global memory while the
// factorization runs: perm[i] is the global row that holds logical row i, and
// the rows are gathered into logical order once at the end.  Per 32-wide
// panel [k0, k0 + 32):
//   1. the panel's logical rows k0 .. n - 1 are copied into shared memory P
//      (row r of P = logical row k0 + r at the start of the panel);
//   2. column by column, with one CTA barrier per column: thread t keeps
//      logical row k0 + t in registers.  The pivot is the entry of largest
//      modulus (ties to the lower row, NaN never chosen), found by an
//      integer maximum of the keys (bit pattern of |x| plus one, 0 for rows
//      above the column and for NaN) and a ballot, within each warp and
//      then over the 16 warp results; each warp's leading row is written to
//      shared memory before the barrier, so that after it the pivot row is
//      there for every row below it, which scales its multiplier and
//      updates the rest of its panel row.  A zero, NaN or infinite pivot column is reported as
//      FROB_ERR_SINGULAR (bad_index = its 1-based index + info_off) and the
//      elimination continues unscaled, as in getrf_panel_reg_kernel;
//   3. the panel goes back to global memory through P, L21 is kept
//      transposed in Lt, and thread t forms column r0 + t of
//      U12 = L11^{-1} A12 (kept in Ut, then written row by row);
//   4. the 16 warps update the trailing matrix, A22 -= L21 U12, in 32 x 16
//      tiles, each lane a 4 x 4 block in registers from broadcast float4
//      reads of Lt and Ut (the block's old values are loaded before its
//      FMAs).
// Grid: batch.
constexpr int SLU_MAX = 512;
constexpr int SLU_THREADS = 512;
constexpr int SLU_PP = PANEL_MAX + 1;       // row pitch of P
constexpr int SLU_TP = SLU_MAX - 32 + 4;    // row pitch of Lt and Ut
constexpr int SLU_GW = 64;                  // columns per round of the final gather
constexpr int SLU_GP = SLU_GW + 4;          // its row pitch
constexpr int SLU_FLOATS = 2 * PANEL_MAX * SLU_TP + SLU_MAX * SLU_PP + 2 * 16 * PANEL_MAX + 2 * PANEL_MAX;  // Lt, Ut, P, rows
constexpr int SLU_INTS = SLU_MAX + 3 * 2 * 16;  // perm, redk, redi, redb
constexpr int SLU_SMEM = (SLU_FLOATS + SLU_INTS) * 4;
static_assert(SLU_MAX * SLU_GP <= 2 * PANEL_MAX * SLU_TP + SLU_MAX * SLU_PP, "gather buffer (Lt, Ut and P)");
static_assert(SLU_SMEM <= 232448, "shared memory per CTA");

template <typename T>  // float
__global__ void __launch_bounds__(SLU_THREADS, 1) getrf_small_kernel(int n, MatB<T> A, int* piv, frob_info* info,
                                                                     int info_off) {
  static_assert(sizeof(T) == 4 && T(0.5f) == 0.5f, "real FP32 only");
  extern __shared__ float4 slu_raw[];
  float* Lt = reinterpret_cast<float*>(slu_raw);  // Lt[c * SLU_TP + i] = L[r0 + i][k0 + c] (logical rows)
  float* Ut = Lt + PANEL_MAX * SLU_TP;             // Ut[c * SLU_TP + j] = U[k0 + c][r0 + j]
  float* P = Ut + PANEL_MAX * SLU_TP;              // P[r * SLU_PP + c]: the panel
  float* G = Lt;                                   // final gather: [SLU_MAX][SLU_GP] over Lt, Ut and P
  float* cand_rows = P + SLU_MAX * SLU_PP;         // [2][16][PANEL_MAX] each warp's leading candidate row
  float* jrow = cand_rows + 2 * 16 * PANEL_MAX;    // [2][PANEL_MAX] row j
  int* perm = reinterpret_cast<int*>(jrow + 2 * PANEL_MAX);
  unsigned* redk = reinterpret_cast<unsigned*>(perm + SLU_MAX);  // [2][16] warp maxima of the keys
  int* redi = reinterpret_cast<int*>(redk + 32);                 // [2][16] their rows (panel-relative)
  int* redb = redi + 32;                                         // [2][16] NaN / infinity seen
  static_assert(SLU_FLOATS == 2 * PANEL_MAX * SLU_TP + SLU_MAX * SLU_PP + 2 * 16 * PANEL_MAX + 2 * PANEL_MAX &&
                    SLU_INTS == SLU_MAX + 3 * 32,
                "the arrays above fill SLU_FLOATS and SLU_INTS exactly");
  const int b = blockIdx.x;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  float* Ab = A.at(b);
  const int64_t ld = A.ld;
  const bool vec = (ld & 3) == 0 && (reinterpret_cast<uintptr_t>(Ab) & 15) == 0;
  if (t < n) perm[t] = t;
  __syncthreads();
  for (int k0 = 0; k0 < n; k0 += PANEL_MAX) {
    const int kb = n - k0 < PANEL_MAX ? n - k0 : PANEL_MAX;
    const int m = n - k0;   // panel rows
    const int r0 = k0 + kb;
    const int mm = n - r0;  // trailing order (kb = 32 whenever mm > 0)
    // 1. panel -> P (all loads of a thread issued before its stores)
    if (vec && kb == PANEL_MAX) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        float4 v[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int e = t + SLU_THREADS * (4 * h + i);
          if (e < m * 8)
            v[i] = *reinterpret_cast<const float4*>(Ab + (int64_t)perm[k0 + (e >> 3)] * ld + k0 + 4 * (e & 7));
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int e = t + SLU_THREADS * (4 * h + i);
          if (e < m * 8) {
            float* d = P + (e >> 3) * SLU_PP + 4 * (e & 7);
            d[0] = v[i].x;
            d[1] = v[i].y;
            d[2] = v[i].z;
            d[3] = v[i].w;
          }
        }
      }
    } else {
      for (int e = t; e < m * PANEL_MAX; e += SLU_THREADS) {
        const int r = e >> 5, c = e & 31;
        P[r * SLU_PP + c] = c < kb ? Ab[(int64_t)perm[k0 + r] * ld + k0 + c] : 0.f;
      }
    }
    __syncthreads();
    // 2. the panel, column by column, one CTA barrier per column: thread t
    // keeps logical row k0 + t in registers; before the barrier each warp's
    // leading candidate row (and row j) is already in shared memory,
    // double-buffered by column parity.
    const bool mine = t < m;
    float rr[PANEL_MAX];
#pragma unroll
    for (int c = 0; c < PANEL_MAX; ++c) rr[c] = mine ? P[t * SLU_PP + c] : 0.f;
#pragma unroll
    for (int j = 0; j < PANEL_MAX; ++j) {
      if (j < kb) {
        const int buf = j & 1;
        const bool cand = mine && t >= j;
        const float kv = fabsf(rr[j]);
        const bool bad = cand && !(kv < INFINITY);  // NaN or infinite
        const unsigned key = (cand && kv == kv) ? __float_as_uint(kv) + 1u : 0u;
        const unsigned wmax = __reduce_max_sync(0xffffffffu, key);
        const int wl = __ffs(__ballot_sync(0xffffffffu, key == wmax)) - 1;
        const bool wbad = __any_sync(0xffffffffu, bad);
        if (lane == wl) {
          float4* d = reinterpret_cast<float4*>(cand_rows + (buf * 16 + warp) * PANEL_MAX);
#pragma unroll
          for (int q = 0; q < PANEL_MAX / 4; ++q) d[q] = make_float4(rr[4 * q], rr[4 * q + 1], rr[4 * q + 2], rr[4 * q + 3]);
        }
        if (t == j) {
          float4* d = reinterpret_cast<float4*>(jrow + buf * PANEL_MAX);
#pragma unroll
          for (int q = 0; q < PANEL_MAX / 4; ++q) d[q] = make_float4(rr[4 * q], rr[4 * q + 1], rr[4 * q + 2], rr[4 * q + 3]);
        }
        if (lane == 0) {
          redk[buf * 16 + warp] = wmax;
          redi[buf * 16 + warp] = warp * 32 + wl;
          redb[buf * 16 + warp] = wbad ? 1 : 0;
        }
        __syncthreads();
        const unsigned k16 = lane < 16 ? redk[buf * 16 + lane] : 0u;
        const unsigned gmax = __reduce_max_sync(0xffffffffu, k16);
        const int ww = __ffs(__ballot_sync(0xffffffffu, lane < 16 && k16 == gmax)) - 1;
        const bool anybad = __any_sync(0xffffffffu, lane < 16 && redb[buf * 16 + lane] != 0);
        const int p = gmax == 0u ? j : redi[buf * 16 + ww];
        const float4* prw =
            reinterpret_cast<const float4*>(gmax == 0u ? jrow + buf * PANEL_MAX : cand_rows + (buf * 16 + ww) * PANEL_MAX);
        const bool ok = !anybad && gmax > 1u;  // the largest |x| is above zero
        if (t == 0) {
          piv[(int64_t)b * n + k0 + j] = k0 + p;
          if (!ok) report(info, b, FROB_ERR_SINGULAR, info_off + k0 + j + 1);
          const int q = perm[k0 + j];
          perm[k0 + j] = perm[k0 + p];
          perm[k0 + p] = q;
        }
        if ((t == j || t == p) && p != j) {
          const float4* src = t == j ? prw : reinterpret_cast<const float4*>(jrow + buf * PANEL_MAX);
#pragma unroll
          for (int q = 0; q < PANEL_MAX / 4; ++q) {
            const float4 v = src[q];
            rr[4 * q] = v.x;
            rr[4 * q + 1] = v.y;
            rr[4 * q + 2] = v.z;
            rr[4 * q + 3] = v.w;
          }
        }
        if (mine && t > j) {
          float pr[PANEL_MAX];
#pragma unroll
          for (int q = j / 4; q < PANEL_MAX / 4; ++q) {
            const float4 v = prw[q];
            pr[4 * q] = v.x;
            pr[4 * q + 1] = v.y;
            pr[4 * q + 2] = v.z;
            pr[4 * q + 3] = v.w;
          }
          if (ok) rr[j] *= 1.f / pr[j];
          const float l = -rr[j];
#pragma unroll
          for (int c = j + 1; c < PANEL_MAX; ++c)
            if (c < kb) rr[c] = fmaf(l, pr[c], rr[c]);
        }
      }
    }
    // 3. the panel back (P, global memory), L21 into Lt, U12 into Ut
    if (mine) {
#pragma unroll
      for (int c = 0; c < PANEL_MAX; ++c) P[t * SLU_PP + c] = rr[c];
      if (t >= kb)
#pragma unroll
        for (int c = 0; c < PANEL_MAX; ++c) Lt[c * SLU_TP + (t - kb)] = rr[c];
    }
    __syncthreads();
    if (vec && kb == PANEL_MAX) {
      for (int e = t; e < m * 8; e += SLU_THREADS) {
        const int r = e >> 3, q = e & 7;
        const float* sp = P + r * SLU_PP + 4 * q;
        *reinterpret_cast<float4*>(Ab + (int64_t)perm[k0 + r] * ld + k0 + 4 * q) = make_float4(sp[0], sp[1], sp[2], sp[3]);
      }
    } else {
      for (int e = t; e < m * PANEL_MAX; e += SLU_THREADS) {
        const int r = e >> 5, c = e & 31;
        if (c < kb) Ab[(int64_t)perm[k0 + r] * ld + k0 + c] = P[r * SLU_PP + c];
      }
    }
    if (mm <= 0) break;
    if (t < mm) {
      float x[PANEL_MAX];
#pragma unroll
      for (int j = 0; j < PANEL_MAX; ++j) x[j] = Ab[(int64_t)perm[k0 + j] * ld + r0 + t];
#pragma unroll
      for (int j = 0; j < PANEL_MAX; ++j)
#pragma unroll
        for (int i = j + 1; i < PANEL_MAX; ++i) x[i] = fmaf(-P[i * SLU_PP + j], x[j], x[i]);
#pragma unroll
      for (int j = 0; j < PANEL_MAX; ++j) Ut[j * SLU_TP + t] = x[j];
    }
    __syncthreads();
#pragma unroll 8
    for (int j = 0; j < PANEL_MAX; ++j) {  // U12 back to global memory, row by row
      float* g = Ab + (int64_t)perm[k0 + j] * ld + r0;
      for (int c = t; c < mm; c += SLU_THREADS) g[c] = Ut[j * SLU_TP + c];
    }
    // 4. trailing update A22 -= L21 U12 over 32 x 16 tiles, each lane a
    // 4 x 4 block (its old values loaded before the FMAs)
    const int mt = (mm + 31) >> 5, nt = (mm + 15) >> 4;
    const int ty = lane >> 2, tx = lane & 3;
    for (int tile = warp; tile < mt * nt; tile += SLU_THREADS / 32) {
      const int I = tile / nt, J = tile % nt;
      const int rb = 32 * I + 4 * ty, cb = 16 * J + 4 * tx;
      const bool cfull = vec && cb + 3 < mm;
      float old[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int row = rb + i;
        const float* src = Ab + (int64_t)perm[r0 + (row < mm ? row : 0)] * ld + r0 + cb;
        if (row < mm && cfull) {
          const float4 v = *reinterpret_cast<const float4*>(src);
          old[i][0] = v.x;
          old[i][1] = v.y;
          old[i][2] = v.z;
          old[i][3] = v.w;
        } else {
#pragma unroll
          for (int j = 0; j < 4; ++j) old[i][j] = (row < mm && cb + j < mm) ? src[j] : 0.f;
        }
      }
      float acc[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
#pragma unroll 8
      for (int c = 0; c < PANEL_MAX; ++c) {
        const float4 rv = *reinterpret_cast<const float4*>(Lt + c * SLU_TP + rb);
        const float4 cv = *reinterpret_cast<const float4*>(Ut + c * SLU_TP + cb);
        const float ra[4] = {rv.x, rv.y, rv.z, rv.w};
        const float ca[4] = {cv.x, cv.y, cv.z, cv.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(ra[i], ca[j], acc[i][j]);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int row = rb + i;
        if (row >= mm) continue;
        float* dst = Ab + (int64_t)perm[r0 + row] * ld + r0 + cb;
        if (cfull) {
          *reinterpret_cast<float4*>(dst) = make_float4(old[i][0] - acc[i][0], old[i][1] - acc[i][1],
                                                        old[i][2] - acc[i][2], old[i][3] - acc[i][3]);
        } else {
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (cb + j < mm) dst[j] = old[i][j] - acc[i][j];
        }
      }
    }
    __syncthreads();
  }
  __syncthreads();
  // rows into logical order, SLU_GW columns at a time (loads before stores)
  for (int c0 = 0; c0 < n; c0 += SLU_GW) {
    const int w = n - c0 < SLU_GW ? n - c0 : SLU_GW;
    if (vec && w == SLU_GW) {
      float4 v[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int e = t + SLU_THREADS * i;  // row e >> 4, 4 columns (e & 15)
        if (e < n * 16) v[i] = *reinterpret_cast<const float4*>(Ab + (int64_t)perm[e >> 4] * ld + c0 + 4 * (e & 15));
      }
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int e = t + SLU_THREADS * i;
        if (e < n * 16) *reinterpret_cast<float4*>(G + (e >> 4) * SLU_GP + 4 * (e & 15)) = v[i];
      }
      __syncthreads();
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int e = t + SLU_THREADS * i;
        if (e < n * 16)
          *reinterpret_cast<float4*>(Ab + (int64_t)(e >> 4) * ld + c0 + 4 * (e & 15)) =
              *reinterpret_cast<const float4*>(G + (e >> 4) * SLU_GP + 4 * (e & 15));
      }
    } else {
      for (int e = t; e < n * SLU_GW; e += SLU_THREADS) {
        const int r = e / SLU_GW, c = e % SLU_GW;
        if (c < w) G[r * SLU_GP + c] = Ab[(int64_t)perm[r] * ld + c0 + c];
      }
      __syncthreads();
      for (int e = t; e < n * SLU_GW; e += SLU_THREADS) {
        const int r = e / SLU_GW, c = e % SLU_GW;
        if (c < w) Ab[(int64_t)r * ld + c0 + c] = G[r * SLU_GP + c];
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ multi-CTA panel
// LU with partial pivoting of one column panel [k0, k0 + kb) of a large
// matrix by G cooperating CTAs (grid: G x batch, one cooperative launch), for
// matrices too few to fill the GPU one CTA each.  CTA c keeps panel rows
// [c R, c R + R) in shared memory; row j of the panel always lies in CTA 0
// (R >= PANEL_MAX).  Per pivot column j, one grid-wide exchange:
//   1. every CTA finds its local candidate (largest key, lowest row) and
//      publishes it with a copy of that row; CTA 0 also publishes row j;
//   2. a grid barrier (bounded wait);
//   3. every CTA fetches all candidates and their rows in one round trip to
//      L2, reduces the keys in the same order (the same pivot as the one-CTA
//      kernels: largest key, ties to the lowest row, NaN never wins), the
//      owner of row j takes the pivot row, the owner of the pivot row takes
//      the old row j, and every CTA scales and updates its rows below j.
// The candidates are double-buffered by the parity of j, so one barrier per
// column suffices: a CTA can only overwrite buffer j mod 2 after every CTA
// has passed the barrier of column j + 1, i.e. has finished reading it.
// Arithmetic per element is that of getrf_panel_kernel (the same scaling by
// the reciprocal pivot and the same fused updates), so the factors are
// identical.  A wait that gives up sets the per-matrix flag, reports
// FROB_ERR_TIMEOUT and skips every later wait of the call; the results are
// then unusable but no CTA hangs.
constexpr int MC_THREADS = 256;
constexpr int MC_GMAX = 64;          // cooperating CTAs per matrix, at most
constexpr int MC_MIN_ROWS = 128;     // rows per CTA, at least
constexpr int MC_BATCH_MAX = 16;     // matrices per call that take this path
constexpr size_t MC_SMEM_MAX = 200 * 1024;

template <typename K> struct McKey {
  K key;
  int idx;
  int bad;
};
struct McHdr {
  unsigned count, gen;
  int err, pad;
};
// per-matrix scratch: header | keys[2][MC_GMAX] | rows[2][MC_GMAX][PANEL_MAX] | jrow[2][PANEL_MAX]
template <typename T> constexpr size_t mc_keys_off() { return 256; }
template <typename T> constexpr size_t mc_rows_off() {
  return mc_keys_off<T>() + ((2 * MC_GMAX * sizeof(McKey<typename real_of<T>::type>) + 255) & ~(size_t)255);
}
template <typename T> constexpr size_t mc_jrow_off() {
  return mc_rows_off<T>() + ((2 * MC_GMAX * PANEL_MAX * sizeof(T) + 255) & ~(size_t)255);
}
template <typename T> constexpr size_t mc_scratch_per_matrix() {
  return mc_jrow_off<T>() + ((2 * PANEL_MAX * sizeof(T) + 255) & ~(size_t)255);
}
// dynamic shared memory of a CTA holding R panel rows: the rows (stride
// PANEL_MAX + 1), then the G candidate rows and the old row j
template <typename T> constexpr size_t mc_smem(int R) {
  return sizeof(T) * ((size_t)R * (PANEL_MAX + 1) + (size_t)(MC_GMAX + 1) * PANEL_MAX);
}

// loads through L2 (not L1, which is not coherent across SMs) of values
// another CTA wrote
__device__ __forceinline__ double ldcg_(const double* p) { return __ldcg(p); }
__device__ __forceinline__ float ldcg_(const float* p) { return __ldcg(p); }
__device__ __forceinline__ zd ldcg_(const zd* p) {
  const double2 v = __ldcg(reinterpret_cast<const double2*>(p));
  return zd{v.x, v.y};
}
__device__ __forceinline__ zf ldcg_(const zf* p) {
  const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
  return zf{v.x, v.y};
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned atom_add_release_u32(unsigned* p, unsigned v) {
  unsigned old;
  asm volatile("atom.add.release.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

// Barrier of the G CTAs of one matrix (sense by generation count).  The
// CTA's writes before it are ordered by the CTA barrier and published by the
// releasing arrival (release is cumulative); the acquiring load that sees
// the new generation orders every read after the closing CTA barrier.
// Returns true when this or an earlier wait of the call gave up.
__device__ __forceinline__ bool mc_barrier(McHdr* h, unsigned G, long long limit_cycles) {
  __shared__ int s_gaveup;
  __syncthreads();
  if (threadIdx.x == 0) {
    int gaveup = *reinterpret_cast<volatile int*>(&h->err);
    if (!gaveup) {
      const unsigned g = ld_acquire_u32(&h->gen);
      const unsigned arrived = atom_add_release_u32(&h->count, 1u) + 1u;
      if (arrived == G) {
        atomicExch(&h->count, 0u);  // every CTA has arrived; none re-arrives before the new generation
        atom_add_release_u32(&h->gen, 1u);
      } else {
        const long long t0 = clock64();
        while (ld_acquire_u32(&h->gen) == g) {
          if (clock64() - t0 > limit_cycles) {
            atomicExch(&h->err, 1);
            gaveup = 1;
            break;
          }
        }
      }
    }
    s_gaveup = gaveup;
  }
  __syncthreads();
  return s_gaveup != 0;
}

template <typename T>
__global__ void __launch_bounds__(MC_THREADS) getrf_panel_mc_kernel(int n, int k0, int kb, MatB<T> A, int* piv,
                                                                     frob_info* info, int info_off,
                                                                     unsigned char* scr, int64_t scr_bs, int R,
                                                                     long long limit_cycles) {
  using K = typename real_of<T>::type;
  constexpr int PS = PANEL_MAX + 1;
  const int b = blockIdx.y, c = blockIdx.x, G = gridDim.x, t = threadIdx.x;
  const int m = n - k0;
  const int row0 = c * R;
  const int rc = max(0, min(R, m - row0));
  unsigned char* s = scr + (int64_t)b * scr_bs;
  McHdr* hdr = reinterpret_cast<McHdr*>(s);
  McKey<K>* keys = reinterpret_cast<McKey<K>*>(s + mc_keys_off<T>());
  T* rows = reinterpret_cast<T*>(s + mc_rows_off<T>());
  T* jrow = reinterpret_cast<T*>(s + mc_jrow_off<T>());
  extern __shared__ __align__(16) unsigned char smraw[];
  T* P = reinterpret_cast<T*>(smraw);       // [R][PS]
  T* cand = P + (size_t)R * PS;             // [MC_GMAX][PANEL_MAX]
  T* jr = cand + (size_t)MC_GMAX * PANEL_MAX;  // [PANEL_MAX]
  __shared__ KeyIdx<K> red[MC_THREADS / 32];
  __shared__ int redbad[MC_THREADS / 32];
  __shared__ McKey<K> sk[MC_GMAX];
  __shared__ T s_rinv;
  __shared__ int s_lwin, s_win, s_p, s_ok;
  T* g = A.at(b) + (int64_t)(k0 + row0) * A.ld + k0;
  for (int e = t; e < rc * kb; e += MC_THREADS) P[(e / kb) * PS + (e % kb)] = g[(int64_t)(e / kb) * A.ld + (e % kb)];
  __syncthreads();
  for (int j = 0; j < kb; ++j) {
    const int par = j & 1;
    // 1. local candidate over the rows >= j of column j
    KeyIdx<K> best{(K)-1, 0x7fffffff};
    bool bad = false;
    for (int lr = t; lr < rc; lr += MC_THREADS) {
      const int gi = row0 + lr;
      if (gi >= j) {
        const K kv = pkey(P[lr * PS + j]);
        if (!(kv == kv) || kv == (K)INFINITY) bad = true;
        best = kmax(best, KeyIdx<K>{kv, gi});
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      KeyIdx<K> other{__shfl_xor_sync(0xffffffffu, best.key, o), __shfl_xor_sync(0xffffffffu, best.idx, o)};
      best = kmax(best, other);
    }
    const unsigned wbad = __ballot_sync(0xffffffffu, bad);
    if ((t & 31) == 0) {
      red[t >> 5] = best;
      redbad[t >> 5] = wbad != 0;
    }
    __syncthreads();
    if (t == 0) {
      KeyIdx<K> bb = red[0];
      int anybad = redbad[0];
      for (int w = 1; w < MC_THREADS / 32; ++w) {
        bb = kmax(bb, red[w]);
        anybad |= redbad[w];
      }
      McKey<K> kk;
      kk.key = bb.key;
      kk.idx = bb.idx;
      kk.bad = anybad;
      keys[par * MC_GMAX + c] = kk;
      s_lwin = bb.idx;
    }
    __syncthreads();
    if (t < kb) {
      if (s_lwin != 0x7fffffff) rows[((int64_t)par * MC_GMAX + c) * PANEL_MAX + t] = P[(s_lwin - row0) * PS + t];
      if (c == 0) jrow[par * PANEL_MAX + t] = P[j * PS + t];
    }
    // 2. grid barrier
    if (mc_barrier(hdr, (unsigned)G, limit_cycles)) {
      if (c == 0 && t == 0) report(info, b, FROB_ERR_TIMEOUT, info_off + k0 + j + 1);
      break;
    }
    // 3. every candidate, its row and the old row j, fetched at once
    for (int e = t; e < G * kb; e += MC_THREADS)
      cand[(e / kb) * PANEL_MAX + (e % kb)] = ldcg_(&rows[((int64_t)par * MC_GMAX + e / kb) * PANEL_MAX + (e % kb)]);
    if (t < G) {
      const McKey<K>* kp = keys + par * MC_GMAX + t;
      McKey<K> kk;
      kk.key = __ldcg(&kp->key);
      kk.idx = __ldcg(&kp->idx);
      kk.bad = __ldcg(&kp->bad);
      sk[t] = kk;
    }
    if (t >= MC_THREADS - PANEL_MAX && t - (MC_THREADS - PANEL_MAX) < kb)
      jr[t - (MC_THREADS - PANEL_MAX)] = ldcg_(&jrow[par * PANEL_MAX + t - (MC_THREADS - PANEL_MAX)]);
    __syncthreads();
    // the pivot, the same in every CTA (candidates reduced in CTA order); its
    // row is the candidate of the CTA that owns it, p / R
    if (t < 32) {
      KeyIdx<K> bb{(K)-1, 0x7fffffff};
      int anybad = 0;
      for (int q = t; q < G; q += 32) {
        anybad |= sk[q].bad;
        bb = kmax(bb, KeyIdx<K>{sk[q].key, sk[q].idx});
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        KeyIdx<K> other{__shfl_xor_sync(0xffffffffu, bb.key, o), __shfl_xor_sync(0xffffffffu, bb.idx, o)};
        bb = kmax(bb, other);
      }
      anybad = __any_sync(0xffffffffu, anybad);
      if (t == 0) {
        const bool none = bb.idx == 0x7fffffff;
        const int p = none ? j : bb.idx;
        const int win = none ? -1 : bb.idx / R;
        const bool ok = !anybad && bb.key > (K)0;
        s_p = p;
        s_win = win;
        s_ok = ok;
        s_rinv = ok ? recip_(cand[win * PANEL_MAX + j]) : one_v<T>();
        if (c == 0) {
          piv[(int64_t)b * n + k0 + j] = k0 + p;
          if (!ok) report(info, b, FROB_ERR_SINGULAR, info_off + k0 + j + 1);
        }
      }
    }
    __syncthreads();
    const int p = s_p;
    const T* pr = s_win >= 0 ? cand + s_win * PANEL_MAX : P + j * PS;  // the pivot row
    if (p != j && t < kb) {
      const T pv = pr[t];
      if (p >= row0 && p < row0 + rc) P[(p - row0) * PS + t] = jr[t];
      if (c == 0) P[j * PS + t] = pv;
    }
    __syncthreads();
    // scale column j below the pivot, then the rank-1 update of the rest
    if (s_ok) {
      const T rinv = s_rinv;
      for (int lr = t; lr < rc; lr += MC_THREADS)
        if (row0 + lr > j) P[lr * PS + j] = mul_(P[lr * PS + j], rinv);
    }
    __syncthreads();
    // rows by thread modulo MC_THREADS / 2, the columns j + 1 + h, j + 3 + h, ...
    // by half h of the CTA
    {
      constexpr int HALF = MC_THREADS / 2;
      const int h = t / HALF;
      for (int lr = t % HALF; lr < rc; lr += HALF) {
        if (row0 + lr <= j) continue;
        const T l = neg_(P[lr * PS + j]);
        for (int cc = j + 1 + h; cc < kb; cc += 2) mac(P[lr * PS + cc], l, pr[cc]);
      }
    }
    __syncthreads();
  }
  for (int e = t; e < rc * kb; e += MC_THREADS) g[(int64_t)(e / kb) * A.ld + (e % kb)] = P[(e / kb) * PS + (e % kb)];
}

// ------------------------------------------------------------------ cluster panel
// The same factorization as getrf_panel_mc_kernel by one thread-block
// cluster of G <= 16 CTAs per matrix (grid: G x batch, cluster G x 1): CTA c
// keeps panel rows [c R, c R + R) in shared memory, and the candidates of a
// pivot column are exchanged through distributed shared memory with one
// hardware cluster barrier per column (release / acquire at cluster scope)
// instead of a barrier and round trips through L2.  Candidates, candidate
// rows and CTA 0's copy of row j are double-buffered by the parity of j (the
// argument of getrf_panel_mc_kernel: a CTA overwrites buffer j mod 2 only
// after the barrier of column j + 1, which every CTA passes after its reads
// of column j).  Every CTA runs the same loop, so every barrier is reached by
// the whole cluster; a first barrier makes the cluster's shared memory valid
// before any remote access and a last one keeps every CTA resident until the
// others' reads are done.  Pivots and arithmetic are those of the other
// panel kernels (the candidates reduced in CTA order, the same scaling and
// updates).
constexpr int CL_MAX = 16;

template <typename T>
__global__ void __launch_bounds__(MC_THREADS) getrf_panel_cl_kernel(int n, int k0, int kb, MatB<T> A, int* piv,
                                                                     frob_info* info, int info_off, int R) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  using K = typename real_of<T>::type;
  constexpr int PS = PANEL_MAX + 1;
  const int b = blockIdx.y, t = threadIdx.x;
  const int c = (int)cluster.block_rank(), G = (int)cluster.num_blocks();
  const int m = n - k0;
  const int row0 = c * R;
  const int rc = max(0, min(R, m - row0));
  extern __shared__ __align__(16) unsigned char smraw[];
  T* P = reinterpret_cast<T*>(smraw);  // [R][PS]
  __shared__ KeyIdx<K> red[MC_THREADS / 32];
  __shared__ int redbad[MC_THREADS / 32];
  __shared__ McKey<K> ckey[2];          // this CTA's candidate, by column parity
  __shared__ T crow[2][PANEL_MAX];       // ... and its row
  __shared__ T jrw[2][PANEL_MAX];        // CTA 0: row j before the exchange
  __shared__ T pr[PANEL_MAX];            // the pivot row
  __shared__ T jr[PANEL_MAX];            // row j, for the owner of the pivot row
  __shared__ T s_rinv;
  __shared__ int s_lwin, s_win, s_p, s_ok;
  T* g = A.at(b) + (int64_t)(k0 + row0) * A.ld + k0;
  for (int e = t; e < rc * kb; e += MC_THREADS) P[(e / kb) * PS + (e % kb)] = g[(int64_t)(e / kb) * A.ld + (e % kb)];
  cluster.sync();
  for (int j = 0; j < kb; ++j) {
    const int par = j & 1;
    KeyIdx<K> best{(K)-1, 0x7fffffff};
    bool bad = false;
    for (int lr = t; lr < rc; lr += MC_THREADS) {
      const int gi = row0 + lr;
      if (gi >= j) {
        const K kv = pkey(P[lr * PS + j]);
        if (!(kv == kv) || kv == (K)INFINITY) bad = true;
        best = kmax(best, KeyIdx<K>{kv, gi});
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      KeyIdx<K> other{__shfl_xor_sync(0xffffffffu, best.key, o), __shfl_xor_sync(0xffffffffu, best.idx, o)};
      best = kmax(best, other);
    }
    const unsigned wbad = __ballot_sync(0xffffffffu, bad);
    if ((t & 31) == 0) {
      red[t >> 5] = best;
      redbad[t >> 5] = wbad != 0;
    }
    __syncthreads();
    if (t == 0) {
      KeyIdx<K> bb = red[0];
      int anybad = redbad[0];
      for (int w = 1; w < MC_THREADS / 32; ++w) {
        bb = kmax(bb, red[w]);
        anybad |= redbad[w];
      }
      ckey[par].key = bb.key;
      ckey[par].idx = bb.idx;
      ckey[par].bad = anybad;
      s_lwin = bb.idx;
    }
    __syncthreads();
    if (t < kb) {
      if (s_lwin != 0x7fffffff) crow[par][t] = P[(s_lwin - row0) * PS + t];
      if (c == 0) jrw[par][t] = P[j * PS + t];
    }
    cluster.sync();  // publishes every CTA's candidate and CTA 0's row j
    if (t < 32) {
      KeyIdx<K> bb{(K)-1, 0x7fffffff};
      int anybad = 0;
      for (int q = t; q < G; q += 32) {
        const McKey<K>* kq = cluster.map_shared_rank(&ckey[par], (unsigned)q);
        anybad |= kq->bad;
        bb = kmax(bb, KeyIdx<K>{kq->key, kq->idx});
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        KeyIdx<K> other{__shfl_xor_sync(0xffffffffu, bb.key, o), __shfl_xor_sync(0xffffffffu, bb.idx, o)};
        bb = kmax(bb, other);
      }
      anybad = __any_sync(0xffffffffu, anybad);
      if (t == 0) {
        const bool none = bb.idx == 0x7fffffff;
        s_p = none ? j : bb.idx;
        s_win = none ? -1 : bb.idx / R;
        s_ok = !anybad && bb.key > (K)0;
      }
    }
    __syncthreads();
    const int p = s_p;
    if (t < kb) {
      pr[t] = s_win >= 0 ? cluster.map_shared_rank(&crow[par][0], (unsigned)s_win)[t] : P[j * PS + t];
      if (p != j && p >= row0 && p < row0 + rc) jr[t] = cluster.map_shared_rank(&jrw[par][0], 0u)[t];
    }
    __syncthreads();
    if (p != j && t < kb) {
      if (p >= row0 && p < row0 + rc) P[(p - row0) * PS + t] = jr[t];
      if (c == 0) P[j * PS + t] = pr[t];
    }
    if (t == 0) {
      if (c == 0) {
        piv[(int64_t)b * n + k0 + j] = k0 + p;
        if (!s_ok) report(info, b, FROB_ERR_SINGULAR, info_off + k0 + j + 1);
      }
      s_rinv = s_ok ? recip_(pr[j]) : one_v<T>();
    }
    __syncthreads();
    if (s_ok) {
      const T rinv = s_rinv;
      for (int lr = t; lr < rc; lr += MC_THREADS)
        if (row0 + lr > j) P[lr * PS + j] = mul_(P[lr * PS + j], rinv);
    }
    __syncthreads();
    {
      constexpr int HALF = MC_THREADS / 2;
      const int h = t / HALF;
      for (int lr = t % HALF; lr < rc; lr += HALF) {
        if (row0 + lr <= j) continue;
        const T l = neg_(P[lr * PS + j]);
        for (int cc = j + 1 + h; cc < kb; cc += 2) mac(P[lr * PS + cc], l, pr[cc]);
      }
    }
    __syncthreads();
  }
  cluster.sync();  // every remote read of this CTA's shared memory is done
  for (int e = t; e < rc * kb; e += MC_THREADS) g[(int64_t)(e / kb) * A.ld + (e % kb)] = P[(e / kb) * PS + (e % kb)];
}

}  // namespace frob
