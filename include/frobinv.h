/*
 * frobinv.h -- C ABI of the GB300 (sm_103a) Frobenius inversion library.
 *
 * Frobenius inversion (Dai, Lim and Ye, "Complex matrix inversion via real
 * matrix inversions", eq. (1.1) "Finv"): for M = A + iB with A, B real and A
 * invertible,
 *
 *     M^{-1} = S^{-1} - i A^{-1} B S^{-1},   S = A + B A^{-1} B,
 *
 * so a complex inversion costs two real inversions, three real products and
 * one real addition (Sec. 2, Algorithm "Frobenius inversion", tau = 1).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Matrices are square, complex and row-major, with the real and imaginary
 *   parts interleaved: complex128 (two doubles) for FROB_FP64 and the mixed
 *   modes, complex64 (two floats) for FROB_FP32.  Element (b, i, j) of a
 *   strided batch lives at base + b * stride + i * ld + j (counted in complex
 *   elements).  Because (M^T)^{-1} = (M^{-1})^T the row-major reading changes
 *   nothing about the result.
 * - All matrix pointers, the workspace and the info array are DEVICE
 *   pointers owned by the caller.  The library never allocates: it runs in
 *   the workspace of frob_workspace_bytes() bytes (256-byte aligned) that the
 *   caller passes in.  Output and input must not overlap.
 * - `stream` is a cudaStream_t passed as void*; NULL means the legacy default
 *   stream.  Every call is asynchronous with respect to the host.
 * - Host-visible argument errors (n < 1, batch < 1, ld < n, NULL pointers,
 *   overlapping input/output, workspace too small, unsupported precision)
 *   return synchronously and launch nothing.  FROB_ERR_CUDA means a launch
 *   failed; the CUDA error is left for cudaGetLastError().
 * - Numerical failures are per matrix and asynchronous: each matrix b gets a
 *   frob_info record in info[b], written on the device.  status is a
 *   frob_status and bad_index follows LAPACK's info convention (the 1-based
 *   step whose pivot was exactly zero or not finite, or whose Cholesky
 *   diagonal was not positive; n + j when the failure is in the second
 *   factorisation, of S).  The entry point returns FROB_OK once the work has
 *   been launched; read info after the stream has synchronised.
 */
#ifndef FROBINV_H
#define FROBINV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FROB_OK = 0,
  FROB_ERR_ARG = 1,           /* bad argument (host, synchronous) */
  FROB_ERR_SINGULAR = 2,      /* a pivot of A or S is exactly 0 or not finite */
  FROB_ERR_NOT_HPD = 3,       /* a Cholesky diagonal of A or S is not positive */
  FROB_ERR_NOT_CONVERGED = 4, /* refinement did not reach the tolerance */
  FROB_ERR_TIMEOUT = 5,       /* a bounded device wait gave up */
  FROB_ERR_CUDA = 6,          /* a CUDA launch failed */
  FROB_ERR_WORKSPACE = 7,     /* workspace NULL, too small or misaligned */
  FROB_ERR_UNSUPPORTED = 8    /* precision / operation not supported */
} frob_status;

typedef enum {
  FROB_FP64 = 0,       /* complex128 in and out, FP64 arithmetic throughout */
  FROB_FP32 = 1,       /* complex64 in and out, FP32 arithmetic throughout */
  FROB_MIXED_TF32 = 2, /* reserved: every entry point returns FROB_ERR_UNSUPPORTED
                          (a TF32 start does not contract at the workloads'
                          condition numbers; no separate TF32 path exists) */
  FROB_MIXED_BF16 = 3  /* complex128 in and out; FP32 start on the CUDA cores,
                          refinement with FP64-accurate products on the BF16
                          tensor cores */
} frob_prec;

/* Operation codes for frob_workspace_bytes(). */
typedef enum {
  FROB_OP_INV = 0,       /* frob_inv */
  FROB_OP_INV_HPD = 1,   /* frob_inv_hpd */
  FROB_OP_CPLX_LU = 2,   /* cplx_lu_inv */
  FROB_OP_CPLX_CHOL = 3, /* cplx_chol_inv */
  FROB_OP_ADJOINT = 4    /* frob_inv_adjoint */
} frob_op;

typedef struct {
  int32_t prec;        /* frob_prec */
  int32_t almost_sure; /* 1: Algorithm "Almost sure Frobenius inversion"
                          (Sec. 4.2): invert (1 + mu i) M, then multiply the
                          result by (1 + mu i).  Only for frob_inv. */
  uint64_t seed;       /* mu for matrix b is a counter-based draw from
                          (seed, b, attempt), uniform on (0, 1) */
  int32_t attempt;     /* draw index; a caller that sees FROB_ERR_SINGULAR
                          for matrix b may retry with attempt + 1 (Lemma
                          "rand Frob": at most n values of mu fail) */
  int32_t ns_max_iter; /* mixed modes: refinement iteration limit */
  double ns_tol;       /* mixed modes: target ||I - M X||_F/(||M||_F ||X||_F) */
  int32_t part;        /* frob_inv only: which real part is factored (frob_part).
                          FROB_PART_A: eq. "Finv", A invertible.
                          FROB_PART_B: the formula for invertible B (Sec. 4.2),
                          (A + iB)^{-1} = B^{-1}A(AB^{-1}A + B)^{-1}
                          - i(AB^{-1}A + B)^{-1}, computed as the A route on
                          -iM = B - iA followed by a multiplication by -i.
                          FROB_PART_AUTO: per matrix, both A and B are
                          factored (one extra LU, 2n^3/3 flops) and the one
                          whose U has the larger min |u_kk| / max |u_kk| is
                          used (a singular factor counts as 0).  Not with
                          almost_sure. */
  int32_t fp64_gemm;   /* FROB_FP64 only (frob_gemm): how the large real
                          products run.  FROB_GEMM_AUTO: products of at least
                          256 in every dimension as exact digit products on
                          the BF16 tensor cores (FP64-accurate: each operand
                          row / column scaled by a power of two and split into
                          eight 7-bit digits, digit products exact in FP32
                          over K chunks of 512, summed exactly in 64-bit fixed
                          point); FROB_GEMM_FP64_PIPE: every product on the
                          FP64 pipe.  Other values: FROB_ERR_ARG. */
} frob_opts;           /* NULL => {FROB_FP64, 0, 0, 0, 8, 1e-14, FROB_PART_A, FROB_GEMM_AUTO} */

typedef enum { FROB_GEMM_AUTO = 0, FROB_GEMM_FP64_PIPE = 1 } frob_gemm;

typedef enum { FROB_PART_A = 0, FROB_PART_B = 1, FROB_PART_AUTO = 2 } frob_part;

typedef struct {
  int32_t status;    /* frob_status of this matrix */
  int32_t bad_index; /* LAPACK-style 1-based failing step, 0 if none */
  int32_t ns_iters;  /* refinement iterations taken (mixed modes) */
  int32_t fell_back; /* 1 if the mixed mode fell back to a wider format */
  double mu;         /* the rotation used by the almost sure variant, else 0 */
  double residual;   /* mixed modes: the last residual measured */
} frob_info;         /* 32 bytes */

/* Workspace size in bytes for `op` on `batch` matrices of order n in
 * precision `prec`; 0 for invalid arguments. */
size_t frob_workspace_bytes(int op, int n, int batch, int prec);

/*
 * frob_inv -- Frobenius inversion of a strided batch of general complex
 * matrices (eq. (1.1); Algorithm "Frobenius inversion with LU decomposition",
 * Sec. 4.1).  Per matrix: split M into planes A, B; LU with partial pivoting
 * A = P1^T L1 U1; X1 = A^{-1} B by two triangular solves; S = A + B X1; LU of
 * S; S^{-1} = U2^{-1} L2^{-1} P2; X = S^{-1} - i X1 S^{-1}, written
 * interleaved.  With opts->almost_sure the input is first rotated,
 * A' = A - mu B, B' = mu A + B, and the result un-rotated, X = (X3 - mu X4) +
 * i (mu X3 + X4) (Sec. 4.2).  Fails per matrix with FROB_ERR_SINGULAR if A
 * (bad_index = k) or S (bad_index = n + k) has an exactly zero pivot.
 *
 *   n, batch   order and number of matrices (n >= 1, batch >= 1)
 *   M, ldm, sm input base, leading dimension (>= n), batch stride (elements)
 *   X, ldx, sx output base, leading dimension, batch stride (elements)
 *   opts       NULL or options.  FROB_FP64 / FROB_FP32: the algorithm in that
 *              precision.  FROB_MIXED_BF16 (n <= 512,
 *              complex128 in and out): X0 by the FP32 algorithm, then
 *              Newton-Schulz refinement X <- X + X (I - M X) until
 *              ||I - M X||_F/(||M||_F ||X||_F) <= opts->ns_tol, at most
 *              opts->ns_max_iter corrections; the products are FP64-accurate
 *              (exact digit products on the BF16 tensor cores).  A matrix that
 *              does not reach the tolerance gets FROB_ERR_NOT_CONVERGED;
 *              info.ns_iters and info.residual report the iteration.
 *   ws, wsb    device workspace and its size in bytes
 *   info       device array of `batch` frob_info records (written)
 */
frob_status frob_inv(int n, int batch, const void* M, int64_t ldm, int64_t sm, void* X, int64_t ldx, int64_t sx,
                     const frob_opts* opts, void* ws, size_t wsb, frob_info* info, void* stream);

/*
 * frob_inv_hpd -- Frobenius inversion of Hermitian positive definite
 * matrices (Sec. 4.3, Algorithm "Frobenius inversion with Cholesky
 * decomposition", and eq. (4.2) "cholesky").  Only the lower triangle of each
 * M is read: A = Re (symmetric), B = Im (skew, zero diagonal).  Per matrix:
 * A = R1^T R1; R1^T X1 = B; R1 X2 = X1; S = A - X1^T X1 (= A + B A^{-1} B);
 * S = R2^T R2; R2^T X5 = I; R2 X6 = X5; X = X6 - i X2 X6, both triangles
 * written.  Fails per matrix with FROB_ERR_NOT_HPD (bad_index = k for A,
 * n + k for S).  Arguments as for frob_inv.  The mixed precisions (n <= 512)
 * start from this algorithm in FP32 and refine like frob_inv's mixed modes.
 */
frob_status frob_inv_hpd(int n, int batch, const void* M, int64_t ldm, int64_t sm, void* X, int64_t ldx, int64_t sx,
                         const frob_opts* opts, void* ws, size_t wsb, frob_info* info, void* stream);

/*
 * cplx_lu_inv -- the baseline: inversion in complex arithmetic by LU with
 * partial pivoting (Sec. 4, Algorithm "Inversion with LU decomposition"):
 * M = P^T L U, then M^{-1} = U^{-1} L^{-1} P.  Arguments as for frob_inv;
 * `prec` is FROB_FP64 (complex128) or FROB_FP32 (complex64), or
 * FROB_MIXED_BF16: cplx_inv_mixed(FROB_OP_CPLX_LU, ...) with the default
 * refinement options.
 */
frob_status cplx_lu_inv(int n, int batch, const void* M, int64_t ldm, int64_t sm, void* X, int64_t ldx, int64_t sx,
                        int prec, void* ws, size_t wsb, frob_info* info, void* stream);

/*
 * cplx_chol_inv -- the HPD baseline: inversion in complex arithmetic by
 * Cholesky (Sec. 4.3, Algorithm "Inversion with Cholesky decomposition"):
 * M = R^H R, R^H X1 = I, R X2 = X1, M^{-1} = X2.  Lower triangle read.
 * `prec` as for cplx_lu_inv (FROB_MIXED_BF16: the refined control).
 */
frob_status cplx_chol_inv(int n, int batch, const void* M, int64_t ldm, int64_t sm, void* X, int64_t ldx,
                          int64_t sx, int prec, void* ws, size_t wsb, frob_info* info, void* stream);

/*
 * cplx_inv_mixed -- the control for the mixed-precision Frobenius forms (no
 * counterpart in the paper, which has no mixed precision): X0 by complex LU
 * (op = FROB_OP_CPLX_LU) or complex Cholesky (op = FROB_OP_CPLX_CHOL, lower
 * triangle read) inversion in FP32, then exactly the Newton-Schulz
 * refinement of frob_inv's FROB_MIXED_BF16 mode (the same digit-split
 * residual and correction products, tolerance and iteration limit from
 * opts).  Comparing it with frob_inv / frob_inv_hpd at FROB_MIXED_BF16
 * separates what Frobenius inversion contributes from what the refinement
 * does.  opts: NULL (FROB_MIXED_BF16, ns_tol 1e-14, ns_max_iter 8) or with
 * prec = FROB_MIXED_BF16, almost_sure = 0, part = FROB_PART_A.  n <= 512;
 * complex128 in and out; workspace frob_workspace_bytes(op, n, batch,
 * FROB_MIXED_BF16).  Other arguments and results as for frob_inv's mixed
 * mode.
 */
frob_status cplx_inv_mixed(int op, int n, int batch, const void* M, int64_t ldm, int64_t sm, void* X, int64_t ldx,
                           int64_t sx, const frob_opts* opts, void* ws, size_t wsb, frob_info* info, void* stream);

/*
 * frob_inv_hpd_noalloc -- frob_inv_hpd in FP64 for callers that cannot
 * allocate device memory (no counterpart in the paper: this is a deployment
 * variant).  Some callers own no allocator: a plugin inside a framework that
 * manages every device buffer itself, a latency-bound loop in which a
 * cudaMalloc could stall the device, or a foreign-language caller without a
 * device allocator.  They pass only the input M, the output X and the info
 * records; the workspace is a 32 MiB scratch array inside the library,
 * allocated on every GPU that loads the library and held until the process
 * exits.
 *
 * Arguments and results are those of frob_inv_hpd with prec = FROB_FP64.
 * The problem must fit the scratch: frob_workspace_bytes(FROB_OP_INV_HPD, n,
 * batch, FROB_FP64) <= 32 MiB, about 64 n^2 batch bytes (four FP64 planes and,
 * from n = 256 on, the digits of the final product), i.e. n * n * batch up to
 * about 5e5 (n = 512 with batch 1, n = 256 with batch 7); larger problems
 * return FROB_ERR_WORKSPACE and launch nothing.  Other argument errors return
 * FROB_ERR_ARG.
 *
 * The first call made with a given device current looks up the scratch
 * array's device address on that device and keeps it for the life of the
 * process; make that first call before any stream capture, and do not reset
 * the device (cudaDeviceReset) between calls, since the array may move when
 * the library's module is loaded again.  The function itself calls no cudaMalloc, cudaFree or other
 * allocating routine.  All calls share the one scratch array, which keeps
 * whatever the last call left in it (no call depends on its contents):
 * calls whose work overlaps on the GPU -- on different streams, or from
 * different host threads without ordering -- race on it and give wrong
 * results.
 */
frob_status frob_inv_hpd_noalloc(int n, int batch, const void* M, int64_t ldm, int64_t sm, void* X, int64_t ldx,
                                 int64_t sx, frob_info* info, void* stream);

/*
 * frob_gemm_tc -- the tensor-core GEMM building block (no counterpart in the
 * paper; it serves the mixed-precision forms): C[b] = A[b] . B[b]^T with
 * A (M x K) and B (N x K) row-major FP32 on the device, both rounded to
 * nearest into BF16 (kind 0) or TF32 (kind 1) in the workspace, multiplied
 * by tcgen05.mma with FP32 accumulation in tensor memory, C (M x N) FP32.
 * `err` is a device int set to FROB_ERR_TIMEOUT if a bounded wait inside the
 * kernel gave up (0 otherwise; the caller zeroes it).  Workspace:
 * frob_gemm_tc_workspace_bytes(kind, M, N, K, batch) bytes, 256-aligned.
 */
frob_status frob_gemm_tc(int kind, int M, int N, int K, int batch, const float* A, int64_t lda, int64_t sa,
                         const float* B, int64_t ldb, int64_t sb, float* C, int64_t ldc, int64_t sc, void* ws,
                         size_t wsb, int* err, void* stream);
size_t frob_gemm_tc_workspace_bytes(int kind, int M, int N, int K, int batch);

/*
 * frob_gemm_f64 -- the FP64 digit-product GEMM building block (no
 * counterpart in the paper; it carries Frobenius inversion's FP64 products,
 * see frob_opts.fp64_gemm): C[b] = alpha op(A[b]) op(B[b]) + beta C[b] with
 * op(A) M x K, op(B) K x N, row-major FP64 on the device (op(A) = A^T when
 * transA = 1, likewise B), as exact BF16 digit products on the tensor cores:
 * each row of op(A) and column of op(B) scaled by a power of two and written
 * with eight signed 7-bit digits, the 36 digit pairs of weight 2^-14 ..
 * 2^-63 multiplied with FP32 accumulation (exact per 512-wide K chunk) and
 * summed exactly in 64-bit fixed point.  The error is at most about 2^-57
 * sqrt(K) of the row and column maxima, below an FP64 product's.  A row or
 * column holding an infinity or a NaN gives NaN entries.  beta = 0: C is not
 * read.  M and N are at least 128 and K at least 1 (FROB_ERR_ARG
 * otherwise; K <= 128 is padded to 128, so a thin product costs as much as
 * one of K = 128), batch at most 65535.  `err` is a device int set to FROB_ERR_TIMEOUT if a bounded wait
 * gave up (the caller zeroes it).  Workspace:
 * frob_gemm_f64_workspace_bytes(M, N, K, batch) bytes (0 for invalid sizes),
 * 256-aligned; about 16 (M + N) K batch bytes.
 */
frob_status frob_gemm_f64(int M, int N, int K, int batch, const double* A, int64_t lda, int64_t sa, int transA,
                          const double* B, int64_t ldb, int64_t sb, int transB, double* C, int64_t ldc, int64_t sc,
                          double alpha, double beta, void* ws, size_t wsb, int* err, void* stream);
size_t frob_gemm_f64_workspace_bytes(int M, int N, int K, int batch);

/*
 * frob_inv_adjoint -- reverse-mode derivative of inversion: for X = M^{-1}
 * and the gradient G of a real loss with respect to X (G = dL/dRe X +
 * i dL/dIm X, PyTorch's convention), writes gradM = -X^H G X^H, which follows
 * from d(M^{-1}) = -M^{-1} dM M^{-1}.  Computed as two complex products, each
 * with Gauss's three real multiplications (Sec. 2, Proposition "matrix
 * mult"), on the CUDA cores.  X, G, gradM: strided batches like frob_inv's,
 * complex128 (prec FROB_FP64) or complex64 (FROB_FP32); gradM must not
 * overlap X or G.  Workspace: frob_workspace_bytes(FROB_OP_ADJOINT, ...).
 */
frob_status frob_inv_adjoint(int n, int batch, const void* X, int64_t ldx, int64_t sx, const void* G, int64_t ldg,
                             int64_t sg, void* gradM, int64_t ldr, int64_t sr, int prec, void* ws, size_t wsb,
                             void* stream);

/*
 * frob_inv_batched -- `batch` matrices of different orders in one call (no
 * counterpart in the paper: the batched driver).  Each matrix M_i of order
 * n_i is embedded as M_i (+) I in a bucket of order 32 ceil(n_i / 32) --
 * (M (+) I)^{-1} = M^{-1} (+) I exactly -- and every bucket runs the uniform
 * entry point selected by `op` (FROB_OP_INV, FROB_OP_INV_HPD, FROB_OP_CPLX_LU
 * or FROB_OP_CPLX_CHOL) with `opts` (precision; the almost sure option is not
 * supported here).  Results and info records are scattered back.
 * With FROB_PART_B the padding block is iI, with FROB_PART_AUTO (1 + i)I, so
 * that the factored part of the padding is invertible; with FROB_PART_AUTO
 * the padding's unit pivots enter the pivot ratio min |u_kk| / max |u_kk|
 * that chooses the part, so a matrix in an uneven batch may be inverted
 * through the other part than the same matrix alone (both are correct
 * inverses; results may then differ in rounding).
 *
 *   n_host, n_dev   the orders, on the host (to plan the launches) and on
 *                   the device (identical contents)
 *   M_dev, ldm_dev  device arrays of `batch` input pointers / leading dims
 *   X_dev, ldx_dev  device arrays of `batch` output pointers / leading dims
 *   ws, wsb         frob_inv_batched_workspace_bytes(op, batch, n_host, prec)
 *   info            device array of `batch` frob_info records
 * A call is a fixed launch sequence on `stream` (no allocation, no host
 * synchronisation), so it may be captured into a CUDA graph after a first
 * call on the device.
 */
size_t frob_inv_batched_workspace_bytes(int op, int batch, const int32_t* n_host, int prec);
frob_status frob_inv_batched(int op, int batch, const int32_t* n_host, const int32_t* n_dev,
                             const void* const* M_dev, const int64_t* ldm_dev, void* const* X_dev,
                             const int64_t* ldx_dev, const frob_opts* opts, void* ws, size_t wsb, frob_info* info,
                             void* stream);

/*
 * frob_solve -- solve (A + iB)(X + iY) = C + iD for nrhs right-hand sides
 * without forming the inverse (Sec. 3, Algorithm "Linear system with
 * Frobenius inversion"): A = P1^T L1 U1; X1 = A^{-1} B by two triangular
 * solves; S = A + B X1; S = P2^T L2 U2; [x1, y1] = S^{-1} [C, D];
 * [x2, y2] = A^{-1} B [y1, x1]; X = x1 + x2, Y = y1 - y2 (the imaginary part
 * of M^{-1}(C + iD) by eq. (1.1); the printed last step has the opposite
 * sign).  M: n x n strided batch; B (right-hand sides) and X (solutions):
 * n x nrhs strided batches (row-major, complex, ld >= nrhs).  prec
 * FROB_FP64 (complex128) or FROB_FP32 (complex64).  FROB_ERR_SINGULAR per
 * matrix as for frob_inv.  Workspace: frob_solve_workspace_bytes(0, ...).
 *
 * cplx_lu_solve -- the baseline: M = P^T L U in complex arithmetic, then
 * L U X = P B.  Workspace: frob_solve_workspace_bytes(1, ...).
 *
 * aug_real_solve -- the third method of Sec. 5.2: the 2n real augmented
 * system [[A, -B], [B, A]] [x; y] = [c; d], by real LU with partial pivoting
 * of the 2n x 2n matrix (bad_index up to 2n).  Workspace:
 * frob_solve_workspace_bytes(2, ...).
 */
size_t frob_solve_workspace_bytes(int op, int n, int nrhs, int batch, int prec);
frob_status frob_solve(int n, int nrhs, int batch, const void* M, int64_t ldm, int64_t sm, const void* B, int64_t ldb,
                       int64_t sb, void* X, int64_t ldx, int64_t sx, int prec, void* ws, size_t wsb, frob_info* info,
                       void* stream);
frob_status cplx_lu_solve(int n, int nrhs, int batch, const void* M, int64_t ldm, int64_t sm, const void* B,
                          int64_t ldb, int64_t sb, void* X, int64_t ldx, int64_t sx, int prec, void* ws, size_t wsb,
                          frob_info* info, void* stream);
frob_status aug_real_solve(int n, int nrhs, int batch, const void* M, int64_t ldm, int64_t sm, const void* B,
                           int64_t ldb, int64_t sb, void* X, int64_t ldx, int64_t sx, int prec, void* ws, size_t wsb,
                           frob_info* info, void* stream);

/*
 * Newton drivers over the batched inversions (Sec. 5.3-5.5), each step a
 * Frobenius inversion of the whole batch (route FROB_ROUTE_FROB, any
 * precision frob_inv accepts) or, as the baseline, a complex-LU inversion
 * (FROB_ROUTE_CPLX_LU, FROB_FP64 or FROB_FP32).
 *
 * frob_newton -- X_0 = M and, for kind FROB_NEWTON_SIGN, the matrix sign
 * iteration X_{k+1} = (X_k + X_k^{-1}) / 2 (Sec. 5.3, eq. "iter"); for
 * FROB_NEWTON_POLAR, X_{k+1} = (X_k + X_k^{-H}) / 2 (Sec. 5.5, eq. "iter2"),
 * whose limit is the unitary polar factor.  A matrix stops after the first
 * step k with ||X_k - X_{k-1}||_max <= eps ||X_k||_max (max of the entries'
 * moduli; the rule of Sec. 5.3) or after kmax steps; the call returns when
 * every matrix of the batch has stopped, with X holding the last iterates and
 * steps[b] (device, int32 per matrix) the steps matrix b took.  The host
 * reads one 4-byte count after each step (a stream synchronisation) to stop
 * early; while `stream` is being captured into a CUDA graph it reads
 * nothing, the graph holds all kmax steps, and the matrices that met the
 * rule stay unchanged in the later ones, so a replay gives the results and
 * step counts of an uncaptured call (at the cost of the remaining steps'
 * work; choose kmax accordingly).  M and X as for frob_inv (complex128, or
 * complex64 for FROB_FP32; X may equal M exactly, other overlap is an
 * error).  info[b] (device) is zero unless an inversion failed, in which case
 * it is that inversion's record and matrix b stopped there.  opts as for
 * frob_inv (the almost sure option is ignored).  Workspace:
 * frob_newton_workspace_bytes(n, batch, prec, route).
 *
 * frob_sylvester -- Y with A Y + Y B = C (A p x p, B q x q, C and Y p x q;
 * lyapunov = 1: B = A^H and the B argument is ignored) through the sign of
 * [[A, -C], [0, -B]], which is [[I, -2Y], [0, -I]] when sign(A) = I and
 * sign(B) = I (Sec. 5.4): the sign iteration above on the block matrix, then
 * Y = -1/2 its top-right block.  Workspace:
 * frob_sylvester_workspace_bytes(p, q, batch, prec, route).
 *
 * frob_polar -- X = Q P (Sec. 5.5): Q by the FROB_NEWTON_POLAR iteration from
 * X, then P = Q^H X.  Q and P must not overlap X.  Workspace:
 * frob_polar_workspace_bytes(n, batch, prec, route).
 */
typedef enum { FROB_NEWTON_SIGN = 0, FROB_NEWTON_POLAR = 1 } frob_newton_kind;
typedef enum { FROB_ROUTE_FROB = 0, FROB_ROUTE_CPLX_LU = 1 } frob_inv_route;
size_t frob_newton_workspace_bytes(int n, int batch, int prec, int route);
frob_status frob_newton(int kind, int route, int n, int batch, const void* M, int64_t ldm, int64_t sm, void* X,
                        int64_t ldx, int64_t sx, const frob_opts* opts, double eps, int kmax, void* ws, size_t wsb,
                        frob_info* info, int32_t* steps, void* stream);
size_t frob_sylvester_workspace_bytes(int p, int q, int batch, int prec, int route);
frob_status frob_sylvester(int route, int p, int q, int batch, const void* A, int64_t lda, int64_t sa, const void* B,
                           int64_t ldb, int64_t sb, int lyapunov, const void* C, int64_t ldc, int64_t sc, void* Y,
                           int64_t ldy, int64_t sy, const frob_opts* opts, double eps, int kmax, void* ws, size_t wsb,
                           frob_info* info, int32_t* steps, void* stream);
size_t frob_polar_workspace_bytes(int n, int batch, int prec, int route);
frob_status frob_polar(int route, int n, int batch, const void* X, int64_t ldx, int64_t sx, void* Q, int64_t ldq,
                       int64_t sq, void* P, int64_t ldp, int64_t sp, const frob_opts* opts, double eps, int kmax,
                       void* ws, size_t wsb, frob_info* info, int32_t* steps, void* stream);

/*
 * frob_inv_bicomplex -- inversion over the iterated quadratic extension of
 * Sec. 2.4 with m = 2 (Theorem "GFiter"): X = A + jB with A, B complex n x n
 * (complex128, or complex64 for FROB_FP32), j^2 = -1 and j commuting with i.
 * Frobenius inversion over C: X1 = A^{-1}, X2 = X1 B, X4 = A + B X2,
 * X5 = X4^{-1}, X6 = X2 X5, X^{-1} = Y0 + jY1 with Y0 = X5, Y1 = -X6; each
 * complex inversion a frob_inv call (any precision it accepts), each complex
 * product by Gauss's three real multiplications: 15 real products and 4 real
 * inversions.  info[b]: the first failing inversion's record (bad_index as
 * frob_inv reports it for A, plus 2n for A + B X2).  Y0 and Y1 must not
 * overlap A, B or each other.  opts as for frob_inv (part FROB_PART_A, no
 * almost sure option).  Workspace: frob_inv_bicomplex_workspace_bytes.
 */
size_t frob_inv_bicomplex_workspace_bytes(int n, int batch, int prec);
frob_status frob_inv_bicomplex(int n, int batch, const void* A, int64_t lda, int64_t sa, const void* B, int64_t ldb,
                               int64_t sb, void* Y0, int64_t ldy0, int64_t sy0, void* Y1, int64_t ldy1, int64_t sy1,
                               const frob_opts* opts, void* ws, size_t wsb, frob_info* info, void* stream);

/* Human-readable name of a status code (static storage). */
const char* frob_status_str(int status);

/* Library version string (static storage). */
const char* frob_version(void);

/* Number of CUDA kernels this library has launched in this process (all
 * devices, all threads) since it was loaded.  Diagnostics: lets a caller count
 * the kernels behind a call. */
uint64_t frob_kernel_launches(void);

/* Per-kernel device-time profiling (diagnostics, off by default).
 * frob_profile_enable(1) discards earlier records and starts bracketing every
 * kernel launch of the library with a pair of CUDA events recorded on the
 * launching stream; frob_profile_enable(0) stops recording.
 * frob_profile_report() waits for the recorded events, writes a JSON object
 * {"<kernel variant>": [launches, total_ms, flops], ...} into buf (flops: the
 * real floating-point operations the launches were asked to compute, 2 M N K
 * per real product and 8 M N K per complex one over the tiles a product
 * computes, plus the substitutions of the triangular solves; 0 for kernels
 * that do not count them) (truncated to len
 * bytes, NUL-terminated), releases the records and returns the length needed
 * including the NUL.  Not for use inside CUDA graph capture.  While profiling
 * is on, a call whose batch is split over internal streams runs the slices
 * one after the other on the caller's stream (each kernel then runs alone). */
void frob_profile_enable(int on);
size_t frob_profile_report(char* buf, size_t len);

/* Autotuning of the stream split (off by default).  A batch of two or more
 * matrices normally runs as two slices on two internal streams; with
 * frob_autotune_enable(1), the first call of frob_inv, frob_inv_hpd,
 * cplx_lu_inv or cplx_chol_inv for a given (operation, precision, n, batch)
 * runs three times (an untimed two-slice warm-up, then one slice and two
 * slices timed with CUDA events, with a host synchronisation) and caches the
 * faster split, which later calls use.  The FP64 / FP32 results do not
 * depend on the split (every matrix runs the same kernels); the mixed
 * precisions' only through the order of atomic residual sums.  No tuning
 * happens during a CUDA-graph capture or while the per-kernel profiler is
 * on, and not when the workspace is too small for the one-slice layout.
 * frob_autotune_report writes {"op,prec,n,batch": [slices, ms_one_slice,
 * ms_two_slices], ...} like frob_profile_report; frob_autotune_clear empties
 * the cache. */
void frob_autotune_enable(int on);
void frob_autotune_clear(void);
size_t frob_autotune_report(char* buf, size_t len);

#ifdef __cplusplus
}
#endif

#endif /* FROBINV_H */
