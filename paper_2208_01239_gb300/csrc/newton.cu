// Newton drivers over the batched inversions (Sec. 5.3-5.5 of Dai, Lim and
// Ye): the matrix sign function by X_{k+1} = (X_k + X_k^{-1}) / 2 (eq.
// "iter"), the unitary polar factor by X_{k+1} = (X_k + X_k^{-H}) / 2 (eq.
// "iter2") with P = Q^H X, and the Sylvester / Lyapunov equation
// A Y + Y B = C through sign([[A, -C], [0, -B]]) = [[I, -2Y], [0, -I]].
//
// Each step inverts the whole batch with frob_inv (or, for the baseline
// route, cplx_lu_inv), then one fused kernel forms the average in place and
// the per-matrix maxima of |X_{k+1} - X_k| and |X_{k+1}| (the stopping rule
// of Sec. 5.3 compares their ratio with eps in the max norm); a second kernel
// applies the rule, counts the matrices still running, and the host reads
// that count after each step (one 4-byte copy and a stream synchronisation),
// so the driver is not graph-capturable.  Matrices that have stopped keep
// their iterate; they are still inverted with the rest of the batch.
#include <cstdint>
#include <cstring>
#include <cuda_runtime.h>

#include "../../include/frobinv.h"
#include "common.cuh"
#include "ops_impl.cuh"

namespace frob {
namespace newton {

constexpr int TILE = 32;
constexpr int ROWS = 8;  // threads per tile column; a block is TILE x ROWS threads

__device__ __forceinline__ zd cadd_half(zd a, zd b) { return zd{(a.x + b.x) * 0.5, (a.y + b.y) * 0.5}; }
__device__ __forceinline__ zf cadd_half(zf a, zf b) { return zf{(a.x + b.x) * 0.5f, (a.y + b.y) * 0.5f}; }
__device__ __forceinline__ zd conj_c(zd a) { return zd{a.x, -a.y}; }
__device__ __forceinline__ zf conj_c(zf a) { return zf{a.x, -a.y}; }
__device__ __forceinline__ double abs2d(zd a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ double abs2d(zf a) { return (double)a.x * a.x + (double)a.y * a.y; }

// Per-matrix state in the workspace.
struct State {
  unsigned long long* dmax2;  // [batch] max |X_{k+1} - X_k|^2 (bit pattern of a non-negative double)
  unsigned long long* xmax2;  // [batch] max |X_{k+1}|^2
  int* done;                  // [batch] 1 once the rule has stopped the matrix (or its inversion failed)
  int* remaining;             // [1] matrices still running after this step
  frob_info* inner;           // [batch] info of this step's inversion
};

__global__ void init_kernel(int batch, State s, frob_info* info, int32_t* steps) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch) return;
  s.dmax2[b] = 0ull;
  s.xmax2[b] = 0ull;
  s.done[b] = 0;
  steps[b] = 0;
  frob_info z = {};
  info[b] = z;
}

// A failed inversion stops its matrix and its info becomes the result's.
__global__ void merge_kernel(int batch, State s, frob_info* info) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b == 0) *s.remaining = 0;
  if (b >= batch || s.done[b]) return;
  if (s.inner[b].status != FROB_OK) {
    info[b] = s.inner[b];
    s.done[b] = 1;
  }
}

// X <- (X + Y') / 2 for the running matrices, Y' = Xinv (sign) or Xinv^H
// (polar); the maxima of |X_new - X_old|^2 and |X_new|^2 per matrix.
// Grid: (n / TILE, n / TILE, batch) rounded up; block TILE x ROWS.
template <typename C, bool POLAR>
__global__ void __launch_bounds__(TILE * ROWS) average_kernel(int n, MatB<C> X, MatB<const C> Xinv, State s) {
  const int b = blockIdx.z;
  if (s.done[b]) return;
  __shared__ C tile[TILE][TILE + 1];
  const int i0 = blockIdx.y * TILE, j0 = blockIdx.x * TILE;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const C* yb = Xinv.at(b);
  if (POLAR) {
    // (Xinv^H)[i][j] = conj(Xinv[j][i]): read the transposed tile coalesced
    for (int r = ty; r < TILE; r += ROWS) {
      const int jj = j0 + r, ii = i0 + tx;
      if (jj < n && ii < n) tile[tx][r] = conj_c(yb[(int64_t)jj * Xinv.ld + ii]);
    }
    __syncthreads();
  }
  double dm = 0.0, am = 0.0;
  C* xb = X.at(b);
  for (int r = ty; r < TILE; r += ROWS) {
    const int i = i0 + r, j = j0 + tx;
    if (i < n && j < n) {
      const C y = POLAR ? tile[r][tx] : yb[(int64_t)i * Xinv.ld + j];
      C* px = xb + (int64_t)i * X.ld + j;
      const C x = *px;
      const C nx = cadd_half(x, y);
      *px = nx;
      const C d = C{nx.x - x.x, nx.y - x.y};
      dm = fmax(dm, abs2d(d));
      am = fmax(am, abs2d(nx));
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    dm = fmax(dm, __shfl_xor_sync(0xffffffffu, dm, o));
    am = fmax(am, __shfl_xor_sync(0xffffffffu, am, o));
  }
  if (tx == 0) {
    // non-negative doubles order like their bit patterns
    atomicMax(s.dmax2 + b, (unsigned long long)__double_as_longlong(dm));
    atomicMax(s.xmax2 + b, (unsigned long long)__double_as_longlong(am));
  }
}

// The stopping rule of Sec. 5.3 after step k: stop once
// ||X_k - X_{k-1}||_max <= eps ||X_k||_max, or at step kmax.
__global__ void check_kernel(int batch, int k, int kmax, double eps, State s, int32_t* steps) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch) return;
  if (!s.done[b]) {
    steps[b] = k;
    const double d = sqrt(__longlong_as_double((long long)s.dmax2[b]));
    const double a = sqrt(__longlong_as_double((long long)s.xmax2[b]));
    if (d <= eps * a || k >= kmax) s.done[b] = 1;
    else atomicAdd(s.remaining, 1);
  }
  s.dmax2[b] = 0ull;
  s.xmax2[b] = 0ull;
}

// X0 = [[A, -C], [0, -B]] (B = A^H for the Lyapunov equation), n = p + q.
template <typename C>
__global__ void sylvester_build_kernel(int p, int q, MatB<const C> A, MatB<const C> B, bool lyap, MatB<const C> Cm,
                                       MatB<C> X0) {
  const int b = blockIdx.z;
  const int n = p + q;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * n) return;
  const int i = (int)(e / n), j = (int)(e % n);
  C v = C{0, 0};
  if (i < p && j < p) {
    v = A.at(b)[(int64_t)i * A.ld + j];
  } else if (i < p) {
    const C c = Cm.at(b)[(int64_t)i * Cm.ld + (j - p)];
    v = C{-c.x, -c.y};
  } else if (j >= p) {
    const C w = lyap ? conj_c(A.at(b)[(int64_t)(j - p) * A.ld + (i - p)]) : B.at(b)[(int64_t)(i - p) * B.ld + (j - p)];
    v = C{-w.x, -w.y};
  }
  X0.at(b)[(int64_t)i * X0.ld + j] = v;
}

// Y = -1/2 times the top-right p x q block of the limit.
template <typename C>
__global__ void sylvester_extract_kernel(int p, int q, MatB<const C> X, MatB<C> Y) {
  const int b = blockIdx.z;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)p * q) return;
  const int i = (int)(e / q), j = (int)(e % q);
  const C v = X.at(b)[(int64_t)i * X.ld + p + j];
  Y.at(b)[(int64_t)i * Y.ld + j] = C{-0.5f * v.x, -0.5f * v.y};
}

template <typename C>
__global__ void copy_kernel(int rows, int cols, MatB<const C> S, MatB<C> D) {
  const int b = blockIdx.z;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)rows * cols) return;
  const int i = (int)(e / cols), j = (int)(e % cols);
  D.at(b)[(int64_t)i * D.ld + j] = S.at(b)[(int64_t)i * S.ld + j];
}

inline size_t r256(size_t x) { return (x + 255) & ~(size_t)255; }
inline size_t elem(int prec) { return prec == FROB_FP32 ? 8 : 16; }
inline int inner_op(int route) { return route == FROB_ROUTE_CPLX_LU ? FROB_OP_CPLX_LU : FROB_OP_INV; }

// Workspace of newton_core: Xinv, the state, the inner inversion's workspace.
size_t core_ws(int n, int batch, int prec, int route) {
  const size_t inner = frob_workspace_bytes(inner_op(route), n, batch, prec);
  if (inner == 0) return 0;
  return r256((size_t)batch * n * n * elem(prec)) + 2 * r256((size_t)batch * 8) + r256((size_t)batch * 4) + 256 +
         r256((size_t)batch * sizeof(frob_info)) + inner;
}

template <typename C>
frob_status newton_core(bool polar, int route, int n, int batch, MatB<C> X, const frob_opts& o, double eps,
                        int kmax, unsigned char* ws, frob_info* info, int32_t* steps, cudaStream_t st) {
  unsigned char* w = ws;
  auto take = [&](size_t bytes) {
    unsigned char* p = w;
    w += r256(bytes);
    return p;
  };
  C* xinv = reinterpret_cast<C*>(take((size_t)batch * n * n * sizeof(C)));
  State s;
  s.dmax2 = reinterpret_cast<unsigned long long*>(take((size_t)batch * 8));
  s.xmax2 = reinterpret_cast<unsigned long long*>(take((size_t)batch * 8));
  s.done = reinterpret_cast<int*>(take((size_t)batch * 4));
  s.remaining = reinterpret_cast<int*>(take(4));
  s.inner = reinterpret_cast<frob_info*>(take((size_t)batch * sizeof(frob_info)));
  const size_t inner_bytes = frob_workspace_bytes(inner_op(route), n, batch, o.prec);
  void* inner_ws = take(inner_bytes);

  const int tb = 128, gb = (batch + tb - 1) / tb;
  // Recorded into a graph, the host cannot read the running count: every
  // step up to kmax is recorded, and the matrices that met the rule stay as
  // they are (average_kernel and check_kernel skip them), so the results and
  // step counts are those of an uncaptured call.
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  const bool captured = cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone;
  FROB_LAUNCH("newton_init", st, init_kernel<<<gb, tb, 0, st>>>(batch, s, info, steps));
  const dim3 ag((unsigned)((n + TILE - 1) / TILE), (unsigned)((n + TILE - 1) / TILE), (unsigned)batch);
  const dim3 ab(TILE, ROWS);
  MatB<const C> yv{xinv, n, (int64_t)n * n};
  for (int k = 1; k <= kmax; ++k) {
    frob_status r;
    if (route == FROB_ROUTE_CPLX_LU)
      r = cplx_lu_inv(n, batch, X.p, X.ld, X.bs, xinv, n, (int64_t)n * n, o.prec, inner_ws, inner_bytes, s.inner, st);
    else
      r = frob_inv(n, batch, X.p, X.ld, X.bs, xinv, n, (int64_t)n * n, &o, inner_ws, inner_bytes, s.inner, st);
    if (r != FROB_OK) return r;
    FROB_LAUNCH("newton_merge", st, merge_kernel<<<gb, tb, 0, st>>>(batch, s, info));
    if (polar)
      FROB_LAUNCH("newton_average<polar>", st, (average_kernel<C, true><<<ag, ab, 0, st>>>(n, X, yv, s)));
    else
      FROB_LAUNCH("newton_average<sign>", st, (average_kernel<C, false><<<ag, ab, 0, st>>>(n, X, yv, s)));
    FROB_LAUNCH("newton_check", st, check_kernel<<<gb, tb, 0, st>>>(batch, k, kmax, eps, s, steps));
    if (captured) continue;
    int rem = 0;
    if (cudaMemcpyAsync(&rem, s.remaining, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return FROB_ERR_CUDA;
    if (rem == 0) break;
  }
  return cudaGetLastError() == cudaSuccess ? FROB_OK : FROB_ERR_CUDA;
}

bool valid_route(int route) { return route == FROB_ROUTE_FROB || route == FROB_ROUTE_CPLX_LU; }

// Byte ranges of two strided batches (ra x ca and rb x cb matrices) overlap.
bool overlaps(const void* a, int64_t lda, int64_t sa, int ra, int ca, const void* b, int64_t ldb, int64_t sb, int rb,
              int cb, int batch, size_t eb) {
  auto span = [&](int64_t ld, int64_t s, int r, int c) {
    return (size_t)(((int64_t)(batch - 1) * s + (int64_t)(r - 1) * ld + c) * (int64_t)eb);
  };
  const char* pa = static_cast<const char*>(a);
  const char* pb = static_cast<const char*>(b);
  return pa < pb + span(ldb, sb, rb, cb) && pb < pa + span(lda, sa, ra, ca);
}
bool valid_prec_for(int route, int prec) {
  if (prec == FROB_FP64 || prec == FROB_FP32) return true;
  return route == FROB_ROUTE_FROB && prec == FROB_MIXED_BF16;
}

frob_opts opts_of(const frob_opts* opts) {
  frob_opts o;
  std::memset(&o, 0, sizeof(o));
  o.prec = FROB_FP64;
  o.ns_max_iter = 8;
  o.ns_tol = 1e-14;
  if (opts) o = *opts;
  o.almost_sure = 0;
  return o;
}

}  // namespace newton
}  // namespace frob

using namespace frob;
using namespace frob::newton;

extern "C" size_t frob_newton_workspace_bytes(int n, int batch, int prec, int route) {
  if (n < 1 || batch < 1 || !valid_route(route) || !valid_prec_for(route, prec)) return 0;
  return core_ws(n, batch, prec, route);
}

extern "C" frob_status frob_newton(int kind, int route, int n, int batch, const void* M, int64_t ldm, int64_t sm,
                                   void* X, int64_t ldx, int64_t sx, const frob_opts* opts, double eps, int kmax,
                                   void* ws, size_t wsb, frob_info* info, int32_t* steps, void* stream) {
  frob_opts o = opts_of(opts);
  if ((kind != FROB_NEWTON_SIGN && kind != FROB_NEWTON_POLAR) || !valid_route(route)) return FROB_ERR_ARG;
  if (!valid_prec_for(route, o.prec)) return FROB_ERR_UNSUPPORTED;
  if (n < 1 || batch < 1 || batch > 65535 || kmax < 0 || !(eps >= 0.0)) return FROB_ERR_ARG;
  if (!M || !X || !info || !steps || ldm < n || ldx < n) return FROB_ERR_ARG;
  if (batch > 1 && (sm < ldm * (int64_t)n || sx < ldx * (int64_t)n)) return FROB_ERR_ARG;
  const bool same = M == X && ldm == ldx && (batch == 1 || sm == sx);
  if (!same && overlaps(M, ldm, sm, n, n, X, ldx, sx, n, n, batch, elem(o.prec))) return FROB_ERR_ARG;
  const size_t need = core_ws(n, batch, o.prec, route);
  if (need == 0) return FROB_ERR_UNSUPPORTED;
  if (!ws || wsb < need || (reinterpret_cast<uintptr_t>(ws) & 255)) return FROB_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const dim3 eg((unsigned)(((int64_t)n * n + 255) / 256), 1, (unsigned)batch);
  if (o.prec == FROB_FP32) {
    FROB_LAUNCH("newton_copy", st,
                copy_kernel<zf><<<eg, 256, 0, st>>>(n, n, MatB<const zf>{static_cast<const zf*>(M), ldm, sm},
                                                    MatB<zf>{static_cast<zf*>(X), ldx, sx}));
    return newton_core<zf>(kind == FROB_NEWTON_POLAR, route, n, batch, MatB<zf>{static_cast<zf*>(X), ldx, sx}, o, eps,
                           kmax, static_cast<unsigned char*>(ws), info, steps, st);
  }
  FROB_LAUNCH("newton_copy", st,
              copy_kernel<zd><<<eg, 256, 0, st>>>(n, n, MatB<const zd>{static_cast<const zd*>(M), ldm, sm},
                                                  MatB<zd>{static_cast<zd*>(X), ldx, sx}));
  return newton_core<zd>(kind == FROB_NEWTON_POLAR, route, n, batch, MatB<zd>{static_cast<zd*>(X), ldx, sx}, o, eps,
                         kmax, static_cast<unsigned char*>(ws), info, steps, st);
}

extern "C" size_t frob_sylvester_workspace_bytes(int p, int q, int batch, int prec, int route) {
  if (p < 1 || q < 1 || batch < 1 || !valid_route(route) || !valid_prec_for(route, prec)) return 0;
  const size_t core = core_ws(p + q, batch, prec, route);
  return core == 0 ? 0 : r256((size_t)batch * (p + q) * (p + q) * elem(prec)) + core;
}

extern "C" frob_status frob_sylvester(int route, int p, int q, int batch, const void* A, int64_t lda, int64_t sa,
                                      const void* B, int64_t ldb, int64_t sb, int lyapunov, const void* C,
                                      int64_t ldc, int64_t sc, void* Y, int64_t ldy, int64_t sy,
                                      const frob_opts* opts, double eps, int kmax, void* ws, size_t wsb,
                                      frob_info* info, int32_t* steps, void* stream) {
  frob_opts o = opts_of(opts);
  if (!valid_route(route) || (lyapunov != 0 && lyapunov != 1)) return FROB_ERR_ARG;
  if (!valid_prec_for(route, o.prec)) return FROB_ERR_UNSUPPORTED;
  if (p < 1 || q < 1 || batch < 1 || batch > 65535 || kmax < 0 || !(eps >= 0.0)) return FROB_ERR_ARG;
  if (lyapunov && p != q) return FROB_ERR_ARG;
  if (!A || (!lyapunov && !B) || !C || !Y || !info || !steps) return FROB_ERR_ARG;
  if (lda < p || (!lyapunov && ldb < q) || ldc < q || ldy < q) return FROB_ERR_ARG;
  if (batch > 1 && (sa < lda * (int64_t)p || (!lyapunov && sb < ldb * (int64_t)q) || sc < ldc * (int64_t)p ||
                    sy < ldy * (int64_t)p))
    return FROB_ERR_ARG;
  const int n = p + q;
  {
    const size_t eb = elem(o.prec);
    if (overlaps(Y, ldy, sy, p, q, A, lda, sa, p, p, batch, eb) || overlaps(Y, ldy, sy, p, q, C, ldc, sc, p, q, batch, eb) ||
        (!lyapunov && overlaps(Y, ldy, sy, p, q, B, ldb, sb, q, q, batch, eb)))
      return FROB_ERR_ARG;
  }
  const size_t need = frob_sylvester_workspace_bytes(p, q, batch, o.prec, route);
  if (need == 0) return FROB_ERR_UNSUPPORTED;
  if (!ws || wsb < need || (reinterpret_cast<uintptr_t>(ws) & 255)) return FROB_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned char* w = static_cast<unsigned char*>(ws);
  unsigned char* core = w + r256((size_t)batch * n * n * elem(o.prec));
  const dim3 bg((unsigned)(((int64_t)n * n + 255) / 256), 1, (unsigned)batch);
  const dim3 yg((unsigned)(((int64_t)p * q + 255) / 256), 1, (unsigned)batch);
  const int64_t nn = (int64_t)n * n;
  frob_status r;
  if (o.prec == FROB_FP32) {
    MatB<zf> X0{reinterpret_cast<zf*>(w), n, nn};
    FROB_LAUNCH("sylvester_build", st,
                sylvester_build_kernel<zf><<<bg, 256, 0, st>>>(
                    p, q, MatB<const zf>{static_cast<const zf*>(A), lda, sa},
                    MatB<const zf>{static_cast<const zf*>(B), ldb, sb}, lyapunov != 0,
                    MatB<const zf>{static_cast<const zf*>(C), ldc, sc}, X0));
    r = newton_core<zf>(false, route, n, batch, X0, o, eps, kmax, core, info, steps, st);
    FROB_LAUNCH("sylvester_extract", st,
                sylvester_extract_kernel<zf><<<yg, 256, 0, st>>>(p, q, MatB<const zf>{X0.p, n, nn},
                                                                 MatB<zf>{static_cast<zf*>(Y), ldy, sy}));
  } else {
    MatB<zd> X0{reinterpret_cast<zd*>(w), n, nn};
    FROB_LAUNCH("sylvester_build", st,
                sylvester_build_kernel<zd><<<bg, 256, 0, st>>>(
                    p, q, MatB<const zd>{static_cast<const zd*>(A), lda, sa},
                    MatB<const zd>{static_cast<const zd*>(B), ldb, sb}, lyapunov != 0,
                    MatB<const zd>{static_cast<const zd*>(C), ldc, sc}, X0));
    r = newton_core<zd>(false, route, n, batch, X0, o, eps, kmax, core, info, steps, st);
    FROB_LAUNCH("sylvester_extract", st,
                sylvester_extract_kernel<zd><<<yg, 256, 0, st>>>(p, q, MatB<const zd>{X0.p, n, nn},
                                                                 MatB<zd>{static_cast<zd*>(Y), ldy, sy}));
  }
  if (r != FROB_OK) return r;
  return cudaGetLastError() == cudaSuccess ? FROB_OK : FROB_ERR_CUDA;
}

extern "C" size_t frob_polar_workspace_bytes(int n, int batch, int prec, int route) {
  return frob_newton_workspace_bytes(n, batch, prec, route);
}

extern "C" frob_status frob_polar(int route, int n, int batch, const void* X, int64_t ldx, int64_t sx, void* Q,
                                  int64_t ldq, int64_t sq, void* P, int64_t ldp, int64_t sp, const frob_opts* opts,
                                  double eps, int kmax, void* ws, size_t wsb, frob_info* info, int32_t* steps,
                                  void* stream) {
  if (!P || !Q || !X || ldp < n || (batch > 1 && sp < ldp * (int64_t)n)) return FROB_ERR_ARG;
  {
    const size_t eb = elem(opts_of(opts).prec);
    if (overlaps(X, ldx, sx, n, n, Q, ldq, sq, n, n, batch, eb) || overlaps(X, ldx, sx, n, n, P, ldp, sp, n, n, batch, eb) ||
        overlaps(Q, ldq, sq, n, n, P, ldp, sp, n, n, batch, eb))
      return FROB_ERR_ARG;
  }
  frob_status r = frob_newton(FROB_NEWTON_POLAR, route, n, batch, X, ldx, sx, Q, ldq, sq, opts, eps, kmax, ws, wsb,
                              info, steps, stream);
  if (r != FROB_OK) return r;
  // P = Q^H X
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const frob_opts o = opts_of(opts);
  if (o.prec == FROB_FP32) {
    MatB<zf> Pm{static_cast<zf*>(P), ldp, sp};
    gemm_launch<zf, OP_C, OP_N>(n, n, n, batch, MatB<const zf>{static_cast<const zf*>(Q), ldq, sq},
                                MatB<const zf>{static_cast<const zf*>(X), ldx, sx},
                                axpby<zf>(Pm, zf{1.f, 0.f}, zf{0.f, 0.f}, true), 0, st);
  } else {
    MatB<zd> Pm{static_cast<zd*>(P), ldp, sp};
    gemm_launch<zd, OP_C, OP_N>(n, n, n, batch, MatB<const zd>{static_cast<const zd*>(Q), ldq, sq},
                                MatB<const zd>{static_cast<const zd*>(X), ldx, sx},
                                axpby<zd>(Pm, zd{1.0, 0.0}, zd{0.0, 0.0}, true), 0, st);
  }
  return cudaGetLastError() == cudaSuccess ? FROB_OK : FROB_ERR_CUDA;
}
