// Inversion over an iterated quadratic extension (Sec. 2.4, Theorem "GFiter")
// for m = 2 with xi_1^2 = xi_2^2 = -1: bicomplex matrices X = A + jB, A and B
// complex, j^2 = -1 and j commuting with i.  Frobenius inversion over
// F_1 = C (Algorithm "Frobenius inversion", tau = 1):
//   X1 = A^{-1}; X2 = X1 B; X4 = A + B X2; X5 = X4^{-1}; X6 = X2 X5;
//   X^{-1} = X5 - j X6,
// with each complex inversion a Frobenius inversion over R (frob_inv) and
// each complex product by Gauss's three real multiplications (Proposition
// "matrix mult"): 3 x 3 + 2 x 3 = 15 = 3 (3^2 - 2^2) real products and
// 2 x 2 = 4 real inversions, as the theorem counts.
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/frobinv.h"
#include "common.cuh"
#include "ops_impl.cuh"

namespace frob {
namespace iqe {

// Gauss multiplication: (Ar + i Ai)(Br + i Bi) with T1 = Ar Br, T2 = Ai Bi,
// T3 = (Ar + Ai)(Br + Bi); real part T1 - T2, imaginary part T3 - T1 - T2.
template <typename R>
__global__ void gauss_split_kernel(int n, MatB<const typename cplx_of<R>::type> A,
                                   MatB<const typename cplx_of<R>::type> B, MatB<R> Ar, MatB<R> Ai, MatB<R> As,
                                   MatB<R> Br, MatB<R> Bi, MatB<R> Bs) {
  const int b = blockIdx.z;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * n) return;
  const int i = (int)(e / n), j = (int)(e % n);
  const auto a = A.at(b)[(int64_t)i * A.ld + j];
  const auto v = B.at(b)[(int64_t)i * B.ld + j];
  const int64_t o = (int64_t)i * n + j;
  Ar.at(b)[o] = a.x;
  Ai.at(b)[o] = a.y;
  As.at(b)[o] = a.x + a.y;
  Br.at(b)[o] = v.x;
  Bi.at(b)[o] = v.y;
  Bs.at(b)[o] = v.x + v.y;
}

// Out = sign * (T1 - T2 + i (T3 - T1 - T2)) + Add (Add.p may be NULL).
template <typename R>
__global__ void gauss_combine_kernel(int n, MatB<const R> T1, MatB<const R> T2, MatB<const R> T3,
                                     MatB<const typename cplx_of<R>::type> Add, R sign,
                                     MatB<typename cplx_of<R>::type> Out) {
  const int b = blockIdx.z;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * n) return;
  const int i = (int)(e / n), j = (int)(e % n);
  const int64_t o = (int64_t)i * n + j;
  const R t1 = T1.at(b)[o], t2 = T2.at(b)[o], t3 = T3.at(b)[o];
  typename cplx_of<R>::type r;
  r.x = sign * (t1 - t2);
  r.y = sign * (t3 - t1 - t2);
  if (Add.p) {
    const auto a = Add.at(b)[(int64_t)i * Add.ld + j];
    r.x += a.x;
    r.y += a.y;
  }
  Out.at(b)[(int64_t)i * Out.ld + j] = r;
}

// The second inversion's failure (if the first succeeded) becomes the
// result's, its step index shifted past the first inversion's 2n steps.
__global__ void merge_info_kernel(int n, int batch, const frob_info* second, frob_info* info) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch || info[b].status != FROB_OK || second[b].status == FROB_OK) return;
  frob_info f = second[b];
  f.bad_index += 2 * n;
  info[b] = f;
}

inline size_t r256(size_t x) { return (x + 255) & ~(size_t)255; }

template <typename R> struct Work {
  using C = typename cplx_of<R>::type;
  MatB<C> X1, X2, X4;
  MatB<R> P[9];  // Ar Ai As Br Bi Bs T1 T2 T3
  frob_info* info2;
  unsigned char* inner;
  size_t inner_bytes;
};

template <typename R> size_t work_bytes(int n, int batch, int prec) {
  using C = typename cplx_of<R>::type;
  const size_t inner = frob_workspace_bytes(FROB_OP_INV, n, batch, prec);
  if (inner == 0) return 0;
  return 3 * r256((size_t)batch * n * n * sizeof(C)) + 9 * r256((size_t)batch * n * n * sizeof(R)) +
         r256((size_t)batch * sizeof(frob_info)) + inner;
}

template <typename R> Work<R> carve(int n, int batch, int prec, unsigned char* ws) {
  using C = typename cplx_of<R>::type;
  Work<R> w;
  unsigned char* p = ws;
  const int64_t nn = (int64_t)n * n;
  auto takec = [&]() {
    MatB<C> m{reinterpret_cast<C*>(p), n, nn};
    p += r256((size_t)batch * nn * sizeof(C));
    return m;
  };
  w.X1 = takec();
  w.X2 = takec();
  w.X4 = takec();
  for (int k = 0; k < 9; ++k) {
    w.P[k] = MatB<R>{reinterpret_cast<R*>(p), n, nn};
    p += r256((size_t)batch * nn * sizeof(R));
  }
  w.info2 = reinterpret_cast<frob_info*>(p);
  p += r256((size_t)batch * sizeof(frob_info));
  w.inner = p;
  w.inner_bytes = frob_workspace_bytes(FROB_OP_INV, n, batch, prec);
  return w;
}

// Out = sign * A B + Add by Gauss multiplication.
template <typename R>
void gauss_mul(int n, int batch, MatB<const typename cplx_of<R>::type> A, MatB<const typename cplx_of<R>::type> B,
               MatB<const typename cplx_of<R>::type> Add, R sign, MatB<typename cplx_of<R>::type> Out,
               Work<R>& w, cudaStream_t st) {
  auto cst = [](MatB<R> m) { return MatB<const R>{m.p, m.ld, m.bs}; };
  const dim3 g((unsigned)(((int64_t)n * n + 255) / 256), 1, (unsigned)batch);
  FROB_LAUNCH("gauss_split", st,
              gauss_split_kernel<R><<<g, 256, 0, st>>>(n, A, B, w.P[0], w.P[1], w.P[2], w.P[3], w.P[4], w.P[5]));
  gemm_launch<R, OP_N, OP_N>(n, n, n, batch, cst(w.P[0]), cst(w.P[3]), axpby<R>(w.P[6], (R)1, (R)0, true), 0, st);
  gemm_launch<R, OP_N, OP_N>(n, n, n, batch, cst(w.P[1]), cst(w.P[4]), axpby<R>(w.P[7], (R)1, (R)0, true), 0, st);
  gemm_launch<R, OP_N, OP_N>(n, n, n, batch, cst(w.P[2]), cst(w.P[5]), axpby<R>(w.P[8], (R)1, (R)0, true), 0, st);
  FROB_LAUNCH("gauss_combine", st,
              gauss_combine_kernel<R><<<g, 256, 0, st>>>(n, cst(w.P[6]), cst(w.P[7]), cst(w.P[8]), Add, sign, Out));
}

template <typename R>
frob_status run(int n, int batch, MatB<const typename cplx_of<R>::type> A, MatB<const typename cplx_of<R>::type> B,
                MatB<typename cplx_of<R>::type> Y0, MatB<typename cplx_of<R>::type> Y1, const frob_opts& o,
                unsigned char* ws, frob_info* info, cudaStream_t st) {
  using C = typename cplx_of<R>::type;
  Work<R> w = carve<R>(n, batch, o.prec, ws);
  auto cc = [](MatB<C> m) { return MatB<const C>{m.p, m.ld, m.bs}; };
  const MatB<const C> none{nullptr, 0, 0};
  frob_status r = frob_inv(n, batch, A.p, A.ld, A.bs, w.X1.p, n, (int64_t)n * n, &o, w.inner, w.inner_bytes, info,
                           st);  // X1 = A^{-1}
  if (r != FROB_OK) return r;
  gauss_mul<R>(n, batch, cc(w.X1), B, none, (R)1, w.X2, w, st);  // X2 = X1 B
  gauss_mul<R>(n, batch, B, cc(w.X2), A, (R)1, w.X4, w, st);     // X4 = A + B X2
  r = frob_inv(n, batch, w.X4.p, n, (int64_t)n * n, Y0.p, Y0.ld, Y0.bs, &o, w.inner, w.inner_bytes, w.info2,
               st);  // X5 = X4^{-1}, written to Y0
  if (r != FROB_OK) return r;
  gauss_mul<R>(n, batch, cc(w.X2), cc(Y0), none, (R)-1, Y1, w, st);  // Y1 = -X6 = -X2 X5
  FROB_LAUNCH("iqe_merge_info", st, merge_info_kernel<<<(batch + 127) / 128, 128, 0, st>>>(n, batch, w.info2, info));
  return cudaGetLastError() == cudaSuccess ? FROB_OK : FROB_ERR_CUDA;
}

bool disjoint(const void* a, int64_t lda, int64_t sa, const void* b, int64_t ldb, int64_t sb, int n, int batch,
              size_t eb) {
  auto span = [&](int64_t ld, int64_t s) { return (size_t)(((int64_t)(batch - 1) * s + (int64_t)(n - 1) * ld + n) * (int64_t)eb); };
  const char* pa = static_cast<const char*>(a);
  const char* pb = static_cast<const char*>(b);
  return !(pa < pb + span(ldb, sb) && pb < pa + span(lda, sa));
}

}  // namespace iqe
}  // namespace frob

using namespace frob;

extern "C" size_t frob_inv_bicomplex_workspace_bytes(int n, int batch, int prec) {
  if (n < 1 || batch < 1) return 0;
  return prec == FROB_FP32 ? iqe::work_bytes<float>(n, batch, prec) : iqe::work_bytes<double>(n, batch, prec);
}

extern "C" frob_status frob_inv_bicomplex(int n, int batch, const void* A, int64_t lda, int64_t sa, const void* B,
                                          int64_t ldb, int64_t sb, void* Y0, int64_t ldy0, int64_t sy0, void* Y1,
                                          int64_t ldy1, int64_t sy1, const frob_opts* opts, void* ws, size_t wsb,
                                          frob_info* info, void* stream) {
  frob_opts o{};
  o.prec = FROB_FP64;
  o.ns_max_iter = 8;
  o.ns_tol = 1e-14;
  if (opts) o = *opts;
  if (o.almost_sure || o.part != FROB_PART_A) return FROB_ERR_ARG;
  if (n < 1 || batch < 1 || batch > 65535 || !A || !B || !Y0 || !Y1 || !info) return FROB_ERR_ARG;
  if (lda < n || ldb < n || ldy0 < n || ldy1 < n) return FROB_ERR_ARG;
  if (batch > 1 && (sa < lda * (int64_t)n || sb < ldb * (int64_t)n || sy0 < ldy0 * (int64_t)n ||
                    sy1 < ldy1 * (int64_t)n))
    return FROB_ERR_ARG;
  const size_t eb = o.prec == FROB_FP32 ? 8 : 16;
  const void* ins[2] = {A, B};
  const int64_t ild[2] = {lda, ldb}, ist[2] = {sa, sb};
  for (int k = 0; k < 2; ++k)
    if (!iqe::disjoint(ins[k], ild[k], ist[k], Y0, ldy0, sy0, n, batch, eb) ||
        !iqe::disjoint(ins[k], ild[k], ist[k], Y1, ldy1, sy1, n, batch, eb))
      return FROB_ERR_ARG;
  if (!iqe::disjoint(Y0, ldy0, sy0, Y1, ldy1, sy1, n, batch, eb)) return FROB_ERR_ARG;
  const size_t need = frob_inv_bicomplex_workspace_bytes(n, batch, o.prec);
  if (need == 0) return FROB_ERR_UNSUPPORTED;
  if (!ws || wsb < need || (reinterpret_cast<uintptr_t>(ws) & 255)) return FROB_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned char* w = static_cast<unsigned char*>(ws);
  if (o.prec == FROB_FP32)
    return iqe::run<float>(n, batch, MatB<const zf>{static_cast<const zf*>(A), lda, sa},
                           MatB<const zf>{static_cast<const zf*>(B), ldb, sb}, MatB<zf>{static_cast<zf*>(Y0), ldy0, sy0},
                           MatB<zf>{static_cast<zf*>(Y1), ldy1, sy1}, o, w, info, st);
  return iqe::run<double>(n, batch, MatB<const zd>{static_cast<const zd*>(A), lda, sa},
                          MatB<const zd>{static_cast<const zd*>(B), ldb, sb}, MatB<zd>{static_cast<zd*>(Y0), ldy0, sy0},
                          MatB<zd>{static_cast<zd*>(Y1), ldy1, sy1}, o, w, info, st);
}
