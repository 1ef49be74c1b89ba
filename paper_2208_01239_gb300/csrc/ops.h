// Declarations shared between the per-precision instantiation units and the
// C-ABI entry points.
#pragma once

#include <cstddef>
#include <cuda_runtime.h>

#include "common.cuh"

namespace frob {

// Set while the mixed precisions compute their FP32 start: its products stay
// on the CUDA cores, whose FP32 rounding gives the refinement a closer start
// than split-TF32 products with tensor-core accumulation (measured: fewer
// Newton-Schulz steps on the HPD workload).
inline thread_local bool t_tc_off = false;
struct TcOff {
  bool saved;
  TcOff() : saved(t_tc_off) { t_tc_off = true; }
  ~TcOff() { t_tc_off = saved; }
};
// bytes an FP32 driver reserves for its largest tensor-core product (order n,
// K = n): the two split operands of tc_gemm.cuh's split-TF32 form
size_t tc_scratch_for(int n, int batch);

template <typename R> struct cplx_of;
template <> struct cplx_of<double> { using type = zd; };
template <> struct cplx_of<float> { using type = zf; };

// Workspace planes of the Frobenius routines (real, n x n per matrix).
template <typename R> struct Planes {
  MatB<R> LA, S, Bp, X1, Y;
  int *piv1, *piv2, *rp1, *rp2;
  int* partb;         // [batch] 1: B factored (frob_lu_run)
  frob_info* infoB;   // [batch] status of the LU of B (FROB_PART_AUTO)
  unsigned char* mcs = nullptr;  // scratch of the multi-CTA LU panels (0 bytes when unused)
  unsigned char* tcs = nullptr;  // scratch of the FP32 tensor-core products (0 bytes when unused)
  size_t tcs_bytes = 0;
};
// Workspace of the complex baselines.
template <typename C> struct CPlanes {
  MatB<C> W, Y;
  int *piv, *rp;
  unsigned char* mcs = nullptr;  // scratch of the multi-CTA LU panels (0 bytes when unused)
};

template <typename R> size_t frob_lu_ws(int n, int batch, void* ws, Planes<R>* out);
template <typename R>
void frob_lu_run(int n, int batch, MatB<const typename cplx_of<R>::type> M, MatB<typename cplx_of<R>::type> X,
                 const frob_opts& o, void* ws, frob_info* info, cudaStream_t st);
template <typename R> size_t frob_chol_ws(int n, int batch, void* ws, Planes<R>* out);
template <typename R>
void frob_chol_run(int n, int batch, MatB<const typename cplx_of<R>::type> M, MatB<typename cplx_of<R>::type> X,
                   void* ws, frob_info* info, cudaStream_t st, int fp64_gemm = FROB_GEMM_AUTO);
template <typename C> size_t cplx_lu_ws(int n, int batch, void* ws, CPlanes<C>* out);
template <typename C> void cplx_lu_run(int n, int batch, MatB<const C> M, MatB<C> X, void* ws, frob_info* info,
                                       cudaStream_t st);
template <typename C> size_t cplx_chol_ws(int n, int batch, void* ws, CPlanes<C>* out);
template <typename C> void cplx_chol_run(int n, int batch, MatB<const C> M, MatB<C> X, void* ws, frob_info* info,
                                         cudaStream_t st);

template <typename R> struct SolvePlanes;
template <typename R> size_t frob_solve_ws(int n, int nrhs, int batch, SolvePlanes<R>* out, void* ws);
template <typename R>
void frob_solve_run(int n, int nrhs, int batch, MatB<const typename cplx_of<R>::type> M,
                    MatB<const typename cplx_of<R>::type> Bc, MatB<typename cplx_of<R>::type> X, void* ws,
                    frob_info* info, cudaStream_t st);
template <typename C> size_t cplx_solve_ws(int n, int nrhs, int batch);
template <typename R> size_t aug_solve_ws(int n, int nrhs, int batch);
template <typename R>
void aug_solve_run(int n, int nrhs, int batch, MatB<const typename cplx_of<R>::type> M,
                   MatB<const typename cplx_of<R>::type> Bc, MatB<typename cplx_of<R>::type> X, void* ws,
                   frob_info* info, cudaStream_t st);
template <typename C>
void cplx_solve_run(int n, int nrhs, int batch, MatB<const C> M, MatB<const C> Bc, MatB<C> X, void* ws,
                    frob_info* info, cudaStream_t st);

template <typename R> size_t adjoint_ws(int n, int batch);
template <typename R>
void adjoint_run(int n, int batch, MatB<const typename cplx_of<R>::type> X, MatB<const typename cplx_of<R>::type> G,
                 MatB<typename cplx_of<R>::type> out, void* ws, cudaStream_t st);

namespace mixed {
// Mixed-precision Frobenius inversion with Newton-Schulz refinement (n <= 512);
// complex_start: the FP32 start is complex LU / Cholesky inversion instead
// (the control that separates the refinement's gain from Frobenius's).
size_t mixed_ws(int n, int batch);
frob_status mixed_run(int n, int batch, MatB<const zd> M, MatB<zd> X, const frob_opts& o, void* ws, frob_info* info,
                      cudaStream_t st, bool hpd, bool complex_start = false);
}  // namespace mixed

}  // namespace frob
