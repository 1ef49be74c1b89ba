// Explicit instantiation of the complex-arithmetic baselines for zd.
#include "ops_impl.cuh"

namespace frob {
template size_t cplx_lu_ws<zd>(int, int, void*, CPlanes<zd>*);
template void cplx_lu_run<zd>(int, int, MatB<const zd>, MatB<zd>, void*, frob_info*, cudaStream_t);
template size_t cplx_chol_ws<zd>(int, int, void*, CPlanes<zd>*);
template void cplx_chol_run<zd>(int, int, MatB<const zd>, MatB<zd>, void*, frob_info*, cudaStream_t);
template size_t cplx_solve_ws<zd>(int, int, int);
template void cplx_solve_run<zd>(int, int, int, MatB<const zd>, MatB<const zd>, MatB<zd>, void*, frob_info*,
                                  cudaStream_t);
}  // namespace frob
