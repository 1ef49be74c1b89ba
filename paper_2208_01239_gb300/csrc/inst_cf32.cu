// Explicit instantiation of the complex-arithmetic baselines for zf.
#include "ops_impl.cuh"

namespace frob {
template size_t cplx_lu_ws<zf>(int, int, void*, CPlanes<zf>*);
template void cplx_lu_run<zf>(int, int, MatB<const zf>, MatB<zf>, void*, frob_info*, cudaStream_t);
template size_t cplx_chol_ws<zf>(int, int, void*, CPlanes<zf>*);
template void cplx_chol_run<zf>(int, int, MatB<const zf>, MatB<zf>, void*, frob_info*, cudaStream_t);
template size_t cplx_solve_ws<zf>(int, int, int);
template void cplx_solve_run<zf>(int, int, int, MatB<const zf>, MatB<const zf>, MatB<zf>, void*, frob_info*,
                                  cudaStream_t);
}  // namespace frob
