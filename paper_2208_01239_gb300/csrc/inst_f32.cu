// Explicit instantiation of the inversion drivers for float / zf.
#include "ops_impl.cuh"

namespace frob {
template size_t frob_lu_ws<float>(int, int, void*, Planes<float>*);
template void frob_lu_run<float>(int, int, MatB<const zf>, MatB<zf>, const frob_opts&, void*, frob_info*, cudaStream_t);
template size_t frob_chol_ws<float>(int, int, void*, Planes<float>*);
template void frob_chol_run<float>(int, int, MatB<const zf>, MatB<zf>, void*, frob_info*, cudaStream_t, int);
template size_t adjoint_ws<float>(int, int);
template void adjoint_run<float>(int, int, MatB<const zf>, MatB<const zf>, MatB<zf>, void*, cudaStream_t);
template size_t frob_solve_ws<float>(int, int, int, SolvePlanes<float>*, void*);
template void frob_solve_run<float>(int, int, int, MatB<const zf>, MatB<const zf>, MatB<zf>, void*, frob_info*,
                                  cudaStream_t);
template size_t aug_solve_ws<float>(int, int, int);
template void aug_solve_run<float>(int, int, int, MatB<const zf>, MatB<const zf>, MatB<zf>, void*, frob_info*,
                                 cudaStream_t);
}  // namespace frob
