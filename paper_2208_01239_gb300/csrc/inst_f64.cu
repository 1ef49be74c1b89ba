// Explicit instantiation of the inversion drivers for double / zd.
#include "ops_impl.cuh"

namespace frob {
template size_t frob_lu_ws<double>(int, int, void*, Planes<double>*);
template void frob_lu_run<double>(int, int, MatB<const zd>, MatB<zd>, const frob_opts&, void*, frob_info*, cudaStream_t);
template size_t frob_chol_ws<double>(int, int, void*, Planes<double>*);
template void frob_chol_run<double>(int, int, MatB<const zd>, MatB<zd>, void*, frob_info*, cudaStream_t, int);
template size_t adjoint_ws<double>(int, int);
template void adjoint_run<double>(int, int, MatB<const zd>, MatB<const zd>, MatB<zd>, void*, cudaStream_t);
template size_t frob_solve_ws<double>(int, int, int, SolvePlanes<double>*, void*);
template void frob_solve_run<double>(int, int, int, MatB<const zd>, MatB<const zd>, MatB<zd>, void*, frob_info*,
                                  cudaStream_t);
template size_t aug_solve_ws<double>(int, int, int);
template void aug_solve_run<double>(int, int, int, MatB<const zd>, MatB<const zd>, MatB<zd>, void*, frob_info*,
                                 cudaStream_t);
}  // namespace frob
