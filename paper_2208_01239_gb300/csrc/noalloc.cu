// frob_inv_hpd_noalloc: the Hermitian positive definite Frobenius inversion
// (same kernels as frob_inv_hpd, FP64) running in scratch memory that the
// library itself owns, for callers that cannot allocate device memory.
//
// Who needs this: code that runs where a device allocation is not allowed or
// not affordable -- a plugin or callback inside a host framework that owns
// every device buffer through its own pool and hands out only the input and
// output tensors; a latency-bound loop (for example a detector in a radio
// receive chain that inverts small HPD channel matrices every slot) where a
// cudaMalloc may synchronise the device and break the time budget; or a
// foreign-language caller with no device allocator at hand.  Such a caller
// passes only inputs, outputs and the info records; the workspace comes from
// the fixed array below.
//
// The array is a file-scope __device__ object of SCRATCH_BYTES bytes: every
// GPU that loads this library holds it until the process exits.  Host code
// must not take its name as a device address (in host code the name denotes
// a host-side stand-in), so the device address is fetched once per device
// with cudaGetSymbolAddress, with that device current, and passed to the
// kernels as their workspace.
#include <cstdint>
#include <mutex>
#include <cuda_runtime.h>

#include "../../include/frobinv.h"
#include "common.cuh"
#include "ops.h"

namespace {

constexpr size_t SCRATCH_BYTES = size_t(32) << 20;  // 32 MiB
constexpr int MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_scratch[SCRATCH_BYTES];

std::mutex g_mu;
void* g_addr[MAX_DEVICES] = {};

// Device address of g_scratch on the current device, looked up on the first
// call made with that device current and cached afterwards.
frob_status scratch_on_current_device(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return FROB_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_addr[dev] == nullptr) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || p == nullptr) return FROB_ERR_CUDA;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return FROB_OK;
}

bool ranges_overlap(const void* a, int64_t lda, int64_t sa, const void* b, int64_t ldb, int64_t sb, int n,
                    int batch) {
  auto span = [&](int64_t ld, int64_t s) { return (size_t)(((int64_t)(batch - 1) * s + (int64_t)(n - 1) * ld + n) * 16); };
  const char* pa = static_cast<const char*>(a);
  const char* pb = static_cast<const char*>(b);
  return pa < pb + span(ldb, sb) && pb < pa + span(lda, sa);
}

}  // namespace

extern "C" frob_status frob_inv_hpd_noalloc(int n, int batch, const void* M, int64_t ldm, int64_t sm, void* X,
                                            int64_t ldx, int64_t sx, frob_info* info, void* stream) {
  if (n < 1 || batch < 1 || batch > 65535 || !M || !X || !info) return FROB_ERR_ARG;
  if (ldm < n || ldx < n) return FROB_ERR_ARG;
  if (batch > 1 && (sm < ldm * (int64_t)n || sx < ldx * (int64_t)n)) return FROB_ERR_ARG;
  if (ranges_overlap(M, ldm, sm, X, ldx, sx, n, batch)) return FROB_ERR_ARG;
  const size_t need = frob_workspace_bytes(FROB_OP_INV_HPD, n, batch, FROB_FP64);
  if (need == 0) return FROB_ERR_ARG;
  if (need > SCRATCH_BYTES) return FROB_ERR_WORKSPACE;  // problem larger than the fixed scratch
  void* ws = nullptr;
  frob_status s = scratch_on_current_device(&ws);
  if (s != FROB_OK) return s;
  // An error left pending by an earlier runtime call of this thread is not
  // this call's: clear it so that the check after the launches sees only
  // their own status (a sticky error would make the launches fail anyway).
  (void)cudaGetLastError();
  // Every scratch byte the kernels read is first written by this same call
  // (the split writes A, S and B; the identity solve writes every tile of
  // its output, zeros included), so nothing has to be cleared between calls.
  frob::frob_chol_run<double>(n, batch, frob::MatB<const frob::zd>{static_cast<const frob::zd*>(M), ldm, sm},
                              frob::MatB<frob::zd>{static_cast<frob::zd*>(X), ldx, sx}, ws, info,
                              static_cast<cudaStream_t>(stream));
  return cudaGetLastError() == cudaSuccess ? FROB_OK : FROB_ERR_CUDA;
}
