// Batched inversion of matrices of different orders in one call.
//
// Every matrix M_i (order n_i) is embedded as M_i (+) cI in a bucket of order
// N = 32 ceil(n_i / 32): (M (+) cI)^{-1} = M^{-1} (+) c^{-1} I, the padding
// block never takes part in pivoting (its columns hold a single nonzero on
// the diagonal).  c = 1 keeps Hermitian positive definite input Hermitian
// positive definite; with the part options of frob_inv c = i (B factored) or
// 1 + i (either part), so that the factored real part of the padding is
// invertible.
// Each bucket then runs the uniform strided-batch path (frob_inv,
// frob_inv_hpd or a baseline), and the results and info records are
// scattered back.  The slot of each matrix in its bucket is computed on the
// device from the device copy of the orders, so a call is a fixed sequence of
// kernel launches on one stream (it can be captured in a CUDA graph once the
// first call on the device has run).  Buckets are processed largest first.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>
#include <cuda_runtime.h>

#include "../../include/frobinv.h"
#include "common.cuh"
#include "ops.h"

namespace frob {
namespace batched {

constexpr int GRAN = 32;
constexpr int MAX_BUCKETS = 64;

struct Plan {
  int nb = 0;
  int N[MAX_BUCKETS];
  int count[MAX_BUCKETS];
  int offset[MAX_BUCKETS];
};

struct BucketTable {
  int nb;
  int N[MAX_BUCKETS];
  int offset[MAX_BUCKETS];
};

__host__ __device__ inline int padded(int n) { return ((n + GRAN - 1) / GRAN) * GRAN; }

bool make_plan(int batch, const int32_t* n_host, Plan& p) {
  std::vector<int> sizes;
  for (int i = 0; i < batch; ++i) {
    if (n_host[i] < 1) return false;
    sizes.push_back(padded(n_host[i]));
  }
  std::vector<int> uniq = sizes;
  std::sort(uniq.begin(), uniq.end(), std::greater<int>());
  uniq.erase(std::unique(uniq.begin(), uniq.end()), uniq.end());
  if ((int)uniq.size() > MAX_BUCKETS) return false;
  p.nb = (int)uniq.size();
  int off = 0;
  for (int b = 0; b < p.nb; ++b) {
    p.N[b] = uniq[b];
    p.count[b] = (int)std::count(sizes.begin(), sizes.end(), uniq[b]);
    p.offset[b] = off;
    off += p.count[b];
  }
  return true;
}

size_t elem_size(int prec) { return prec == FROB_FP32 ? 8 : 16; }

size_t sub_ws(int op, int N, int count, int prec) { return frob_workspace_bytes(op, N, count, prec); }

struct Layout {
  int* map;
  frob_info* tinfo;
  unsigned char *pin, *pout, *sws;
  size_t sws_bytes, bytes;
};

Layout carve(const Plan& p, int batch, int op, int prec, void* ws) {
  Layout L{};
  unsigned char* base = static_cast<unsigned char*>(ws);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    unsigned char* q = base ? base + off : nullptr;
    off += (bytes + 255) & ~(size_t)255;
    return q;
  };
  size_t maxio = 0, maxws = 0;
  for (int b = 0; b < p.nb; ++b) {
    maxio = std::max(maxio, (size_t)p.count[b] * p.N[b] * p.N[b] * elem_size(prec));
    maxws = std::max(maxws, sub_ws(op, p.N[b], p.count[b], prec));
  }
  L.map = reinterpret_cast<int*>(take((size_t)batch * sizeof(int)));
  L.tinfo = reinterpret_cast<frob_info*>(take((size_t)batch * sizeof(frob_info)));
  L.pin = take(maxio);
  L.pout = take(maxio);
  L.sws_bytes = maxws;
  L.sws = take(maxws);
  L.bytes = off;
  return L;
}

// slot of matrix i = number of earlier matrices in the same bucket
__global__ void map_kernel(int batch, const int32_t* n_dev, BucketTable t, int* map) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= batch) return;
  const int Ni = padded(n_dev[i]);
  int slot = 0;
  for (int j = 0; j < i; ++j) slot += (padded(n_dev[j]) == Ni);
  for (int b = 0; b < t.nb; ++b)
    if (t.N[b] == Ni) map[t.offset[b] + slot] = i;
}

template <typename C>
__global__ void gather_kernel(int N, int offset, const int* map, const int32_t* n_dev, const void* const* M,
                              const int64_t* ldm, C* pin, C pad) {
  const int s = blockIdx.z;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)N * N) return;
  const int r = (int)(e / N), c = (int)(e % N);
  const int i = map[offset + s];
  const int n = n_dev[i];
  C v = zero_v<C>();
  if (r < n && c < n)
    v = static_cast<const C*>(M[i])[(int64_t)r * ldm[i] + c];
  else if (r == c)
    v = pad;
  pin[(int64_t)s * N * N + e] = v;
}

template <typename C>
__global__ void scatter_kernel(int N, int offset, const int* map, const int32_t* n_dev, void* const* X,
                               const int64_t* ldx, const C* pout, const frob_info* tinfo, frob_info* info) {
  const int s = blockIdx.z;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int i = map[offset + s];
  const int n = n_dev[i];
  if (e == 0) info[i] = tinfo[s];
  if (e >= (int64_t)N * N) return;
  const int r = (int)(e / N), c = (int)(e % N);
  if (r < n && c < n) static_cast<C*>(X[i])[(int64_t)r * ldx[i] + c] = pout[(int64_t)s * N * N + e];
}

}  // namespace batched
}  // namespace frob

using namespace frob;
using namespace frob::batched;

extern "C" size_t frob_inv_batched_workspace_bytes(int op, int batch, const int32_t* n_host, int prec) {
  if (batch < 1 || !n_host || op < FROB_OP_INV || op > FROB_OP_CPLX_CHOL) return 0;
  Plan p;
  if (!make_plan(batch, n_host, p)) return 0;
  for (int b = 0; b < p.nb; ++b)
    if (sub_ws(op, p.N[b], p.count[b], prec) == 0) return 0;
  return carve(p, batch, op, prec, nullptr).bytes;
}

extern "C" frob_status frob_inv_batched(int op, int batch, const int32_t* n_host, const int32_t* n_dev,
                                        const void* const* M_dev, const int64_t* ldm_dev, void* const* X_dev,
                                        const int64_t* ldx_dev, const frob_opts* opts, void* ws, size_t wsb,
                                        frob_info* info, void* stream) {
  if (batch < 1 || !n_host || !n_dev || !M_dev || !ldm_dev || !X_dev || !ldx_dev || !info) return FROB_ERR_ARG;
  if (op < FROB_OP_INV || op > FROB_OP_CPLX_CHOL) return FROB_ERR_ARG;
  frob_opts o;
  if (opts) {
    o = *opts;
  } else {
    std::memset(&o, 0, sizeof(o));
    o.prec = FROB_FP64;
    o.ns_max_iter = 8;
    o.ns_tol = 1e-14;
  }
  if (o.almost_sure) return FROB_ERR_UNSUPPORTED;  // mu is a function of the index inside a uniform call
  Plan p;
  if (!make_plan(batch, n_host, p)) return FROB_ERR_ARG;
  const size_t need = frob_inv_batched_workspace_bytes(op, batch, n_host, o.prec);
  if (need == 0) return FROB_ERR_UNSUPPORTED;
  if (!ws || wsb < need || (reinterpret_cast<uintptr_t>(ws) & 255)) return FROB_ERR_WORKSPACE;
  Layout L = carve(p, batch, op, o.prec, ws);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  BucketTable t{};
  t.nb = p.nb;
  for (int b = 0; b < p.nb; ++b) {
    t.N[b] = p.N[b];
    t.offset[b] = p.offset[b];
  }
  FROB_LAUNCH("batched_map", st, map_kernel<<<(batch + 127) / 128, 128, 0, st>>>(batch, n_dev, t, L.map));
  const bool f32 = o.prec == FROB_FP32;
  // the padding block's diagonal: its factored real part must be invertible
  // (i for FROB_PART_B, 1 + i for FROB_PART_AUTO so that either part is;
  // 1 otherwise); its inverse is discarded
  const double pr = (op == FROB_OP_INV && o.part == FROB_PART_B) ? 0.0 : 1.0;
  const double pi = (op == FROB_OP_INV && o.part != FROB_PART_A) ? 1.0 : 0.0;
  for (int b = 0; b < p.nb; ++b) {
    const int N = p.N[b], cnt = p.count[b];
    const int64_t NN = (int64_t)N * N;
    const dim3 g((unsigned)((NN + 255) / 256), 1, (unsigned)cnt);
    if (f32)
      FROB_LAUNCH("batched_gather", st,
                  gather_kernel<zf><<<g, 256, 0, st>>>(N, p.offset[b], L.map, n_dev, M_dev, ldm_dev,
                                                       reinterpret_cast<zf*>(L.pin), zf{(float)pr, (float)pi}));
    else
      FROB_LAUNCH("batched_gather", st,
                  gather_kernel<zd><<<g, 256, 0, st>>>(N, p.offset[b], L.map, n_dev, M_dev, ldm_dev,
                                                       reinterpret_cast<zd*>(L.pin), zd{pr, pi}));
    frob_status s;
    switch (op) {
      case FROB_OP_INV:
        s = frob_inv(N, cnt, L.pin, N, NN, L.pout, N, NN, &o, L.sws, L.sws_bytes, L.tinfo, stream);
        break;
      case FROB_OP_INV_HPD:
        s = frob_inv_hpd(N, cnt, L.pin, N, NN, L.pout, N, NN, &o, L.sws, L.sws_bytes, L.tinfo, stream);
        break;
      case FROB_OP_CPLX_LU:
        s = o.prec == FROB_MIXED_BF16
                ? cplx_inv_mixed(op, N, cnt, L.pin, N, NN, L.pout, N, NN, &o, L.sws, L.sws_bytes, L.tinfo, stream)
                : cplx_lu_inv(N, cnt, L.pin, N, NN, L.pout, N, NN, o.prec, L.sws, L.sws_bytes, L.tinfo, stream);
        break;
      default:
        s = o.prec == FROB_MIXED_BF16
                ? cplx_inv_mixed(op, N, cnt, L.pin, N, NN, L.pout, N, NN, &o, L.sws, L.sws_bytes, L.tinfo, stream)
                : cplx_chol_inv(N, cnt, L.pin, N, NN, L.pout, N, NN, o.prec, L.sws, L.sws_bytes, L.tinfo, stream);
        break;
    }
    if (s != FROB_OK) return s;
    if (f32)
      FROB_LAUNCH("batched_scatter", st,
                  scatter_kernel<zf><<<g, 256, 0, st>>>(N, p.offset[b], L.map, n_dev, X_dev, ldx_dev,
                                                        reinterpret_cast<const zf*>(L.pout), L.tinfo, info));
    else
      FROB_LAUNCH("batched_scatter", st,
                  scatter_kernel<zd><<<g, 256, 0, st>>>(N, p.offset[b], L.map, n_dev, X_dev, ldx_dev,
                                                        reinterpret_cast<const zd*>(L.pout), L.tinfo, info));
  }
  return cudaGetLastError() == cudaSuccess ? FROB_OK : FROB_ERR_CUDA;
}
