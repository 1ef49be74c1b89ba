// C-ABI entry points of libfrobinv (declared in include/frobinv.h): argument
// checks, workspace sizing, dispatch to the per-precision drivers, the split
// of a batch over two internal streams (and its opt-in autotuner), and the
// launch counter and per-kernel profiler.  The Newton drivers, the bicomplex
// inverse, the uneven-batch driver, the mixed precisions and the tensor-core
// GEMM have their entry points in newton.cu, iqe.cu, batched.cu, mixed.cu /
// api (dispatch) and tc_gemm.cu.
#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <vector>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <cuda_runtime.h>

#include "../../include/frobinv.h"
#include "common.cuh"
#include "ops.h"

using namespace frob;

namespace frob {
static std::atomic<uint64_t> g_launches{0};
static int debug_level() {
  static int level = [] {
    const char* e = std::getenv("FROB_DEBUG_SYNC");
    return e ? std::atoi(e) : 0;
  }();
  return level;
}
struct ProfRec {
  const char* name;
  cudaEvent_t a, b;
  double flops;
};
static std::mutex g_prof_mu;
static std::atomic<int> g_prof_on{0};
static std::vector<ProfRec> g_prof_recs;
static std::vector<cudaEvent_t> g_prof_pool;
static thread_local ProfRec t_pending{nullptr, nullptr, nullptr, 0.0};
static thread_local double t_next_flops = 0.0;

void set_launch_flops(double flops) { t_next_flops = flops; }

static cudaEvent_t prof_event() {
  if (!g_prof_pool.empty()) {
    cudaEvent_t e = g_prof_pool.back();
    g_prof_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void launch_begin(const char* name, cudaStream_t st) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  if (debug_level()) {
    std::fprintf(stderr, "[frob] launch %s\n", name);
    std::fflush(stderr);
  }
  const double flops = t_next_flops;
  t_next_flops = 0.0;
  if (g_prof_on.load(std::memory_order_relaxed)) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    t_pending = ProfRec{name, prof_event(), prof_event(), flops};
    cudaEventRecord(t_pending.a, st);
  }
}
void launch_end(const char* name, cudaStream_t st) {
  if (t_pending.name == name && t_pending.a) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    cudaEventRecord(t_pending.b, st);
    g_prof_recs.push_back(t_pending);
    t_pending = ProfRec{nullptr, nullptr, nullptr, 0.0};
  }
  if (debug_level()) {
    cudaError_t e1 = cudaGetLastError();
    cudaError_t e2 = cudaStreamSynchronize(st);
    std::fprintf(stderr, "[frob] done %s: launch=%s sync=%s\n", name, cudaGetErrorString(e1), cudaGetErrorString(e2));
    std::fflush(stderr);
  }
}
}  // namespace frob

namespace {

frob_opts default_opts() {
  frob_opts o;
  std::memset(&o, 0, sizeof(o));
  o.prec = FROB_FP64;
  o.ns_max_iter = 8;
  o.ns_tol = 1e-14;
  return o;
}

bool valid_prec(int p) { return p == FROB_FP64 || p == FROB_FP32; }
// FROB_MIXED_TF32 has no path of its own (its start would need TF32 operands,
// which do not contract at the workloads' condition numbers): unsupported.
bool mixed_prec(int p) { return p == FROB_MIXED_BF16; }

size_t elem_bytes(int prec) { return prec == FROB_FP32 ? 8 : 16; }

// Overlap test of the byte ranges touched by two strided batches.
bool overlaps(const void* a, int64_t lda, int64_t sa, const void* b, int64_t ldb, int64_t sb, int n, int batch,
              size_t eb) {
  auto span = [&](int64_t ld, int64_t s) {
    return (size_t)(((int64_t)(batch - 1) * s + (int64_t)(n - 1) * ld + n) * (int64_t)eb);
  };
  const char* pa = static_cast<const char*>(a);
  const char* pb = static_cast<const char*>(b);
  size_t la = span(lda, sa), lb = span(ldb, sb);
  return pa < pb + lb && pb < pa + la;
}

frob_status check_common(int n, int batch, const void* M, int64_t ldm, int64_t sm, const void* X, int64_t ldx,
                         int64_t sx, void* ws, size_t wsb, size_t need, frob_info* info, int prec,
                         bool need_info = true) {
  if (n < 1 || batch < 1 || batch > 65535) return FROB_ERR_ARG;
  if (!M || !X || (need_info && !info)) return FROB_ERR_ARG;
  if (ldm < n || ldx < n) return FROB_ERR_ARG;
  if (batch > 1 && (sm < ldm * (int64_t)n || sx < ldx * (int64_t)n)) return FROB_ERR_ARG;
  if (overlaps(M, ldm, sm, X, ldx, sx, n, batch, elem_bytes(prec))) return FROB_ERR_ARG;
  if (!valid_prec(prec) && !mixed_prec(prec)) return FROB_ERR_UNSUPPORTED;
  if (!ws || wsb < need || (reinterpret_cast<uintptr_t>(ws) & 255)) return FROB_ERR_WORKSPACE;
  return FROB_OK;
}

frob_status launched() {
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? FROB_OK : FROB_ERR_CUDA;
}

// Batch slices on internal streams.  The blocked factorisations and solves
// are sequences of launches of a few hundred CTAs each; running two halves of
// the batch on two streams forked from the caller's stream (and joined back
// before the call returns to it) lets one half's wave tails and short launches
// overlap the other half's work.  The streams and events belong to the host
// thread and device: created on first use, destroyed when the thread exits
// (a thread pool does not accumulate them); the fork / join pattern is also
// valid inside a CUDA-graph capture of the caller's stream.
constexpr int NSPLIT = 2;
struct SplitStreams {
  cudaStream_t s[NSPLIT];
  cudaEvent_t fork, join[NSPLIT];
};
struct SplitStreamSets {
  std::map<int, SplitStreams> by_device;
  ~SplitStreamSets() {
    // at thread exit; errors (a runtime already shut down at process exit)
    // are ignored
    for (auto& kv : by_device) {
      for (int k = 0; k < NSPLIT; ++k) {
        cudaStreamDestroy(kv.second.s[k]);
        cudaEventDestroy(kv.second.join[k]);
      }
      cudaEventDestroy(kv.second.fork);
    }
  }
};
SplitStreams* split_streams() {
  thread_local SplitStreamSets holder;
  std::map<int, SplitStreams>& sets = holder.by_device;
  int dev = 0;
  cudaGetDevice(&dev);
  auto it = sets.find(dev);
  if (it != sets.end()) return &it->second;
  SplitStreams ss{};
  for (int k = 0; k < NSPLIT; ++k) {
    cudaStreamCreateWithFlags(&ss.s[k], cudaStreamNonBlocking);
    cudaEventCreateWithFlags(&ss.join[k], cudaEventDisableTiming);
  }
  cudaEventCreateWithFlags(&ss.fork, cudaEventDisableTiming);
  return &(sets[dev] = ss);
}
// slice k of a batch: [first, first + count)
inline int slice_first(int batch, int k) { return (int)(((int64_t)batch * k) / NSPLIT); }
inline int slice_count(int batch, int k) { return slice_first(batch, k + 1) - slice_first(batch, k); }
inline size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }
// Workspace of a split call: one carve per slice.
template <class WsOf> size_t split_ws(int batch, WsOf ws_of) {
  if (batch < NSPLIT) return ws_of(batch);
  size_t total = 0;
  for (int k = 0; k < NSPLIT; ++k) total += round256(ws_of(slice_count(batch, k)));
  return total;
}
// Autotuning of the split (opt-in, frob_autotune_enable): per (operation,
// precision, n, batch) the call is timed once as one slice and once as two
// (after an untimed two-slice run), and the faster is cached for later calls.
// Every matrix goes through the same kernels whatever the split, so the
// FP64 / FP32 results do not depend on the choice (the mixed precisions'
// residual sums only through the order of their atomic additions).  No
// tuning while a graph capture or the per-kernel profiler is active.
struct TuneKey {
  int op, prec, n, batch;
  bool operator<(const TuneKey& o) const {
    if (op != o.op) return op < o.op;
    if (prec != o.prec) return prec < o.prec;
    if (n != o.n) return n < o.n;
    return batch < o.batch;
  }
};
struct TuneRec {
  int slices;
  float ms_one, ms_two;
};
std::atomic<int> g_tune_on{0};
std::mutex g_tune_mu;
std::map<TuneKey, TuneRec> g_tune;

bool capturing(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  return cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone;
}

// run(first, count, workspace, stream) per slice.  While per-kernel profiling
// is on, the slices run one after the other on the caller's stream, so that
// the events around a launch time that kernel alone.
template <class WsOf, class Run> void split_slices(int slices, int batch, void* ws, cudaStream_t st, WsOf ws_of, Run run);

template <class WsOf, class Run>
void split_run(int batch, void* ws, cudaStream_t st, WsOf ws_of, Run run, const TuneKey* key = nullptr,
               size_t wsb = 0) {
  if (batch < NSPLIT) {
    run(0, batch, ws, st);
    return;
  }
  int slices = NSPLIT;
  if (key && g_tune_on.load(std::memory_order_relaxed)) {
    bool found = false;
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      auto it = g_tune.find(*key);
      if (it != g_tune.end()) {
        slices = it->second.slices;
        found = true;
      }
    }
    if (!found && !g_prof_on.load(std::memory_order_relaxed) && !capturing(st) && round256(ws_of(batch)) <= wsb) {
      cudaEvent_t ev[3];
      for (auto& e : ev) cudaEventCreate(&e);
      split_slices(NSPLIT, batch, ws, st, ws_of, run);  // warm-up (first-use setup)
      cudaEventRecord(ev[0], st);
      split_slices(1, batch, ws, st, ws_of, run);
      cudaEventRecord(ev[1], st);
      split_slices(NSPLIT, batch, ws, st, ws_of, run);  // the output of this run stands
      cudaEventRecord(ev[2], st);
      float t1 = 0.f, t2 = 0.f;
      if (cudaEventSynchronize(ev[2]) == cudaSuccess) {
        cudaEventElapsedTime(&t1, ev[0], ev[1]);
        cudaEventElapsedTime(&t2, ev[1], ev[2]);
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune[*key] = TuneRec{t1 <= t2 ? 1 : NSPLIT, t1, t2};
      }
      for (auto& e : ev) cudaEventDestroy(e);
      return;
    }
  }
  split_slices(slices, batch, ws, st, ws_of, run);
}

template <class WsOf, class Run> void split_slices(int slices, int batch, void* ws, cudaStream_t st, WsOf ws_of, Run run) {
  if (slices < NSPLIT) {
    run(0, batch, ws, st);
    return;
  }
  if (g_prof_on.load(std::memory_order_relaxed)) {
    unsigned char* w = static_cast<unsigned char*>(ws);
    for (int k = 0; k < NSPLIT; ++k) {
      run(slice_first(batch, k), slice_count(batch, k), w, st);
      w += round256(ws_of(slice_count(batch, k)));
    }
    return;
  }
  SplitStreams* ss = split_streams();
  cudaEventRecord(ss->fork, st);
  unsigned char* w = static_cast<unsigned char*>(ws);
  for (int k = 0; k < NSPLIT; ++k) {
    const int first = slice_first(batch, k), count = slice_count(batch, k);
    cudaStreamWaitEvent(ss->s[k], ss->fork, 0);
    run(first, count, w, ss->s[k]);
    w += round256(ws_of(count));
    cudaEventRecord(ss->join[k], ss->s[k]);
  }
  for (int k = 0; k < NSPLIT; ++k) cudaStreamWaitEvent(st, ss->join[k], 0);
}

template <typename T> MatB<const T> in_view(const void* p, int64_t ld, int64_t s) {
  return MatB<const T>{static_cast<const T*>(p), ld, s};
}
template <typename T> MatB<T> out_view(void* p, int64_t ld, int64_t s) {
  return MatB<T>{static_cast<T*>(p), ld, s};
}

}  // namespace

extern "C" {

size_t frob_workspace_bytes(int op, int n, int batch, int prec) {
  if (n < 1 || batch < 1) return 0;
  if (mixed_prec(prec))
    return (op >= FROB_OP_INV && op <= FROB_OP_CPLX_CHOL && n <= 512)
               ? split_ws(batch, [&](int b) { return mixed::mixed_ws(n, b); })
               : 0;
  if (!valid_prec(prec)) return 0;
  const bool f32 = prec == FROB_FP32;
  switch (op) {
    case FROB_OP_INV:
      return split_ws(batch, [&](int b) {
        return f32 ? frob_lu_ws<float>(n, b, nullptr, nullptr) : frob_lu_ws<double>(n, b, nullptr, nullptr);
      });
    case FROB_OP_INV_HPD:
      return split_ws(batch, [&](int b) {
        return f32 ? frob_chol_ws<float>(n, b, nullptr, nullptr) : frob_chol_ws<double>(n, b, nullptr, nullptr);
      });
    case FROB_OP_CPLX_LU:
      return split_ws(batch, [&](int b) {
        return f32 ? cplx_lu_ws<zf>(n, b, nullptr, nullptr) : cplx_lu_ws<zd>(n, b, nullptr, nullptr);
      });
    case FROB_OP_CPLX_CHOL:
      return split_ws(batch, [&](int b) {
        return f32 ? cplx_chol_ws<zf>(n, b, nullptr, nullptr) : cplx_chol_ws<zd>(n, b, nullptr, nullptr);
      });
    case FROB_OP_ADJOINT:
      return f32 ? adjoint_ws<float>(n, batch) : adjoint_ws<double>(n, batch);
    default:
      return 0;
  }
}

frob_status frob_inv(int n, int batch, const void* M, int64_t ldm, int64_t sm, void* X, int64_t ldx, int64_t sx,
                     const frob_opts* opts, void* ws, size_t wsb, frob_info* info, void* stream) {
  frob_opts o = opts ? *opts : default_opts();
  if (o.almost_sure != 0 && o.almost_sure != 1) return FROB_ERR_ARG;
  if (o.part < FROB_PART_A || o.part > FROB_PART_AUTO) return FROB_ERR_ARG;
  if (o.fp64_gemm != FROB_GEMM_AUTO && o.fp64_gemm != FROB_GEMM_FP64_PIPE) return FROB_ERR_ARG;
  if (o.part != FROB_PART_A && o.almost_sure) return FROB_ERR_ARG;
  frob_status s = check_common(n, batch, M, ldm, sm, X, ldx, sx, ws, wsb,
                               frob_workspace_bytes(FROB_OP_INV, n, batch, o.prec), info, o.prec);
  if (s != FROB_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (mixed_prec(o.prec)) {
    if (o.almost_sure) return FROB_ERR_UNSUPPORTED;
    if (n > 512) return FROB_ERR_UNSUPPORTED;
    frob_status ms = FROB_OK;
    const TuneKey key{FROB_OP_INV, o.prec, n, batch};
    split_run(batch, ws, st, [&](int b) { return mixed::mixed_ws(n, b); },
              [&](int first, int count, void* w, cudaStream_t s2) {
                frob_status r = mixed::mixed_run(n, count, in_view<zd>(M, ldm, sm).at_batch(first),
                                                 out_view<zd>(X, ldx, sx).at_batch(first), o, w, info + first, s2,
                                                 false);
                if (r != FROB_OK) ms = r;
              }, &key, wsb);
    return ms != FROB_OK ? ms : launched();
  }
  // (the almost-sure draw of mu depends on the matrix index: one slice)
  const int sb = o.almost_sure ? 1 : batch;
  auto run = [&](int first, int count, void* w, cudaStream_t s2) {
    if (o.prec == FROB_FP32)
      frob_lu_run<float>(n, count, in_view<zf>(M, ldm, sm).at_batch(first), out_view<zf>(X, ldx, sx).at_batch(first), o,
                         w, info + first, s2);
    else
      frob_lu_run<double>(n, count, in_view<zd>(M, ldm, sm).at_batch(first), out_view<zd>(X, ldx, sx).at_batch(first),
                          o, w, info + first, s2);
  };
  const TuneKey key{FROB_OP_INV, o.prec, n, batch};
  if (sb == 1)
    run(0, batch, ws, st);
  else
    split_run(batch, ws, st, [&](int b) {
      return o.prec == FROB_FP32 ? frob_lu_ws<float>(n, b, nullptr, nullptr) : frob_lu_ws<double>(n, b, nullptr, nullptr);
    }, run, &key, wsb);
  return launched();
}

frob_status frob_inv_hpd(int n, int batch, const void* M, int64_t ldm, int64_t sm, void* X, int64_t ldx, int64_t sx,
                         const frob_opts* opts, void* ws, size_t wsb, frob_info* info, void* stream) {
  frob_opts o = opts ? *opts : default_opts();
  if (o.almost_sure) return FROB_ERR_ARG;  // A is SPD for HPD input (Lemma "positive real part")
  if (o.fp64_gemm != FROB_GEMM_AUTO && o.fp64_gemm != FROB_GEMM_FP64_PIPE) return FROB_ERR_ARG;
  frob_status s = check_common(n, batch, M, ldm, sm, X, ldx, sx, ws, wsb,
                               frob_workspace_bytes(FROB_OP_INV_HPD, n, batch, o.prec), info, o.prec);
  if (s != FROB_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (mixed_prec(o.prec)) {
    if (n > 512) return FROB_ERR_UNSUPPORTED;
    frob_status ms = FROB_OK;
    const TuneKey key{FROB_OP_INV_HPD, o.prec, n, batch};
    split_run(batch, ws, st, [&](int b) { return mixed::mixed_ws(n, b); },
              [&](int first, int count, void* w, cudaStream_t s2) {
                frob_status r = mixed::mixed_run(n, count, in_view<zd>(M, ldm, sm).at_batch(first),
                                                 out_view<zd>(X, ldx, sx).at_batch(first), o, w, info + first, s2,
                                                 true);
                if (r != FROB_OK) ms = r;
              }, &key, wsb);
    return ms != FROB_OK ? ms : launched();
  }
  const TuneKey key{FROB_OP_INV_HPD, o.prec, n, batch};
  split_run(batch, ws, st, [&](int b) {
    return o.prec == FROB_FP32 ? frob_chol_ws<float>(n, b, nullptr, nullptr) : frob_chol_ws<double>(n, b, nullptr, nullptr);
  }, [&](int first, int count, void* w, cudaStream_t s2) {
    if (o.prec == FROB_FP32)
      frob_chol_run<float>(n, count, in_view<zf>(M, ldm, sm).at_batch(first), out_view<zf>(X, ldx, sx).at_batch(first),
                           w, info + first, s2);
    else
      frob_chol_run<double>(n, count, in_view<zd>(M, ldm, sm).at_batch(first), out_view<zd>(X, ldx, sx).at_batch(first),
                            w, info + first, s2, o.fp64_gemm);
  }, &key, wsb);
  return launched();
}

frob_status cplx_inv_mixed(int op, int n, int batch, const void* M, int64_t ldm, int64_t sm, void* X, int64_t ldx,
                           int64_t sx, const frob_opts* opts, void* ws, size_t wsb, frob_info* info, void* stream) {
  if (op != FROB_OP_CPLX_LU && op != FROB_OP_CPLX_CHOL) return FROB_ERR_ARG;
  frob_opts o = opts ? *opts : default_opts();
  if (!opts) o.prec = FROB_MIXED_BF16;
  if (o.almost_sure || o.part != FROB_PART_A || o.fp64_gemm != FROB_GEMM_AUTO) return FROB_ERR_ARG;
  frob_status s = check_common(n, batch, M, ldm, sm, X, ldx, sx, ws, wsb, frob_workspace_bytes(op, n, batch, o.prec),
                               info, o.prec);
  if (s != FROB_OK) return s;
  if (!mixed_prec(o.prec) || n > 512) return FROB_ERR_UNSUPPORTED;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  frob_status ms = FROB_OK;
  const TuneKey key{op, o.prec, n, batch};
  split_run(batch, ws, st, [&](int b) { return mixed::mixed_ws(n, b); },
            [&](int first, int count, void* w, cudaStream_t s2) {
              frob_status r = mixed::mixed_run(n, count, in_view<zd>(M, ldm, sm).at_batch(first),
                                               out_view<zd>(X, ldx, sx).at_batch(first), o, w, info + first, s2,
                                               op == FROB_OP_CPLX_CHOL, true);
              if (r != FROB_OK) ms = r;
            }, &key, wsb);
  return ms != FROB_OK ? ms : launched();
}

frob_status cplx_lu_inv(int n, int batch, const void* M, int64_t ldm, int64_t sm, void* X, int64_t ldx, int64_t sx,
                        int prec, void* ws, size_t wsb, frob_info* info, void* stream) {
  if (mixed_prec(prec)) {
    frob_opts o = default_opts();
    o.prec = prec;
    return cplx_inv_mixed(FROB_OP_CPLX_LU, n, batch, M, ldm, sm, X, ldx, sx, &o, ws, wsb, info, stream);
  }
  frob_status s = check_common(n, batch, M, ldm, sm, X, ldx, sx, ws, wsb,
                               frob_workspace_bytes(FROB_OP_CPLX_LU, n, batch, prec), info, prec);
  if (s != FROB_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const TuneKey key{FROB_OP_CPLX_LU, prec, n, batch};
  split_run(batch, ws, st, [&](int b) {
    return prec == FROB_FP32 ? cplx_lu_ws<zf>(n, b, nullptr, nullptr) : cplx_lu_ws<zd>(n, b, nullptr, nullptr);
  }, [&](int first, int count, void* w, cudaStream_t s2) {
    if (prec == FROB_FP32)
      cplx_lu_run<zf>(n, count, in_view<zf>(M, ldm, sm).at_batch(first), out_view<zf>(X, ldx, sx).at_batch(first), w,
                      info + first, s2);
    else
      cplx_lu_run<zd>(n, count, in_view<zd>(M, ldm, sm).at_batch(first), out_view<zd>(X, ldx, sx).at_batch(first), w,
                      info + first, s2);
  }, &key, wsb);
  return launched();
}

frob_status cplx_chol_inv(int n, int batch, const void* M, int64_t ldm, int64_t sm, void* X, int64_t ldx,
                          int64_t sx, int prec, void* ws, size_t wsb, frob_info* info, void* stream) {
  if (mixed_prec(prec)) {
    frob_opts o = default_opts();
    o.prec = prec;
    return cplx_inv_mixed(FROB_OP_CPLX_CHOL, n, batch, M, ldm, sm, X, ldx, sx, &o, ws, wsb, info, stream);
  }
  frob_status s = check_common(n, batch, M, ldm, sm, X, ldx, sx, ws, wsb,
                               frob_workspace_bytes(FROB_OP_CPLX_CHOL, n, batch, prec), info, prec);
  if (s != FROB_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const TuneKey key{FROB_OP_CPLX_CHOL, prec, n, batch};
  split_run(batch, ws, st, [&](int b) {
    return prec == FROB_FP32 ? cplx_chol_ws<zf>(n, b, nullptr, nullptr) : cplx_chol_ws<zd>(n, b, nullptr, nullptr);
  }, [&](int first, int count, void* w, cudaStream_t s2) {
    if (prec == FROB_FP32)
      cplx_chol_run<zf>(n, count, in_view<zf>(M, ldm, sm).at_batch(first), out_view<zf>(X, ldx, sx).at_batch(first), w,
                        info + first, s2);
    else
      cplx_chol_run<zd>(n, count, in_view<zd>(M, ldm, sm).at_batch(first), out_view<zd>(X, ldx, sx).at_batch(first), w,
                        info + first, s2);
  }, &key, wsb);
  return launched();
}

frob_status frob_inv_adjoint(int n, int batch, const void* X, int64_t ldx, int64_t sx, const void* G, int64_t ldg,
                             int64_t sg, void* gradM, int64_t ldr, int64_t sr, int prec, void* ws, size_t wsb,
                             void* stream) {
  if (mixed_prec(prec)) return FROB_ERR_UNSUPPORTED;
  if (!G || ldg < n || (batch > 1 && sg < ldg * (int64_t)n)) return FROB_ERR_ARG;
  frob_status s = check_common(n, batch, X, ldx, sx, gradM, ldr, sr, ws, wsb,
                               frob_workspace_bytes(FROB_OP_ADJOINT, n, batch, prec), nullptr, prec, false);
  if (s != FROB_OK) return s;
  if (overlaps(G, ldg, sg, gradM, ldr, sr, n, batch, elem_bytes(prec))) return FROB_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (prec == FROB_FP32)
    adjoint_run<float>(n, batch, in_view<zf>(X, ldx, sx), in_view<zf>(G, ldg, sg), out_view<zf>(gradM, ldr, sr), ws, st);
  else
    adjoint_run<double>(n, batch, in_view<zd>(X, ldx, sx), in_view<zd>(G, ldg, sg), out_view<zd>(gradM, ldr, sr), ws,
                        st);
  return launched();
}

size_t frob_solve_workspace_bytes(int op, int n, int nrhs, int batch, int prec) {
  if (n < 1 || nrhs < 1 || batch < 1 || !valid_prec(prec)) return 0;
  const bool f32 = prec == FROB_FP32;
  if (op == 0) return f32 ? frob_solve_ws<float>(n, nrhs, batch, nullptr, nullptr)
                          : frob_solve_ws<double>(n, nrhs, batch, nullptr, nullptr);
  if (op == 1) return f32 ? cplx_solve_ws<zf>(n, nrhs, batch) : cplx_solve_ws<zd>(n, nrhs, batch);
  if (op == 2) return f32 ? aug_solve_ws<float>(n, nrhs, batch) : aug_solve_ws<double>(n, nrhs, batch);
  return 0;
}

static frob_status solve_common(int op, int n, int nrhs, int batch, const void* M, int64_t ldm, int64_t sm,
                                const void* B, int64_t ldb, int64_t sb, void* X, int64_t ldx, int64_t sx, int prec,
                                void* ws, size_t wsb, frob_info* info, void* stream) {
  if (n < 1 || nrhs < 1 || batch < 1 || batch > 65535 || !M || !B || !X || !info) return FROB_ERR_ARG;
  if (ldm < n || ldb < nrhs || ldx < nrhs) return FROB_ERR_ARG;
  if (batch > 1 && (sm < ldm * (int64_t)n || sb < ldb * (int64_t)n || sx < ldx * (int64_t)n)) return FROB_ERR_ARG;
  if (!valid_prec(prec)) return FROB_ERR_UNSUPPORTED;
  const size_t eb = elem_bytes(prec);
  auto span = [&](int64_t ld, int64_t s, int cols) { return (size_t)(((int64_t)(batch - 1) * s + (int64_t)(n - 1) * ld + cols) * (int64_t)eb); };
  auto ovl = [&](const void* a, size_t la, const void* c, size_t lc) {
    const char* pa = static_cast<const char*>(a);
    const char* pc = static_cast<const char*>(c);
    return pa < pc + lc && pc < pa + la;
  };
  if (ovl(X, span(ldx, sx, nrhs), M, span(ldm, sm, n)) || ovl(X, span(ldx, sx, nrhs), B, span(ldb, sb, nrhs)))
    return FROB_ERR_ARG;
  const size_t need = frob_solve_workspace_bytes(op, n, nrhs, batch, prec);
  if (!ws || wsb < need || (reinterpret_cast<uintptr_t>(ws) & 255)) return FROB_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (op == 0) {
    if (prec == FROB_FP32)
      frob_solve_run<float>(n, nrhs, batch, in_view<zf>(M, ldm, sm), in_view<zf>(B, ldb, sb), out_view<zf>(X, ldx, sx),
                            ws, info, st);
    else
      frob_solve_run<double>(n, nrhs, batch, in_view<zd>(M, ldm, sm), in_view<zd>(B, ldb, sb),
                             out_view<zd>(X, ldx, sx), ws, info, st);
  } else if (op == 2) {
    if (prec == FROB_FP32)
      aug_solve_run<float>(n, nrhs, batch, in_view<zf>(M, ldm, sm), in_view<zf>(B, ldb, sb), out_view<zf>(X, ldx, sx),
                           ws, info, st);
    else
      aug_solve_run<double>(n, nrhs, batch, in_view<zd>(M, ldm, sm), in_view<zd>(B, ldb, sb),
                            out_view<zd>(X, ldx, sx), ws, info, st);
  } else {
    if (prec == FROB_FP32)
      cplx_solve_run<zf>(n, nrhs, batch, in_view<zf>(M, ldm, sm), in_view<zf>(B, ldb, sb), out_view<zf>(X, ldx, sx),
                         ws, info, st);
    else
      cplx_solve_run<zd>(n, nrhs, batch, in_view<zd>(M, ldm, sm), in_view<zd>(B, ldb, sb), out_view<zd>(X, ldx, sx),
                         ws, info, st);
  }
  return launched();
}

frob_status frob_solve(int n, int nrhs, int batch, const void* M, int64_t ldm, int64_t sm, const void* B, int64_t ldb,
                       int64_t sb, void* X, int64_t ldx, int64_t sx, int prec, void* ws, size_t wsb, frob_info* info,
                       void* stream) {
  return solve_common(0, n, nrhs, batch, M, ldm, sm, B, ldb, sb, X, ldx, sx, prec, ws, wsb, info, stream);
}

frob_status cplx_lu_solve(int n, int nrhs, int batch, const void* M, int64_t ldm, int64_t sm, const void* B,
                          int64_t ldb, int64_t sb, void* X, int64_t ldx, int64_t sx, int prec, void* ws, size_t wsb,
                          frob_info* info, void* stream) {
  return solve_common(1, n, nrhs, batch, M, ldm, sm, B, ldb, sb, X, ldx, sx, prec, ws, wsb, info, stream);
}

frob_status aug_real_solve(int n, int nrhs, int batch, const void* M, int64_t ldm, int64_t sm, const void* B,
                           int64_t ldb, int64_t sb, void* X, int64_t ldx, int64_t sx, int prec, void* ws, size_t wsb,
                           frob_info* info, void* stream) {
  return solve_common(2, n, nrhs, batch, M, ldm, sm, B, ldb, sb, X, ldx, sx, prec, ws, wsb, info, stream);
}

const char* frob_status_str(int status) {
  switch (status) {
    case FROB_OK: return "FROB_OK";
    case FROB_ERR_ARG: return "FROB_ERR_ARG";
    case FROB_ERR_SINGULAR: return "FROB_ERR_SINGULAR";
    case FROB_ERR_NOT_HPD: return "FROB_ERR_NOT_HPD";
    case FROB_ERR_NOT_CONVERGED: return "FROB_ERR_NOT_CONVERGED";
    case FROB_ERR_TIMEOUT: return "FROB_ERR_TIMEOUT";
    case FROB_ERR_CUDA: return "FROB_ERR_CUDA";
    case FROB_ERR_WORKSPACE: return "FROB_ERR_WORKSPACE";
    case FROB_ERR_UNSUPPORTED: return "FROB_ERR_UNSUPPORTED";
    default: return "FROB_ERR_UNKNOWN";
  }
}

const char* frob_version(void) { return "frobinv 0.1 sm_103a"; }

uint64_t frob_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

void frob_autotune_enable(int on) { g_tune_on.store(on ? 1 : 0); }

void frob_autotune_clear(void) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune.clear();
}

size_t frob_autotune_report(char* buf, size_t len) {
  std::string out = "{";
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    bool first = true;
    for (const auto& kv : g_tune) {
      char item[160];
      std::snprintf(item, sizeof(item), "%s\"%d,%d,%d,%d\": [%d, %.6g, %.6g]", first ? "" : ", ", kv.first.op,
                    kv.first.prec, kv.first.n, kv.first.batch, kv.second.slices, (double)kv.second.ms_one,
                    (double)kv.second.ms_two);
      out += item;
      first = false;
    }
  }
  out += "}";
  if (buf && len > 0) {
    const size_t k = out.size() < len - 1 ? out.size() : len - 1;
    std::memcpy(buf, out.data(), k);
    buf[k] = '\0';
  }
  return out.size() + 1;
}

void frob_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (on) {
    for (auto& r : g_prof_recs) {
      g_prof_pool.push_back(r.a);
      g_prof_pool.push_back(r.b);
    }
    g_prof_recs.clear();
  }
  g_prof_on.store(on ? 1 : 0);
}

size_t frob_profile_report(char* buf, size_t len) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  struct Acc {
    long launches = 0;
    double ms = 0.0, flops = 0.0;
  };
  std::map<std::string, Acc> acc;
  for (auto& r : g_prof_recs) {
    float ms = 0.f;
    if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      auto& e = acc[r.name];
      e.launches += 1;
      e.ms += ms;
      e.flops += r.flops;
    }
    g_prof_pool.push_back(r.a);
    g_prof_pool.push_back(r.b);
  }
  g_prof_recs.clear();
  std::string out = "{";
  bool first = true;
  for (auto& kv : acc) {
    char tmp[128];
    std::snprintf(tmp, sizeof(tmp), "[%ld, %.6f, %.6e]", kv.second.launches, kv.second.ms, kv.second.flops);
    out += (first ? "\"" : ", \"") + kv.first + "\": " + tmp;
    first = false;
  }
  out += "}";
  if (buf && len) {
    size_t k = out.size() < len - 1 ? out.size() : len - 1;
    std::memcpy(buf, out.data(), k);
    buf[k] = 0;
  }
  return out.size() + 1;
}

}  // extern "C"
