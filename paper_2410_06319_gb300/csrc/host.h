// Host infrastructure shared by the C ABI translation units: the handle, its
// workspace and CUDA-graph cache, stage timers, the call context (argument tuple and
// options) with its validation, and device-state reads.
#pragma once
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <functional>
#include <thread>
#include <stdexcept>
#include <string>
#include <unordered_map>
#include <vector>

#include "common.cuh"
#include "gauss.cuh"
#include "iter.h"
#include "kernels.h"
#include "lsq.h"

namespace {

using namespace lsq;

struct CudaFail {
  cudaError_t e;
  const char* what;
};
struct StatusFail {
  lsq_status st;
};

#define CK(expr)                                     \
  do {                                               \
    cudaError_t e_ = (expr);                         \
    if (e_ != cudaSuccess) throw CudaFail{e_, #expr}; \
  } while (0)

constexpr int kBatch = 8;        // iterations enqueued between host checks
constexpr size_t kRecMaxBytes = (size_t)4 << 30;   // deferred sketch-correction lists, at most
constexpr int kMaxGmres = 127;   // cap of the FGMRES basis size

struct Buf {
  void* p = nullptr;
  size_t bytes = 0;
};

}  // namespace

namespace {
// An instantiated CUDA graph of a batch of solver iterations, cached in the
// handle by the pointers and sizes it was captured with.
struct CachedGraph {
  cudaGraph_t g = nullptr;
  cudaGraphExec_t e = nullptr;
  int64_t kernels = 0;  // kernel nodes
  ~CachedGraph() {
    if (e) cudaGraphExecDestroy(e);
    if (g) cudaGraphDestroy(g);
  }
};
}  // namespace

struct lsq_handle {
  cudaStream_t user_stream = nullptr;  // the caller's stream (ordering only)
  cudaStream_t stream = nullptr;       // the handle's own non-blocking work stream
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  std::unordered_map<std::string, CachedGraph*> graphs;
  CachedGraph* cap = nullptr;          // graph being captured
  double kern_acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  int64_t kern_cnt[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  int device = 0;
  int num_sms = 0;
  std::unordered_map<std::string, Buf> bufs;
  int* d_err = nullptr;
  unsigned char* h_pinned = nullptr;   // 4 KB pinned host block for state reads
  std::string last_cuda;
  int64_t launches = 0;
  std::vector<cudaEvent_t> events;
  size_t next_event = 0;
  struct Mark {
    int stage;
    cudaEvent_t a, b;
  };
  std::vector<Mark> marks;
  std::vector<lsq_handle*> workers;    // sub-handles of lsq_lsir_batched (own streams)
  std::unordered_map<std::string, int64_t> tuned;   // grouped-launch grid sizes chosen by timing
};

namespace {

void* ws(lsq_handle* h, const char* name, size_t bytes, bool zero = false) {
  if (bytes == 0) bytes = 16;
  Buf& b = h->bufs[name];
  if (b.bytes < bytes) {
    if (b.p) CK(cudaFree(b.p));
    b.p = nullptr;
    b.bytes = 0;
    if (cudaMalloc(&b.p, bytes) != cudaSuccess) {
      cudaGetLastError();
      throw StatusFail{LSQ_E_NOMEM};
    }
    b.bytes = bytes;
    CK(cudaMemsetAsync(b.p, 0, bytes, h->stream));
  } else if (zero) {
    CK(cudaMemsetAsync(b.p, 0, bytes, h->stream));
  }
  return b.p;
}

cudaEvent_t next_event(lsq_handle* h) {
  if (h->next_event == h->events.size()) {
    cudaEvent_t e;
    CK(cudaEventCreate(&e));
    h->events.push_back(e);
  }
  return h->events[h->next_event++];
}

struct StageTimer {
  lsq_handle* h;
  int stage;
  cudaEvent_t a;
  StageTimer(lsq_handle* hh, int s) : h(hh), stage(s) {
    a = next_event(h);
    CK(cudaEventRecord(a, h->stream));
  }
  ~StageTimer() {
    try {
      cudaEvent_t b = next_event(h);
      if (cudaEventRecord(b, h->stream) == cudaSuccess) h->marks.push_back({stage, a, b});
    } catch (...) {
    }
  }
};

enum Stage { ST_CAST = 0, ST_SKETCH, ST_QR, ST_LSQR, ST_RES, ST_FGMRES, ST_UPDATE, ST_TOTAL };
enum Kern { K_SKETCH = 0, K_LSQR_PASS, K_FGM_PASS, K_RES_PASS, K_ARNOLDI, K_TRSV, K_SKETCH_FIX,
            K_NKERN = 8 };
constexpr int kKernMark = 100;   // marks with stage >= kKernMark time single kernels

// Brackets one launch with events when timing is on (opts.timing).
struct KernTimer {
  lsq_handle* h;
  int k;
  bool on;
  cudaEvent_t a{};
  KernTimer(lsq_handle* hh, int kk, bool enabled) : h(hh), k(kk), on(enabled && !hh->cap) {
    if (!on) return;
    a = next_event(h);
    CK(cudaEventRecord(a, h->stream));
  }
  ~KernTimer() {
    if (!on) return;
    try {
      cudaEvent_t b = next_event(h);
      if (cudaEventRecord(b, h->stream) == cudaSuccess) h->marks.push_back({kKernMark + k, a, b});
    } catch (...) {
    }
  }
};

int fmt_of(lsq_prec p) {
  switch (p) {
    case LSQ_F64: return FMT_F64;
    case LSQ_F32: return FMT_F32;
    case LSQ_F16: return FMT_F16;
    case LSQ_BF16: return FMT_BF16;
    case LSQ_E4M3: return FMT_E4M3;
    case LSQ_BF16X3: return FMT_BF16X3;
  }
  return -1;
}

double unit_roundoff(lsq_prec p) {
  switch (p) {
    case LSQ_F64: return std::ldexp(1.0, -53);
    case LSQ_F32: return std::ldexp(1.0, -24);
    case LSQ_F16: return std::ldexp(1.0, -11);
    case LSQ_BF16: return std::ldexp(1.0, -8);
    case LSQ_E4M3: return std::ldexp(1.0, -4);
    case LSQ_BF16X3: return std::ldexp(1.0, -24);   // three BF16 terms, FP32 accumulation
  }
  return 1.0;
}

int64_t round_up(int64_t v, int64_t q) { return ((v + q - 1) / q) * q; }

struct Ctx {
  lsq_handle* h;
  const double* A;
  const double* b;
  int64_t m, n, s, lda, lda32;
  lsq_prec us, up, uw, ur;
  double tol;
  uint64_t seed;
  lsq_opts o;
  cudaStream_t st;
  int nblk;        // pass grid
  int nblk2;       // vector-kernel grid
  double alpha;    // scaling of the augmented system (Sec. 4.1); 1 unscaled
};

#define L(expr)         \
  do {                  \
    CK(expr);           \
    ++c.h->launches;    \
  } while (0)

lsq_status validate(const Ctx& c, bool need_b) {
  if (!c.h) return LSQ_E_INVAL;
  if (!c.A || (need_b && !c.b)) return LSQ_E_INVAL;
  if (c.n < 1 || c.m < c.n || c.s < c.n || c.s > c.m) return LSQ_E_INVAL;
  if (c.n > 1024 || c.s > 16384) return LSQ_E_INVAL;
  if (c.m > ((int64_t)1 << 36)) return LSQ_E_INVAL;
  if (c.lda < c.n) return LSQ_E_INVAL;
  if (!(c.tol > 0.0) || !std::isfinite(c.tol)) return LSQ_E_INVAL;
  if (fmt_of(c.us) < 0 && c.us != LSQ_AUTO) return LSQ_E_INVAL;
  if (c.up != LSQ_F32 && c.up != LSQ_F64) return LSQ_E_INVAL;
  if (c.uw != LSQ_F32 && c.uw != LSQ_F64) return LSQ_E_INVAL;
  if (c.ur != LSQ_F64 && c.ur != LSQ_F64X2) return LSQ_E_INVAL;
  if (c.o.ops_escalated < 0 || c.o.ops_escalated > 1) return LSQ_E_INVAL;
  if (c.o.h_in_ur < 0 || c.o.h_in_ur > 1) return LSQ_E_INVAL;
  if (c.o.arnoldi < 0 || c.o.arnoldi > 3) return LSQ_E_INVAL;
  if (!(c.o.aug_alpha >= 0.0) || !std::isfinite(c.o.aug_alpha)) return LSQ_E_INVAL;
  if (c.o.gmres_maxit < 0 || c.o.gmres_maxit > kMaxGmres) return LSQ_E_INVAL;
  if (c.o.ir_maxit < 0 || c.o.ir_maxit > 32) return LSQ_E_INVAL;
  if (c.o.lsqr_maxit < 0) return LSQ_E_INVAL;
  if (c.o.sketch_kchunk < 0) return LSQ_E_INVAL;
  if (c.o.sketch_kind < 0 || c.o.sketch_kind > 1) return LSQ_E_INVAL;
  if (c.o.sparse_zeta < 0 || c.o.sparse_zeta > 8 || c.o.sparse_zeta > c.s) return LSQ_E_INVAL;
  if (c.o.sketch_kind == 1 && c.o.sparse_zeta == 0 && c.s < 8) return LSQ_E_INVAL;
  return LSQ_OK;
}

Ctx make_ctx(lsq_handle* h, const double* A, const double* b, int64_t m, int64_t n, int64_t s,
             lsq_prec us, lsq_prec up, lsq_prec uw, lsq_prec ur, double tol, uint64_t seed,
             const lsq_opts* opts) {
  Ctx c{};
  c.h = h;
  c.A = A;
  c.b = b;
  c.m = m;
  c.n = n;
  c.s = s;
  c.us = us;
  c.up = up;
  c.uw = uw;
  c.ur = ur;
  c.tol = tol;
  c.seed = seed;
  if (opts) c.o = *opts;
  else std::memset(&c.o, 0, sizeof(c.o));
  c.alpha = c.o.aug_alpha > 0.0 ? c.o.aug_alpha : 1.0;
  c.lda = c.o.lda > 0 ? c.o.lda : n;
  c.lda32 = round_up(n, 4);
  // the sparse sign sketch is exact up to a 2^-47 fixed-point grid: it counts as an FP64
  // sketch in the rules that use u_s (condition warning, escalation, LSQ_AUTO)
  if (c.o.sketch_kind == 1) c.us = LSQ_F64;
  if (h) {
    c.st = h->stream;
    c.nblk = pass_blocks(h->num_sms);
    c.nblk2 = 2 * h->num_sms;
  }
  return c;
}

// Reads the handle's device error word; a recorded error is cleared and thrown
// (a NaN or infinity in the input: LSQ_E_NONFINITE; an expired wait: LSQ_E_TIMEOUT).
void check_dev_error(lsq_handle* h) {
  int e = 0;
  CK(cudaMemcpyAsync(h->h_pinned, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  std::memcpy(&e, h->h_pinned, sizeof(int));
  if (e != 0) {
    CK(cudaMemsetAsync(h->d_err, 0, sizeof(int), h->stream));
    throw StatusFail{e == DEV_NONFINITE ? LSQ_E_NONFINITE : LSQ_E_TIMEOUT};
  }
}

template <typename S>
S read_state(Ctx& c, const S* d) {
  S s;
  CK(cudaMemcpyAsync(c.h->h_pinned, d, sizeof(S), cudaMemcpyDeviceToHost, c.st));
  CK(cudaStreamSynchronize(c.st));
  std::memcpy(&s, c.h->h_pinned, sizeof(S));
  return s;
}

double read_scalar(Ctx& c, const double* d) { return read_state<double>(c, d); }

// Returns the cached graph for `key`, capturing `body` on the work stream if needed.
CachedGraph* get_graph(Ctx& c, const std::string& key, const std::function<void()>& body) {
  auto it = c.h->graphs.find(key);
  if (it != c.h->graphs.end()) return it->second;
  if (c.h->graphs.size() >= 32) {
    for (auto& kv : c.h->graphs) delete kv.second;
    c.h->graphs.clear();
  }
  auto* G = new CachedGraph();
  const int64_t l0 = c.h->launches;
  c.h->cap = G;
  cudaError_t e = cudaStreamBeginCapture(c.st, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    c.h->cap = nullptr;
    delete G;
    throw CudaFail{e, "cudaStreamBeginCapture"};
  }
  try {
    body();
  } catch (...) {
    c.h->cap = nullptr;
    cudaGraph_t g = nullptr;
    cudaStreamEndCapture(c.st, &g);
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    delete G;
    throw;
  }
  c.h->cap = nullptr;
  e = cudaStreamEndCapture(c.st, &G->g);
  if (e == cudaSuccess) e = cudaGraphInstantiate(&G->e, G->g, 0);
  if (e != cudaSuccess) {
    delete G;
    throw CudaFail{e, "graph capture"};
  }
  G->kernels = c.h->launches - l0;
  c.h->launches = l0;
  c.h->graphs[key] = G;
  return G;
}

void launch_graph(Ctx& c, CachedGraph* G) {
  CK(cudaGraphLaunch(G->e, c.st));
  c.h->launches += G->kernels;
}

std::string graph_key(const char* tag, std::initializer_list<int64_t> vals) {
  std::string k(tag);
  char buf[32];
  for (int64_t v : vals) {
    snprintf(buf, sizeof(buf), ":%llx", (unsigned long long)v);
    k += buf;
  }
  return k;
}

#define PV(p) (int64_t)(uintptr_t)(p)

void finish_timing(lsq_handle* h, lsq_info* info) {
  CK(cudaStreamSynchronize(h->stream));
  if (info) {
    for (int k = 0; k < 8; ++k) info->stage_ms[k] = 0.0;
    for (int k = 0; k < K_NKERN; ++k) {
      info->kern_ms[k] = h->kern_acc[k];
      info->kern_launches[k] = h->kern_cnt[k];
    }
    for (auto& mk : h->marks) {
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, mk.a, mk.b));
      if (mk.stage >= kKernMark) {
        info->kern_ms[mk.stage - kKernMark] += ms;
        info->kern_launches[mk.stage - kKernMark] += 1;
      } else {
        info->stage_ms[mk.stage] += ms;
      }
    }
  }
  h->marks.clear();
  h->next_event = 0;
  for (int k = 0; k < K_NKERN; ++k) {
    h->kern_acc[k] = 0.0;
    h->kern_cnt[k] = 0;
  }
}

lsq_status run_guarded(lsq_handle* h, lsq_info* info, const std::function<lsq_status()>& fn) {
  lsq_status st;
  const int64_t l0 = h->launches;
  try {
    h->marks.clear();
    h->next_event = 0;
    for (int k = 0; k < K_NKERN; ++k) {
      h->kern_acc[k] = 0.0;
      h->kern_cnt[k] = 0;
    }
    CK(cudaEventRecord(h->ev_in, h->user_stream));
    CK(cudaStreamWaitEvent(h->stream, h->ev_in, 0));
    st = fn();
    check_dev_error(h);
    finish_timing(h, info);
    CK(cudaEventRecord(h->ev_out, h->stream));
    CK(cudaStreamWaitEvent(h->user_stream, h->ev_out, 0));
  } catch (const CudaFail& f) {
    h->last_cuda = std::string(f.what) + ": " + cudaGetErrorString(f.e);
    cudaGetLastError();
    st = LSQ_E_CUDA;
    h->marks.clear();
    h->next_event = 0;
  } catch (const StatusFail& f) {
    st = f.st;
    cudaStreamSynchronize(h->stream);
    cudaGetLastError();
    h->marks.clear();
    h->next_event = 0;
  }
  if (info) {
    info->status = st;
    info->gpu_launches = h->launches - l0;
  }
  return st;
}

}  // namespace

// Grouped batched solve (api_batch.cu); LSQ_E_UNSUPPORTED (nothing launched) when the
// batch is outside the grouped path's range.
lsq_status lsq_batch_grouped(lsq_handle* h, int32_t nprob, const lsq_problem* probs, lsq_prec u_s, lsq_prec u_p,
                             lsq_prec u_w, lsq_prec u_r, double tol, const lsq_opts* opts, int32_t* statuses,
                             lsq_info* infos);
