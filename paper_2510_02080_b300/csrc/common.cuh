// Internal definitions shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include "../../include/ec3r.h"

namespace ec3r {

// Device status word bits (ctx->d_flags); read and cleared by ec3r_sync_status.
enum : unsigned {
  FLAG_CAPACITY = 1u,
  FLAG_NOT_SPD = 2u,
  FLAG_TIMEOUT = 4u,
  FLAG_BAD_INDEX = 8u,
};

// A growable device buffer owned by a context.
struct DevBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
};

struct GraphEntry {
  cudaGraphExec_t exec = nullptr;
  uint64_t last_use = 0;
};

// Per-context state of other modules, destroyed with the context.
struct Extension {
  virtual ~Extension() {}
};

}  // namespace ec3r

namespace ec3r {
// Per-kernel CUDA-event timing (ec3r_profile): each profiled launch records an
// event pair on its own stream.
struct ProfRec {
  const char* name;
  cudaEvent_t a, b;
};
}  // namespace ec3r

struct ec3r_ctx {
  int device = 0;
  bool profiling = false;
  std::vector<ec3r::ProfRec> prof;
  std::vector<cudaEvent_t> prof_pool;
  int sm_count = 0;
  std::string last_error;
  unsigned* d_flags = nullptr;  // device status word
  unsigned* h_flags = nullptr;  // pinned mirror
  cudaStream_t capture_stream = nullptr;
  std::map<std::string, ec3r::DevBuf> bufs;
  std::map<std::string, ec3r::GraphEntry> graphs;
  std::map<std::string, ec3r::Extension*> ext;
  uint64_t clock = 0;
  // The last registration call: its token (0: none, or it failed), the key of
  // its inputs and options, and whether it formed the cost.  Its
  // checkpoints, per-pair activity and cost live in the align.* workspace;
  // a backward call given this token reuses them.
  uint64_t align_token = 0;
  uint64_t align_tokens_issued = 0;
  std::string align_args;
  bool align_had_cost = false;
  // Registration sweep variants: a forced choice (-1: choose by timing), per
  // size bucket the chosen variant and every variant's measured time (ms),
  // and the variant and times of the last call.
  int align_force = -1;
  int align_last_variant = -1;
  std::vector<float> align_last_ms;
  std::map<uint64_t, std::pair<int, std::vector<float>>> align_tune;
  // Bounded device waits: the limit (seconds; 0 = the default of two
  // seconds), the SM clock that converts it to cycles, and test-only
  // injections that make a wait run out (EC3R_INJECT_*).
  double wait_limit_s = 0.0;
  int clock_khz = 0;
  unsigned inject = 0;
  // CTAs per SM of the backward call's reduction sweeps (0: one CTA per tile,
  // as many resident as fit)
  int bwd_ctas_per_sm = 0;
};

namespace ec3r {

inline ec3r_status set_error(ec3r_ctx* ctx, ec3r_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (ctx) ctx->last_error = buf;
  return st;
}

#define EC3R_CUDA_TRY(ctx, expr)                                                     \
  do {                                                                               \
    cudaError_t _e = (expr);                                                         \
    if (_e != cudaSuccess)                                                           \
      return ::ec3r::set_error((ctx), EC3R_ERR_CUDA, "%s failed: %s (%s:%d)", #expr, \
                               cudaGetErrorString(_e), __FILE__, __LINE__);          \
  } while (0)

// True when `stream` is currently being captured into a graph.
inline bool stream_capturing(cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return cs != cudaStreamCaptureStatusNone;
}

inline void drop_graphs(ec3r_ctx* ctx) {
  for (auto& kv : ctx->graphs) cudaGraphExecDestroy(kv.second.exec);
  ctx->graphs.clear();
}

// Grow-only workspace: returns the buffer named `name` with at least `bytes`.
inline ec3r_status ensure_buf(ec3r_ctx* ctx, const char* name, size_t bytes, cudaStream_t s,
                              void** out) {
  DevBuf& b = ctx->bufs[name];
  if (b.bytes < bytes) {
    if (stream_capturing(s))
      return set_error(ctx, EC3R_ERR_CAPTURE,
                       "workspace '%s' must grow to %zu bytes during stream capture", name,
                       bytes);
    // Every cached graph may reference the old buffer: drop them.
    drop_graphs(ctx);
    if (b.ptr) {
      cudaDeviceSynchronize();
      cudaFree(b.ptr);
      b.ptr = nullptr;
      b.bytes = 0;
    }
    size_t want = bytes + bytes / 4 + 256;
    if (cudaMalloc(&b.ptr, want) != cudaSuccess) {
      cudaGetLastError();
      b.ptr = nullptr;
      return set_error(ctx, EC3R_ERR_OOM, "cudaMalloc(%zu) for workspace '%s' failed", want,
                       name);
    }
    b.bytes = want;
  }
  *out = b.ptr;
  return EC3R_OK;
}

// Runs `enqueue(stream)` either directly (when `user` is being captured, so the
// work lands in the caller's graph) or through a CUDA graph cached under `key`
// and launched on `user`.
template <class F>
ec3r_status run_graph(ec3r_ctx* ctx, const std::string& key, cudaStream_t user, F&& enqueue) {
  if (ctx->profiling || stream_capturing(user)) return enqueue(user);
  auto it = ctx->graphs.find(key);
  if (it == ctx->graphs.end()) {
    if (ctx->graphs.size() >= 32) {
      auto victim = ctx->graphs.begin();
      for (auto j = ctx->graphs.begin(); j != ctx->graphs.end(); ++j)
        if (j->second.last_use < victim->second.last_use) victim = j;
      cudaGraphExecDestroy(victim->second.exec);
      ctx->graphs.erase(victim);
    }
    cudaStream_t cs = ctx->capture_stream;
    EC3R_CUDA_TRY(ctx, cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    ec3r_status st = enqueue(cs);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(cs, &g);
    if (st != EC3R_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    if (e != cudaSuccess)
      return set_error(ctx, EC3R_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess)
      return set_error(ctx, EC3R_ERR_CUDA, "graph instantiate failed: %s",
                       cudaGetErrorString(e));
    it = ctx->graphs.emplace(key, GraphEntry{exec, 0}).first;
  }
  it->second.last_use = ++ctx->clock;
  EC3R_CUDA_TRY(ctx, cudaGraphLaunch(it->second.exec, user));
  return EC3R_OK;
}

inline cudaEvent_t prof_event(ec3r_ctx* ctx) {
  if (!ctx->prof_pool.empty()) {
    cudaEvent_t e = ctx->prof_pool.back();
    ctx->prof_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

// Brackets the kernel launches made by `launch()` with an event pair tagged
// `name` when profiling is on and `s` is not being captured.
template <class F>
inline void traced(ec3r_ctx* ctx, cudaStream_t s, const char* name, F&& launch) {
  if (!ctx->profiling || stream_capturing(s)) {
    launch();
    return;
  }
  cudaEvent_t a = prof_event(ctx), b = prof_event(ctx);
  if (a) cudaEventRecord(a, s);
  launch();
  if (b) cudaEventRecord(b, s);
  if (a && b) ctx->prof.push_back(ProfRec{name, a, b});
}

// The wait limit in SM cycles (clock64 counts at the SM clock, at most the
// peak clock, so the limit in seconds is an upper bound of the real wait).
inline long long wait_limit_cycles(const ec3r_ctx* ctx) {
  const double s = ctx->wait_limit_s > 0.0 ? ctx->wait_limit_s : 2.0;
  const double khz = ctx->clock_khz > 0 ? (double)ctx->clock_khz : 2.0e6;
  return (long long)(s * khz * 1e3);
}

// Launches `kernel` with programmatic stream serialization: it may be
// scheduled before the previous kernel in the stream finishes (the kernel
// itself must wait for it, griddepcontrol.wait, before touching memory).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t s, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

inline std::string key_of(const char* tag, std::initializer_list<uint64_t> vals) {
  std::string k(tag);
  char b[24];
  for (uint64_t v : vals) {
    snprintf(b, sizeof(b), ":%llx", (unsigned long long)v);
    k += b;
  }
  return k;
}

inline uint64_t fbits(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  return u;
}

inline uint64_t dbits(double d) {
  uint64_t u;
  memcpy(&u, &d, 8);
  return u;
}

}  // namespace ec3r
