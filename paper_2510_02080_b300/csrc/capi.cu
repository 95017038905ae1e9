// Context management and status handling of the C ABI (include/ec3r.h).
#include "common.cuh"

using namespace ec3r;

extern "C" {

const char* ec3r_version(void) { return "ec3r 0.1 sm_103a"; }

const char* ec3r_status_string(ec3r_status st) {
  switch (st) {
    case EC3R_OK: return "ok";
    case EC3R_ERR_INVALID_ARG: return "invalid argument";
    case EC3R_ERR_CUDA: return "CUDA error";
    case EC3R_ERR_OOM: return "out of device memory";
    case EC3R_ERR_CAPACITY: return "output capacity exceeded";
    case EC3R_ERR_NOT_SPD: return "normal equations not positive definite";
    case EC3R_ERR_TIMEOUT: return "device wait timed out";
    case EC3R_ERR_DEGENERATE: return "degenerate registration pair";
    case EC3R_ERR_CAPTURE: return "workspace growth during stream capture";
  }
  return "unknown status";
}

ec3r_status ec3r_create(ec3r_ctx** out, int device) {
  if (!out) return EC3R_ERR_INVALID_ARG;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
    cudaGetLastError();
    return EC3R_ERR_INVALID_ARG;
  }
  ec3r_ctx* c = new ec3r_ctx();
  c->device = device;
  if (cudaSetDevice(device) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device) !=
          cudaSuccess ||
      cudaDeviceGetAttribute(&c->clock_khz, cudaDevAttrClockRate, device) != cudaSuccess ||
      cudaMalloc(&c->d_flags, sizeof(unsigned)) != cudaSuccess ||
      cudaMemset(c->d_flags, 0, sizeof(unsigned)) != cudaSuccess ||
      cudaMallocHost(&c->h_flags, sizeof(unsigned)) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    ec3r_destroy(c);
    return EC3R_ERR_CUDA;
  }
  *out = c;
  return EC3R_OK;
}

void ec3r_destroy(ec3r_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  drop_graphs(c);
  for (auto& kv : c->bufs)
    if (kv.second.ptr) cudaFree(kv.second.ptr);
  for (auto& kv : c->ext) delete kv.second;
  for (auto& r : c->prof) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : c->prof_pool) cudaEventDestroy(e);
  if (c->d_flags) cudaFree(c->d_flags);
  if (c->h_flags) cudaFreeHost(c->h_flags);
  if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
  delete c;
}

const char* ec3r_last_error(const ec3r_ctx* c) {
  return c ? c->last_error.c_str() : "null context";
}

ec3r_status ec3r_sync_status(ec3r_ctx* c, void* stream) {
  if (!c) return EC3R_ERR_INVALID_ARG;
  EC3R_CUDA_TRY(c, cudaSetDevice(c->device));
  cudaStream_t s = (cudaStream_t)stream;
  EC3R_CUDA_TRY(c, cudaMemcpyAsync(c->h_flags, c->d_flags, sizeof(unsigned),
                                   cudaMemcpyDeviceToHost, s));
  EC3R_CUDA_TRY(c, cudaMemsetAsync(c->d_flags, 0, sizeof(unsigned), s));
  EC3R_CUDA_TRY(c, cudaStreamSynchronize(s));
  unsigned f = *c->h_flags;
  if (f & FLAG_TIMEOUT) return set_error(c, EC3R_ERR_TIMEOUT, "a bounded device wait gave up");
  if (f & FLAG_NOT_SPD)
    return set_error(c, EC3R_ERR_NOT_SPD, "pose-graph normal equations not positive definite");
  if (f & FLAG_CAPACITY)
    return set_error(c, EC3R_ERR_CAPACITY, "fuse_points output capacity exceeded");
  if (f & FLAG_BAD_INDEX)
    return set_error(c, EC3R_ERR_INVALID_ARG, "an index argument was out of range");
  return EC3R_OK;
}

ec3r_status ec3r_set_wait_limit(ec3r_ctx* c, double seconds) {
  if (!c || !(seconds >= 0.0) || seconds > 3600.0) return EC3R_ERR_INVALID_ARG;
  c->wait_limit_s = seconds;
  drop_graphs(c);  // cached graphs hold the old limit as a launch argument
  return EC3R_OK;
}

ec3r_status ec3r_align_backward_set_ctas_per_sm(ec3r_ctx* c, int ctas_per_sm) {
  if (!c || ctas_per_sm < 0 || ctas_per_sm > 4) return EC3R_ERR_INVALID_ARG;
  if (c->bwd_ctas_per_sm != ctas_per_sm) drop_graphs(c);  // the grid is in the graphs
  c->bwd_ctas_per_sm = ctas_per_sm;
  return EC3R_OK;
}

ec3r_status ec3r_inject(ec3r_ctx* c, unsigned what) {
  if (!c || (what & ~(unsigned)(EC3R_INJECT_LOOPS_NO_COPY | EC3R_INJECT_ALIGN_NO_EPOCH)))
    return EC3R_ERR_INVALID_ARG;
  c->inject = what;
  drop_graphs(c);
  return EC3R_OK;
}

ec3r_status ec3r_profile(ec3r_ctx* c, int enable) {
  if (!c) return EC3R_ERR_INVALID_ARG;
  c->profiling = enable != 0;
  return EC3R_OK;
}

ec3r_status ec3r_profile_read(ec3r_ctx* c, int max_kernels, char* names, int name_len,
                              double* total_ms, int64_t* launches, int* n_kernels) {
  if (!c || max_kernels < 0 || name_len < 1 || !n_kernels ||
      (max_kernels > 0 && (!names || !total_ms || !launches)))
    return EC3R_ERR_INVALID_ARG;
  EC3R_CUDA_TRY(c, cudaSetDevice(c->device));
  std::vector<std::string> order;
  std::map<std::string, std::pair<double, int64_t>> acc;
  for (auto& r : c->prof) {
    EC3R_CUDA_TRY(c, cudaEventSynchronize(r.b));
    float ms = 0.f;
    EC3R_CUDA_TRY(c, cudaEventElapsedTime(&ms, r.a, r.b));
    auto it = acc.find(r.name);
    if (it == acc.end()) {
      order.push_back(r.name);
      acc[r.name] = {ms, 1};
    } else {
      it->second.first += ms;
      it->second.second += 1;
    }
    c->prof_pool.push_back(r.a);
    c->prof_pool.push_back(r.b);
  }
  c->prof.clear();
  *n_kernels = (int)order.size();
  for (int i = 0; i < (int)order.size() && i < max_kernels; ++i) {
    snprintf(names + (size_t)i * name_len, name_len, "%s", order[i].c_str());
    total_ms[i] = acc[order[i]].first;
    launches[i] = acc[order[i]].second;
  }
  return EC3R_OK;
}

}  // extern "C"
