// CUDA-graph cache of the 1D and 2D runtimes (api.cu, api2d.cu).  A launch
// sequence is captured once per key on the handle's private stream,
// instantiated, and afterwards replayed with one cudaGraphLaunch on the
// caller's stream.  If the caller's stream is itself being captured, the
// sequence is issued directly into that capture instead.
//
// H is a handle type with members `cudaStream_t cap`,
// `std::map<std::string, cudaGraphExec_t> graphs` and `std::string err`.
#pragma once
#include <cuda_runtime.h>
#include <stdio.h>

#include <functional>
#include <map>
#include <string>

#include "swept.h"

namespace swept_graphs {

inline std::string key_of(const char* kind, const void* u, int64_t a, int64_t b = 0) {
  char buf[128];
  snprintf(buf, sizeof buf, "%s:%p:%lld:%lld", kind, u, (long long)a, (long long)b);
  return buf;
}

template <class H>
swept_status cuda_error(H* h, cudaError_t e, const char* where) {
  if (h) h->err = std::string(where) + ": " + cudaGetErrorString(e);
  return SWEPT_ECUDA;
}

template <class H>
swept_status run(H* h, const std::string& key, cudaStream_t user,
                 const std::function<cudaError_t(cudaStream_t)>& issue) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(user, &cs);
  if (e != cudaSuccess) return cuda_error(h, e, "cudaStreamIsCapturing");
  if (cs != cudaStreamCaptureStatusNone) {
    e = issue(user);
    return e == cudaSuccess ? SWEPT_OK : cuda_error(h, e, "kernel launch");
  }
  auto it = h->graphs.find(key);
  if (it == h->graphs.end()) {
    e = cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_error(h, e, "cudaStreamBeginCapture");
    const cudaError_t le = issue(h->cap);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(h->cap, &graph);
    if (le != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return cuda_error(h, le, "kernel launch during capture");
    }
    if (e != cudaSuccess) return cuda_error(h, e, "cudaStreamEndCapture");
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_error(h, e, "cudaGraphInstantiate");
    it = h->graphs.emplace(key, exec).first;
  }
  e = cudaGraphLaunch(it->second, user);
  return e == cudaSuccess ? SWEPT_OK : cuda_error(h, e, "cudaGraphLaunch");
}

template <class H>
void drop(H* h) {
  for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
  h->graphs.clear();
}

}  // namespace swept_graphs
