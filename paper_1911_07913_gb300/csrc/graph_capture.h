// Helpers for building CUDA graphs with conditional nodes by stream capture:
// the capturing graph of a stream, a conditional handle in it, a conditional
// node appended to the capture, and the capture of a node's body graph on a
// second stream (the scene's launches are redirected there meanwhile).
#pragma once
#include "internal.h"

namespace hot {

inline cudaGraph_t capturing_graph(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaGraph_t g = nullptr;
  HOT_CUDA(cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, nullptr, nullptr, nullptr));
  if (cs != cudaStreamCaptureStatusActive || !g) fail(MPM_ERR_CUDA, "stream is not capturing");
  return g;
}

inline cudaGraphConditionalHandle new_handle(cudaStream_t st) {
  cudaGraphConditionalHandle h;
  HOT_CUDA(cudaGraphConditionalHandleCreate(&h, capturing_graph(st), 0, 0));
  return h;
}

// appends a conditional node to the capture on st; returns its body graph
inline cudaGraph_t add_conditional(cudaStream_t st, cudaGraphConditionalHandle h,
                                   cudaGraphConditionalNodeType type) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t *deps = nullptr;
  size_t nd = 0;
  HOT_CUDA(cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, nullptr, &nd));
  if (cs != cudaStreamCaptureStatusActive || !g) fail(MPM_ERR_CUDA, "stream is not capturing");
  cudaGraphNodeParams p = {};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = h;
  p.conditional.type = type;
  p.conditional.size = 1;
  cudaGraphNode_t node = nullptr;
  HOT_CUDA(cudaGraphAddNode(&node, g, deps, nullptr, nd, &p));
  HOT_CUDA(cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  return p.conditional.phGraph_out[0];
}

// runs f with the scene's launches going into body (captured on aux stream k)
template <class F>
void capture_into(Scene &s, int k, cudaGraph_t body, F &&f) {
  cudaStream_t outer = s.st, aux = s.aux_st[k];
  HOT_CUDA(cudaStreamBeginCaptureToGraph(aux, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  s.st = aux;
  try {
    f();
  } catch (...) {
    s.st = outer;
    cudaGraph_t g = nullptr;
    cudaStreamEndCapture(aux, &g);
    throw;
  }
  s.st = outer;
  cudaGraph_t g = nullptr;
  HOT_CUDA(cudaStreamEndCapture(aux, &g));
}

inline void end_any_capture(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (st && cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
    cudaGraph_t g = nullptr;
    cudaStreamEndCapture(st, &g);
    if (g) cudaGraphDestroy(g);
  }
}

}  // namespace hot
