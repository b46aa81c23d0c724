// Loop primitives of the device-driven solves in captured CUDA graphs: a
// WHILE conditional node whose body is captured from a stream.  Under an
// active Recorder (launch.cuh) they record the loop instead.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "launch.cuh"

namespace fnpf {

// A conditional handle in the graph being captured on s (or the next recorded
// handle ordinal).
cudaError_t new_handle(cudaStream_t s, cudaGraphConditionalHandle* h);
// Kernel nodes directly in graph g (not inside nested conditional bodies).
int64_t kernel_nodes(cudaGraph_t g);

// Appends a WHILE node controlled by h to the graph captured on s and captures
// body(bs) into its body graph on stream bs; *body_kernels receives the number
// of kernel nodes of the body.
template <typename F>
cudaError_t capture_while(cudaStream_t s, cudaStream_t bs, cudaGraphConditionalHandle h, int64_t* body_kernels,
                          F&& body) {
  if (Recorder* r = active_recorder()) {
    Op op;
    op.kind = OP_LOOP;
    op.handle = (int)h;
    r->ops.push_back(std::move(op));
    const cudaError_t eb = body(s);
    Op end;
    end.kind = OP_END;
    end.handle = (int)h;
    r->ops.push_back(std::move(end));
    return eb;
  }
  cudaStreamCaptureStatus st;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  const cudaGraphEdgeData* ed = nullptr;
  size_t nd = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(s, &st, nullptr, &g, &deps, &ed, &nd);
  if (e != cudaSuccess) return e;
  cudaGraphNodeParams p{};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = h;
  p.conditional.type = cudaGraphCondTypeWhile;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  if ((e = cudaGraphAddNode(&node, g, deps, ed, nd, &p)) != cudaSuccess) return e;
  if ((e = cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies)) != cudaSuccess)
    return e;
  cudaGraph_t bodyg = p.conditional.phGraph_out[0];
  if ((e = cudaStreamBeginCaptureToGraph(bs, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) !=
      cudaSuccess)
    return e;
  cudaError_t eb = body(bs);
  cudaGraph_t out = nullptr;
  e = cudaStreamEndCapture(bs, &out);
  if (e == cudaSuccess && out) *body_kernels = kernel_nodes(out);
  return eb != cudaSuccess ? eb : e;
}

}  // namespace fnpf
