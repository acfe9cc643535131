// Loops and branches whose conditions only the device knows.
//
// A multi-round computation (the sieve rounds of a build, the levels of a
// skeleton) decides after every step whether another one is needed.  Its
// steps are written once, as host code that enqueues kernels on a stream;
// the condition is a 32-bit word of a device control block that the
// kernels of the step compute.  Two ways to run it:
//
//   host mode   the host copies the control block back after each step and
//               branches on it (one stream synchronisation per test);
//   graph mode  the steps are recorded once into a CUDA graph whose
//               conditional nodes (WHILE, IF) test the same word on the
//               device: a one-thread kernel copies the word into the node's
//               condition handle before the node and at the end of every
//               iteration.  The whole computation then runs from one graph
//               launch with no host round trip.
//
// Both modes launch the same kernels with the same arguments, so they give
// the same results; the control words bound every loop on the device.
#pragma once

#include <cuda_runtime.h>

#include <mutex>
#include <vector>

#include "sieve.cuh"

namespace pkd {

static __global__ void k_flow_cond(cudaGraphConditionalHandle h, const uint32_t* word) {
  cudaGraphSetConditional(h, *word != 0u ? 1u : 0u);
}

// True while this thread records a graph (kernel timers are then off).
bool& flow_capturing();

// A stream of the current device for graph level `level` (created on first
// use; level 0 holds the top-level capture).
cudaStream_t flow_stream(int level);

// Serialises captures: the level streams are shared by every host thread.
std::mutex& flow_mutex();

struct Flow {
  cudaStream_t s;                // stream the step's kernels go to
  bool graph = false;            // recording into a graph
  int level = 0;                 // nesting depth (graph mode)
  const uint32_t* dctl = nullptr;  // device control block
  uint32_t* hctl = nullptr;        // pinned host copy (host mode)
  int nctl = 0;                    // words of the block
  int err = PKD_OK;
};

// Host mode: bring the control block back (one synchronisation).
inline int flow_read(Flow& f) {
  PKD_CUDA(cudaMemcpyAsync(f.hctl, f.dctl, (size_t)f.nctl * 4, cudaMemcpyDeviceToHost, f.s));
  PKD_CUDA(cudaStreamSynchronize(f.s));
  return PKD_OK;
}

// Adds a conditional node of `type` after the work recorded so far on f.s,
// its condition the control word `w` (copied by a kernel launched just
// before it); returns the node's body graph.
inline int flow_cond_node(Flow& f, int w, cudaGraphConditionalNodeType type, cudaGraphConditionalHandle* h,
                          cudaGraph_t* body) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  PKD_CUDA(cudaStreamGetCaptureInfo(f.s, &cs, nullptr, &g, &deps, nullptr, &nd));
  if (cs != cudaStreamCaptureStatusActive) return PKD_EINTERNAL;
  PKD_CUDA(cudaGraphConditionalHandleCreate(h, g, 0, 0));
  PKD_LAUNCH(k_flow_cond<<<1, 1, 0, f.s>>>(*h, f.dctl + w));
  PKD_CUDA(cudaStreamGetCaptureInfo(f.s, &cs, nullptr, &g, &deps, nullptr, &nd));
  cudaGraphNodeParams np{};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = *h;
  np.conditional.type = type;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  PKD_CUDA(cudaGraphAddNode(&node, g, deps, nullptr, nd, &np));
  *body = np.conditional.phGraph_out[0];
  PKD_CUDA(cudaStreamUpdateCaptureDependencies(f.s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  return PKD_OK;
}

// Records `fn(inner)` into `body` on the stream of the next level.
template <class F>
inline int flow_record_body(Flow& f, cudaGraph_t body, F&& fn, cudaGraphConditionalHandle h, int w, bool again) {
  Flow in = f;
  in.level = f.level + 1;
  in.s = flow_stream(in.level);
  if (!in.s) return PKD_ECUDA;
  PKD_CUDA(cudaStreamBeginCaptureToGraph(in.s, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  int e = fn(in);
  if (e == PKD_OK && again) {
    // the condition for the next iteration
    k_flow_cond<<<1, 1, 0, in.s>>>(h, f.dctl + w);
    count_launch();
    if (cudaGetLastError() != cudaSuccess) e = PKD_ECUDA;
  }
  cudaGraph_t out = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(in.s, &out);
  if (e == PKD_OK && ce != cudaSuccess) e = PKD_ECUDA;
  return e;
}

// while (ctl[w] != 0) fn(flow).  fn's kernels must recompute ctl[w]; the
// word is tested before the first iteration too.
template <class F>
inline int flow_while(Flow& f, int w, F&& fn) {
  if (!f.graph) {
    for (;;) {
      PKD_TRY(flow_read(f));
      if (f.hctl[w] == 0) return PKD_OK;
      PKD_TRY(fn(f));
    }
  }
  cudaGraphConditionalHandle h;
  cudaGraph_t body;
  PKD_TRY(flow_cond_node(f, w, cudaGraphCondTypeWhile, &h, &body));
  return flow_record_body(f, body, fn, h, w, true);
}

// if (ctl[w] != 0) fn(flow).
template <class F>
inline int flow_if(Flow& f, int w, F&& fn) {
  if (!f.graph) {
    PKD_TRY(flow_read(f));
    if (f.hctl[w] == 0) return PKD_OK;
    return fn(f);
  }
  cudaGraphConditionalHandle h;
  cudaGraph_t body;
  PKD_TRY(flow_cond_node(f, w, cudaGraphCondTypeIf, &h, &body));
  return flow_record_body(f, body, fn, h, w, false);
}

}  // namespace pkd
