// Helpers to build CUDA graphs with conditional nodes from the library's launch
// functions: the straight-line parts are captured from a private stream into a
// given graph, loops and branches are conditional nodes whose conditions the
// kernels set on the device.
#pragma once

#include <vector>

#include "afc_internal.h"

namespace afc {

// Capture the launches `body()` issues (on p->stream, which is redirected to the
// capture stream) into graph g after the nodes `deps`; `frontier` receives the
// nodes the next work must follow.
template <class F>
int capture_into(afc_problem_s* p, cudaStream_t cs, cudaGraph_t g, const std::vector<cudaGraphNode_t>& deps,
                 F&& body, std::vector<cudaGraphNode_t>& frontier) {
  cudaStream_t saved = p->stream;
  cudaError_t e = cudaStreamBeginCaptureToGraph(cs, g, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(),
                                                cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCaptureToGraph");
  p->stream = cs;
  int st = body();
  p->stream = saved;
  cudaStreamCaptureStatus cst;
  const cudaGraphNode_t* d = nullptr;
  size_t nd = 0;
  e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, nullptr, &d, nullptr, &nd);
  std::vector<cudaGraphNode_t> fr;
  if (e == cudaSuccess) fr.assign(d, d + nd);
  cudaGraph_t out = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(cs, &out);
  if (st) return st;
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamGetCaptureInfo");
  if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
  frontier = fr;
  return AFC_OK;
}

// Add a conditional node (while / if) after `deps`; *body receives its body graph.
inline int add_conditional(cudaGraph_t g, const std::vector<cudaGraphNode_t>& deps, cudaGraphConditionalHandle h,
                           cudaGraphConditionalNodeType type, cudaGraph_t* body, cudaGraphNode_t* node) {
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = type;
  np.conditional.size = 1;
  cudaError_t e = cudaGraphAddNode(node, g, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(), &np);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphAddNode(conditional)");
  *body = np.conditional.phGraph_out[0];
  return AFC_OK;
}

// Krylov solve of `system` appended to graph g after `frontier` (updated): the
// solver's loop is a while node whose condition the iteration kernels keep.
int krylov_graph(afc_problem_s* p, int system, const afc_opts* o, const double* rhs, double* x, cudaStream_t cs,
                 cudaGraph_t g, std::vector<cudaGraphNode_t>& frontier, const KrylovEpilogue* epi = nullptr,
                 bool* epi_done = nullptr);

// device address of the solver scalars (iteration count at slot kKrylovItsSlot)
const double* krylov_scalars(afc_problem_s* p);
constexpr int kKrylovItsSlot = 7;
constexpr int kKrylovDoneSlot = 8;
// 1 after a grid barrier of the persistent BiCGStab launch gave up waiting
constexpr int kKrylovBarrierErrSlot = 19;

// fixed-point scalar slots (problem scalars p->scal)
enum : int {
  F_NORMSQ = 0, F_CORR = 1, F_INNER = 2, F_RES0 = 3, F_RESF = 4, F_STATUS = 5, F_THRESH = 6, F_FIXED = 7,
  F_MAXIT = 8, F_KBODY = 9, F_REVAL = 10, F_TIMEOUT = 11
};
// F_STATUS: 0 running, 1 converged / fixed count reached, 2 non-finite or a solver that
// could not finish, 3 iteration limit; F_TIMEOUT: 1 after a grid barrier of the
// persistent BiCGStab gave up waiting (F_STATUS is then 2)
int krylov_cycles_slot();
// Clear the grid barrier state of the persistent BiCGStab after a timeout (its
// counter is left inconsistent when blocks skip barriers); synchronises the stream.
int krylov_reset_barrier(afc_problem_s* p);

}  // namespace afc
