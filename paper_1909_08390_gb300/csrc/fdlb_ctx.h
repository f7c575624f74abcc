// fdlb_ctx.h -- the context object behind the opaque fdlb_ctx handle, shared
// by the host-side translation units of libfdlb.so.  Not part of the ABI.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "fdlb.h"
#include "fdlb_internal.h"

struct fdlb_ctx {
  fdlb::DevParams dp{};
  cudaStream_t stream = nullptr;
  int device = 0;
  int precision = FDLB_FP64;
  fdlb_grid grid{};
  double gamma = 0, tau = 0, dt = 0;
  void* buf = nullptr;  // one allocation: 6 population arrays, 4 moment fields, status
  double* mom = nullptr;  // device moments buffer (n, ux, uy, T) for host copies
  size_t buf_bytes = 0;
  unsigned* status_host = nullptr;  // pinned
  bool prepared = false;
  std::string err;
  // batches of 1-D problems (fdlb_create_batch)
  bool batch = false;
  std::vector<fdlb::BatchProblem> probs;
  fdlb::BatchProblem* probs_dev = nullptr;
  fdlb::WorkItem* work_dev = nullptr;
  int nsm = 0;
  // CUDA graphs of kGraphSteps steps, captured on first use; FDLB_MIXED
  // contexts keep one per state buffer the steps start from (parity)
  cudaStream_t capture_stream = nullptr;
  cudaGraphExec_t graph_exec[2] = {nullptr, nullptr};
  // FDLB_MIXED: the two state buffers {hi, lo}; the current one is
  // pair[parity], the final stage writes pair[1 - parity]
  float* pair[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  int parity = 0;
  // adjoint: per-step forward states of one checkpoint segment, adjoint
  // work arrays and scalar accumulators (allocated on first use)
  void* adj_buf = nullptr;
  size_t adj_bytes = 0;
  bool custom_tableau = false;  // created with a caller tableau (not Table I)
};

namespace fdlb {
int ctx_error(fdlb_ctx* c, int code, const char* msg);
int ctx_prepare(fdlb_ctx* c);
int ctx_launch_stage(fdlb_ctx* c, int stage, cudaStream_t s);
}  // namespace fdlb

