// fdlb_peak.cu -- measurement aid: the binary64 pipe's sustained rate on this
// GPU (no paper counterpart).  The stage kernels of binary64 contexts are
// bound by the binary64 pipe, whose nominal rate (2 lanes per clock per SM on
// GB300) is not a figure a kernel of real instructions reaches; this kernel
// measures what independent fused multiply-adds alone reach, as the roofline
// denominator of those kernels.
#include <cuda_runtime.h>

#include "fdlb.h"

namespace {

constexpr int kChains = 8;     // independent dependency chains per thread
constexpr int kThreads = 256;  // threads per CTA

__device__ double g_sink;  // the chains' sum lands here only if it is -1 (never)

// kChains independent chains x = x * b + c per thread, iters rounds each: one
// DFMA per chain and round.  b and c come from the host so nothing folds; the
// store is conditional on a value the chains never reach (every chain stays
// positive), so nothing is removed.
__global__ void __launch_bounds__(kThreads) dfma_chains(double b, double c, int iters) {
  double x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = (double)(threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  if (s == -1.0) g_sink = s;
}

}  // namespace

extern "C" int fdlb_measure_fp64_pipe(void* cuda_stream, double* dfma_per_s, double* ms_out) {
  if (!dfma_per_s) return FDLB_EINVAL;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return FDLB_ECUDA;
  const int blocks = 8 * nsm;  // 2048 threads per SM resident
  const int iters = 4096;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  float best = 1e30f;
  // b = 1 - 2^-30 and c = 2^-30 keep every chain positive and near its
  // start (no overflow, no subnormals)
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
    e = cudaEventRecord(t0, s);
    if (e == cudaSuccess) {
      dfma_chains<<<blocks, kThreads, 0, s>>>(1.0 - 0x1p-30, 0x1p-30, iters);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(t1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(t1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
    if (e == cudaSuccess && rep > 0 && ms < best) best = ms;  // the first launch warms up
  }
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  if (e != cudaSuccess) return FDLB_ECUDA;
  const double ops = (double)blocks * kThreads * kChains * iters;
  *dfma_per_s = ops / (best * 1e-3);
  if (ms_out) *ms_out = best;
  return FDLB_OK;
}
