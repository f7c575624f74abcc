// fdlb_noalloc.cu -- fdlb_step_noalloc: the IMEX step for callers that must
// not allocate device memory.
//
// The stage kernels need five scratch arrays next to the caller's state
// (stage-2 and stage-3 populations, the two running explicit parts and
// F - F_eq) plus a status word.  fdlb_create obtains them with cudaMalloc;
// this entry point takes them from one file-scope __device__ array of fixed
// size instead, so it calls no allocator at all.  Every GPU that loads the
// library keeps that array for the life of the process.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "fdlb.h"
#include "fdlb_internal.h"

namespace fdlb {
int params_for(const fdlb_grid* grid, int Qphi, int Qchi, double gamma, double tau, double dt,
               const fdlb_tableau* tableau, DevParams* out);
int record_error(int code, const char* msg);
}  // namespace fdlb

namespace {

constexpr size_t kScratchBytes = (size_t)FDLB_NOALLOC_SCRATCH_BYTES;
constexpr size_t kStatusBytes = 256;

// Shared by every call on a device; holds the last call's contents.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device, looked up once per
// device (host code may not take the address of a __device__ symbol).
int scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fdlb::record_error(FDLB_ECUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices)
    return fdlb::record_error(FDLB_EINVAL, "device ordinal out of range for the static scratch");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return fdlb::record_error(FDLB_ECUDA, cudaGetErrorString(e));
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return FDLB_OK;
}

int cuda_fail(cudaError_t e) { return fdlb::record_error(FDLB_ECUDA, cudaGetErrorString(e)); }

}  // namespace

extern "C" int fdlb_step_noalloc(const fdlb_grid* grid, int Qphi, int Qchi, double gamma,
                                 double tau, double dt, const fdlb_tableau* tableau, double* F,
                                 int64_t nsteps, void* cuda_stream) {
  if (!F) return fdlb::record_error(FDLB_EINVAL, "F is NULL");
  if (nsteps < 0) return fdlb::record_error(FDLB_EINVAL, "nsteps < 0");
  fdlb::DevParams p{};
  int rc = fdlb::params_for(grid, Qphi, Qchi, gamma, tau, dt, tableau, &p);
  if (rc) return rc;
  const size_t arr = (size_t)p.P * (size_t)p.N * sizeof(double);
  if (arr > (kScratchBytes - kStatusBytes) / 5)
    return fdlb::record_error(FDLB_EINVAL,
                              "problem too large for fdlb_step_noalloc: 5 * P * cells * 8 bytes "
                              "must not exceed FDLB_NOALLOC_SCRATCH_BYTES - 256");
  void* base = nullptr;
  rc = scratch_address(&base);
  if (rc) return rc;
  char* b = (char*)base;
  p.F = F;
  p.F2 = (double*)(b + 0 * arr);
  p.F3 = (double*)(b + 1 * arr);
  p.A4 = (double*)(b + 2 * arr);
  p.Af = (double*)(b + 3 * arr);
  p.D = (double*)(b + 4 * arr);
  p.status = (unsigned*)(b + 5 * arr);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  // the status word must start at zero; every other scratch element is
  // written before it is read
  cudaError_t e = cudaMemsetAsync(p.status, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return cuda_fail(e);
  int le = fdlb::launch_stage(p, fdlb::kPrep, s);
  for (int64_t k = 0; k < nsteps && !le; ++k)
    for (int st : {fdlb::kStage3, fdlb::kStage4, fdlb::kFinal})
      if (!le) le = fdlb::launch_stage(p, st, s);
  if (le) return cuda_fail((cudaError_t)le);
  unsigned status = 0;
  e = cudaMemcpyAsync(&status, p.status, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e);
  if (status & 1u)
    return fdlb::record_error(FDLB_EUNSTABLE,
                              "a cell reached n <= 0, T <= 0 or a non-finite moment");
  return FDLB_OK;
}
