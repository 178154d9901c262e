// Test hook for the bounded waits of the tensor-core kernels: one CTA waits on
// an mbarrier that nothing completes, with the same bounded wait the
// pipelines use, and reports TIMEOUT when the bound runs out.  No fault, trap
// or endless loop: the wait gives up after `polls` polls and the kernel exits.
#include "common.cuh"
#include "kernels.h"
#include "tc.cuh"
#include "../../include/mrcqr.h"

namespace mrcqr {
namespace {

__global__ void k_wait_timeout(uint32_t polls, int32_t* __restrict__ status) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    tc::mbar_fence_init();
  }
  __syncthreads();
  const bool ok = tc::mbar_wait(&bar, 0u, polls);   // phase 0 never completes: no thread arrives
  if (threadIdx.x == 0) *status = ok ? MRCQR_OK : MRCQR_ERR_TIMEOUT;
}

}  // namespace
}  // namespace mrcqr

extern "C" int mrcqr_debug_wait_timeout(uint32_t polls, int32_t* status, mrcqr_stream_t stream) {
  if (!status || polls < 1 || polls > (1u << 20)) return MRCQR_ERR_INVALID;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  { ::mrcqr::note_launch(); mrcqr::k_wait_timeout<<<1, 32, 0, st>>>(polls, status); }
  return cudaGetLastError() == cudaSuccess ? MRCQR_OK : MRCQR_ERR_CUDA;
}
