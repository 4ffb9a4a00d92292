// Self-tests of the bounded device waits (include/pc.h, pc_selftest_wait_timeout
// and pc_selftest_scatter_timeout).
// One block waits on a shared-memory barrier that nothing completes, through
// the wait the partition uses for its tile copies; the wait gives up, sets the
// error bit and returns, the kernel ends and the host reads the status.  No
// copy is in flight, nothing faults or hangs.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/pc.h"
#include "pc_internal.cuh"
#include "pc_mbar.cuh"

namespace pcx {
namespace {

__device__ uint32_t g_selftest_err;

__global__ void k_selftest_wait(uint32_t limit) {
  __shared__ __align__(8) unsigned long long bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);  // one arrival expected; none comes
    mbar_fence_init();
  }
  __syncthreads();
  wait_buffer(&bar, 0, &g_selftest_err, limit);
}

}  // namespace
}  // namespace pcx

extern "C" int pc_selftest_wait_timeout(void *stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const uint32_t zero = 0;
  uint32_t err = 0;
  if (cudaMemcpyToSymbolAsync(pcx::g_selftest_err, &zero, 4, 0, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return PC_ERR_CUDA;
  pcx::k_selftest_wait<<<1, 32, 0, st>>>(1u << 12);
  if (cudaGetLastError() != cudaSuccess) return PC_ERR_CUDA;
  if (cudaMemcpyFromSymbolAsync(&err, pcx::g_selftest_err, 4, 0, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return PC_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return PC_ERR_CUDA;
  if (err & pcx::kErrTimeout) return PC_ERR_TIMEOUT;
  return err ? PC_ERR_CUDA : PC_OK;
}

// A compress call whose scatter copies are dropped on the calling thread: the
// scatter's waits give up after kSelftestSpinLimit polls, every block leaves
// on its first tile, and the kernels after it find the error word set.
extern "C" int pc_selftest_scatter_timeout(const void *positions, uint64_t n, int dtype, void *out,
                                           uint64_t out_capacity, void *workspace, uint64_t workspace_bytes,
                                           void *stream) {
  if (n <= (1ull << 16)) return PC_ERR_ARG;
  uint64_t size = 0;
  pcx::set_drop_tile_copies(true);
  const int rc = pcx::compress_device(positions, n, dtype, PC_EB_REL, 1e-3, nullptr, out, out_capacity, &size,
                                      workspace, workspace_bytes, static_cast<cudaStream_t>(stream));
  pcx::set_drop_tile_copies(false);
  return rc;
}
