// pc_compress_noalloc: compression with library-owned, statically sized scratch.
//
// Some callers may not allocate device memory at all: code that runs inside
// another framework's memory pool (an in-situ analysis hook or a plugin that is
// only handed its input and output buffers), code on a latency-critical path
// where cudaMalloc / cudaFree could synchronise the device or take driver
// locks, and code that must keep a fixed, known device footprint.  For them
// this entry point takes the scratch that pc_compress would take from the
// caller out of one file-scope device array instead.  The caller still passes
// the positions and the output buffer.
//
// Rules of use (also stated in include/pc.h):
//   - the array is kPcNoallocScratchBytes (48 MiB); every GPU that loads this
//     part of the library keeps it until the process exits;
//   - a problem whose scratch does not fit (above about 2^20 particles at the
//     default leaf size) is rejected with PC_ERR_CAPACITY before any work;
//   - the first call on each device looks up the array's device address
//     (cudaGetSymbolAddress, with that device current) and caches it, so make
//     that first call before any stream capture; a cudaDeviceReset invalidates
//     the cached address (the module is loaded again), so the entry point must
//     not be called on a device after a reset;
//   - every call on a device uses the same array, which keeps the contents of
//     the last call; the parts that must start at zero are cleared on every
//     call, but calls whose work overlaps on the GPU (two streams, two host
//     threads) race on the array and must be serialised by the caller.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "../../include/pc.h"
#include "pc_host.cuh"
#include "pc_internal.cuh"

namespace {

constexpr uint64_t kPcNoallocScratchBytes = uint64_t(PC_NOALLOC_SCRATCH_BYTES);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kPcNoallocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (looked up once).
int scratch_address(void **ptr) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PC_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return PC_ERR_CUDA;
    g_scratch_addr[dev] = p;
  }
  *ptr = g_scratch_addr[dev];
  return PC_OK;
}

}  // namespace

extern "C" int pc_compress_noalloc(const void *positions, uint64_t n, int dtype, int eb_mode, double eb,
                                   const pc_config *cfg, void *out, uint64_t out_capacity, uint64_t *out_size,
                                   void *stream) {
  if (!out || !out_size) return PC_ERR_ARG;
  uint64_t need = 0;
  const int rc = pc_compress_workspace_size(n, dtype, cfg, 0, &need);
  if (rc != PC_OK) return rc;
  if (need > kPcNoallocScratchBytes) return PC_ERR_CAPACITY;
  void *scratch = nullptr;
  const int ac = scratch_address(&scratch);
  if (ac != PC_OK) return ac;
  // nor host memory: no page-locked staging block is allocated for the read-backs
  pcx::set_no_host_alloc(true);
  const int cc = pcx::compress_device(positions, n, dtype, eb_mode, eb, cfg, out, out_capacity, out_size, scratch,
                                      kPcNoallocScratchBytes, static_cast<cudaStream_t>(stream));
  pcx::set_no_host_alloc(false);
  return cc;
}
