// Ladder energy for callers that cannot allocate device memory.
//
// ladder_energy needs a plan and a workspace: the first stage of its
// reduction writes one partial sum per block into caller-provided device
// memory.  Some callers cannot provide that memory: code that runs inside a
// host framework which owns the whole device-memory budget and hands out no
// scratch, or code paths where calling cudaMalloc is not allowed because it
// may block, synchronise the device or fail at an awkward moment.  For them,
// ladder_energy_noalloc runs the same two reduction kernels with the partial
// sums in a fixed array that lives in this library's own device memory.
//
// The array is a file-scope __device__ variable of kNoAllocPartials doubles
// (4 MiB).  Every GPU that loads the library keeps it until the process
// exits.  Host code cannot use the array's name as a device address, so the
// first call on each device looks the address up with cudaGetSymbolAddress
// (with that device current) and caches it; make that first call before any
// stream capture.  All calls share the array and it keeps the last call's
// partial sums; the first stage overwrites every partial it later reads, so
// nothing needs clearing.  Calls that overlap on the GPU (other streams,
// other host threads) race on the array: serialise them.
#include <mutex>

#include "../../include/ladder.h"
#include "kernels.h"

namespace {

constexpr size_t kNoAllocPartials = (size_t)1 << 19;  // 524288 doubles = 4 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_energy_partials[kNoAllocPartials];

std::mutex g_mutex;
double *g_partials[kMaxDevices] = {nullptr};

bool device_pointer(const void *p) {
  if (!p || (reinterpret_cast<uintptr_t>(p) & 7u)) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" ladder_status ladder_energy_noalloc(int o, int v, const double *R, const double *t2,
                                               double *E_dev, void *stream) {
  if (o < 1 || o > 256 || v < 1 || v > 4096) return LADDER_EINVAL;
  // the reduction writes one partial per (32x32 tile of (a,b), pair (i,j))
  if (ladder::energy_partials(o, v) > kNoAllocPartials) return LADDER_ENOTSUP;
  if (!device_pointer(R) || !device_pointer(t2) || !device_pointer(E_dev)) return LADDER_EINVAL;
  // clear an error left on this thread by an earlier, unrelated call, so that
  // the check after the launch reports this call's launch only
  cudaGetLastError();
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return LADDER_ECUDA;
  }
  double *partials = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_partials[dev]) {
      void *addr = nullptr;
      if (cudaGetSymbolAddress(&addr, g_energy_partials) != cudaSuccess || !addr) {
        cudaGetLastError();
        return LADDER_ECUDA;
      }
      g_partials[dev] = static_cast<double *>(addr);
    }
    partials = g_partials[dev];
  }
  ladder::launch_energy(o, v, R, t2, partials, E_dev, static_cast<cudaStream_t>(stream));
  if (cudaGetLastError() != cudaSuccess) return LADDER_ECUDA;
  return LADDER_OK;
}
