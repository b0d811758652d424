// ||A||_2 estimate for callers that cannot allocate device memory.
//
// Some callers may not call cudaMalloc at all: code that runs while a host
// framework owns every byte of device memory and hands out only its own
// buffers, or code that must not add allocations in a phase where the memory
// budget is fixed.  feast_norm2_estimate_static serves them.  It runs the
// power-iteration kernel of the handle path (norm2.cu) on the caller's device
// matrix, and takes the kernel's scratch -- two n-vectors, one partial sum per
// block and the grid-barrier words -- from the fixed array below, which every
// GPU that loads this library holds until the process exits.
//
// Limits and contract:
//   * n <= kStaticMaxN (16384); larger orders return FEAST_ERR_TOO_LARGE.
//   * On each device the first call looks up the array's device address
//     (cudaGetSymbolAddress, with that device current).  Make that first call
//     before any stream capture begins.
//   * Every call shares the one array and leaves the last call's values in
//     it; calls whose work overlaps on the GPU (other streams, other host
//     threads on the same device) race on it.  Serialise them.
//   * No cudaMalloc, cudaFree or other allocating routine is called.
#include <mutex>

#include "../../include/feast_gb300.h"
#include "norm2.cuh"

namespace {

constexpr int kStaticMaxN = 16384;
constexpr size_t kTail = 256;  // output value (offset 0) and flag word (offset 64)
constexpr size_t kKernelBytes = 256 + (size_t)2 * kStaticMaxN * sizeof(double2) + 1024 * sizeof(double);
constexpr size_t kStaticBytes = kKernelBytes + kTail;  // 532,992 bytes (520.5 KiB)

static __device__ __align__(256) unsigned char g_norm2_static[kStaticBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

}  // namespace

extern "C" feast_status feast_norm2_estimate_static(const feast_z* A, int64_t n, int64_t lda, int iters,
                                                     double* norm, void* stream) {
  if (n > kStaticMaxN) return FEAST_ERR_TOO_LARGE;
  if (!A || !norm || n < 1 || lda < n || iters < 1) return FEAST_ERR_ARG;
  if (norm2_scratch_bytes((int)n) > kKernelBytes) return FEAST_ERR_TOO_LARGE;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, A) != cudaSuccess) {
    cudaGetLastError();
    return FEAST_ERR_ARG;
  }
  if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) return FEAST_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return FEAST_ERR_CUDA;
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_norm2_static) != cudaSuccess || !p) return FEAST_ERR_CUDA;
      g_addr[dev] = p;
    }
    base = g_addr[dev];
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  char* b = reinterpret_cast<char*>(base);
  double* out = reinterpret_cast<double*>(b + kKernelBytes);
  unsigned* flags = reinterpret_cast<unsigned*>(b + kKernelBytes + 64);
  // the flag word must start at zero; norm2_power clears the barrier words itself
  if (cudaMemsetAsync(flags, 0, sizeof(unsigned), s) != cudaSuccess) return FEAST_ERR_CUDA;
  if (norm2_power(reinterpret_cast<const double2*>(A), lda, (int)n, iters, b, out, flags, s) != cudaSuccess)
    return FEAST_ERR_CUDA;
  unsigned f = 0;
  if (cudaMemcpyAsync(norm, out, sizeof(double), cudaMemcpyDefault, s) != cudaSuccess) return FEAST_ERR_CUDA;
  if (cudaMemcpyAsync(&f, flags, sizeof(unsigned), cudaMemcpyDeviceToHost, s) != cudaSuccess) return FEAST_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return FEAST_ERR_CUDA;
  if (f & DEVFLAG_TIMEOUT) return FEAST_ERR_DEVICE_TIMEOUT;
  return FEAST_OK;
}
