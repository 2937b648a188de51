// noalloc.cu -- an inner product that performs no device allocation of any kind.
//
// mpk_dot obtains its reduction scratch (per-block partial sums and a completion counter) from
// the stream-ordered allocator on every call.  Some callers cannot let a library allocate: a
// host that hands the library a fixed device-memory budget and forbids further driver
// allocations, a latency-critical loop in which an allocation might synchronise the device, or
// a plugin environment whose allocator owns all device memory.  mpk_dot_noalloc serves them: the
// same kernel and the same fixed summation order as mpk_dot, with the scratch taken from a
// file-scope device array of fixed size that every GPU loading this library keeps until the
// process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "internal.h"

namespace mpk {
namespace {

// Largest vector length accepted: 2^24 entries.  The reduction uses one partial sum (up to 8
// doubles: complex QD) per block of 4096 entries, plus one counter.
constexpr int kNoAllocMaxN = 1 << 24;
constexpr size_t kNoAllocPartials = ((size_t)kNoAllocMaxN / 4096) * 8;  // doubles

// The scratch itself.  In host code this name is only a stand-in for the symbol: its device
// address must be obtained with cudaGetSymbolAddress on each device.
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocPartials + 32];

constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mutex;

// Device address of the scratch on the current device, looked up once per device.
int scratch_address(double** out) {
  int dev = 0;
  MPK_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(MPK_INVALID_ARG, "device index out of range for mpk_dot_noalloc");
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (g_scratch_addr[dev] == nullptr) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr)
      return fail(MPK_CUDA_ERROR, std::string("cudaGetSymbolAddress of the inner-product scratch: ") +
                                      cudaGetErrorString(e));
    g_scratch_addr[dev] = p;
  }
  *out = (double*)g_scratch_addr[dev];
  return MPK_OK;
}

}  // namespace
}  // namespace mpk

using namespace mpk;

extern "C" int mpk_dot_noalloc(int n, int is_complex, int w, const double* a_dev, const double* b_dev,
                               double* out_dev, void* stream) {
  if (n < 1 || a_dev == nullptr || b_dev == nullptr || out_dev == nullptr) return fail(MPK_INVALID_ARG, "bad argument");
  if (w < 1 || w > 4 || (is_complex != 0 && is_complex != 1)) return fail(MPK_INVALID_ARG, "bad w / is_complex");
  if (misaligned(a_dev) || misaligned(b_dev) || misaligned(out_dev))
    return fail(MPK_INVALID_ARG, "device vectors must be 16-byte aligned");
  if (n > kNoAllocMaxN)
    return fail(MPK_INVALID_ARG, "mpk_dot_noalloc: n = " + std::to_string(n) + " exceeds the fixed scratch limit of " +
                                     std::to_string(kNoAllocMaxN) + " entries (use mpk_dot)");
  double* scratch = nullptr;
  int st = scratch_address(&scratch);
  if (st != MPK_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  DotWs ws;
  ws.partial = scratch;
  ws.counter = (unsigned*)(scratch + kNoAllocPartials);
  // the completion counter must start at zero; the array keeps whatever the last call left
  MPK_CUDA(cudaMemsetAsync(ws.counter, 0, sizeof(unsigned), s));
  const Ops* o = get_ops(w, is_complex ? 2 : 1);
  const double* av[1] = {a_dev};
  const double* bv[1] = {b_dev};
  double* ov[1] = {out_dev};
  o->dots(n, 1, av, bv, ov, ws, nullptr, s);
  MPK_CUDA(cudaGetLastError());
  return MPK_OK;
}
