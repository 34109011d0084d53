// igm_noalloc.cu -- igm_norm2_noalloc: the reproducible 2-norm of igm_norm2
// for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc: code running inside a CUDA graph that
// is being captured (allocation is not capturable), a process whose device
// memory is entirely managed by another allocator or pool that forbids
// side allocations, or a hard real-time loop where an allocation's
// synchronisation and latency are not acceptable.  igm_norm2 takes its
// scratch from a workspace it allocates on first use; this variant keeps the
// same kernels' scratch (per-CTA partial sums and the last-CTA counters) in
// one file-scope static device array instead, so it never allocates.
//
// The array exists once per device that loads the library and stays
// allocated until the process exits.  Every call shares it and it keeps the
// last call's contents, so calls whose GPU work overlaps (different streams,
// or different host threads, on the same device) race; calls on one stream
// are ordered and safe.  The counters that must start at zero are cleared at
// the start of every call.
#include <cuda_runtime.h>

#include <mutex>

#include "igm_host.h"

namespace {

// CTAs (and hence partial-sum slots) one call may use; each CTA covers
// kPerCta elements, so n is limited to their product
constexpr int kMaxCtas = 2048;
constexpr int kPerCta = 4096;
constexpr long long kMaxN = (long long)kMaxCtas * kPerCta;  // 8,388,608

// [0, 2*kMaxCtas): int128 / double partials of the CTAs; [2*kMaxCtas, +2):
// the two last-CTA counters' words; then one double for max |x_i|
constexpr int kWords = 2 * kMaxCtas + 2 + 2;
static __device__ __align__(256) long long g_noalloc_scratch[kWords];

std::mutex g_mu;
long long *g_addr[64] = {nullptr};  // device address of the array, per device

}  // namespace

extern "C" igm_status igm_norm2_noalloc(const double *x, int n, double *out, void *stream) {
  g_err.clear();
  if (!out || n < 0 || (n > 0 && !x)) return fail(IGM_EINVAL, "bad arguments");
  if (n > kMaxN)
    return fail(IGM_EINVAL, "n = %d exceeds the static scratch of this entry point (max %lld)",
                n, kMaxN);
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(IGM_EINVAL, "device index %d out of range", dev);
  // x and out must already be device memory: this entry point stages nothing
  cudaPointerAttributes pa;
  for (const void *p : {(const void *)x, (const void *)out}) {
    if (p == x && n == 0) continue;
    if (cudaPointerGetAttributes(&pa, p) != cudaSuccess) {
      cudaGetLastError();
      return fail(IGM_EINVAL, "x and out must be device (or managed) memory");
    }
    if (pa.type != cudaMemoryTypeDevice && pa.type != cudaMemoryTypeManaged)
      return fail(IGM_EINVAL, "x and out must be device (or managed) memory");
    // memory of another GPU would be dereferenced from this one: refused
    if (pa.type == cudaMemoryTypeDevice && pa.device != dev)
      return fail(IGM_EINVAL, "x and out must be on the current device (%d), not device %d",
                  dev, pa.device);
  }
  // once per device, with that device current: the array's device address
  // (in host code the symbol is only a host-side stand-in)
  long long *ws;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
      void *p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(IGM_ECUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
      }
      g_addr[dev] = static_cast<long long *>(p);
    }
    ws = g_addr[dev];
  }
  cudaStream_t s = (cudaStream_t)stream;
  int g = (int)((n + kPerCta - 1) / kPerCta);
  if (g < 1) g = 1;
  // the counters of this grid start at zero
  CK(cudaMemsetAsync(ws + 2 * g, 0, 2 * sizeof(long long), s));
  double *mx = reinterpret_cast<double *>(ws + 2 * kMaxCtas + 2);
  igm::launch_norm2_grid(x, n, g, ws, mx, out, s);
  CKL();
  g_launches += 2;
  return IGM_OK;
}
