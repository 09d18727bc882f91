// Chebyshev mass solve that needs no caller-provided scratch.
//
// Some callers cannot allocate device memory at the point where they need this
// solve: plug-ins hosted by a framework that owns all device memory and hands
// out only the buffers it chose, or real-time paths that forbid allocation after
// start-up.  This entry point takes only its input and output buffers; its two
// iterate buffers live in a fixed file-scope device array.
//
// The array is kNoAllocScratchBytes (16 MiB) on every GPU that loads the
// library and stays allocated until the process exits.  All calls share it:
// two calls whose kernels overlap on the GPU (different streams, or different
// host threads) race on it and give wrong results, so serialize them.  Every
// value a call reads from the array was written earlier in the same call, so no
// clearing is needed between calls.  The array's device address is looked up
// once per device (first call with that device current) and cached for the
// life of the process; a cudaDeviceReset invalidates the cached address.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "kernels.h"
#include "sgoc_internal.h"

namespace sgoc {

constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of g_noalloc_scratch for each device ordinal, looked up the
// first time the entry point runs with that device current.
constexpr int kMaxDevices = 64;
static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[kMaxDevices] = {nullptr};

static sgoc_status noalloc_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) { set_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e)); return SGOC_ERR_CUDA; }
  if (dev < 0 || dev >= kMaxDevices) { set_error("device ordinal out of range"); return SGOC_ERR_INVALID_ARG; }
  std::lock_guard<std::mutex> g(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      set_error(std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
      return SGOC_ERR_CUDA;
    }
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return SGOC_OK;
}

template <typename T>
static sgoc_status cheb_noalloc(sgoc_problem* pb, const void* d_R, void* d_X, int32_t ncols, cudaStream_t st) {
  const size_t per = size_t(ncols) * size_t(pb->n) * sizeof(T);
  if (per > kNoAllocScratchBytes / 2) {
    set_error("sgoc_apply_chebyshev_noalloc: ncols * n * sizeof(element) = " + std::to_string(per) +
              " bytes exceeds the limit of " + std::to_string(kNoAllocScratchBytes / 2) +
              " bytes (half of the 16 MiB built-in scratch)");
    return SGOC_ERR_INVALID_ARG;
  }
  // the problem's device data must live on the current device, whose scratch array is used
  int dev = 0;
  cudaError_t ge = cudaGetDevice(&dev);
  if (ge != cudaSuccess) { set_error(std::string("cudaGetDevice: ") + cudaGetErrorString(ge)); return SGOC_ERR_CUDA; }
  cudaPointerAttributes attr{};
  ge = cudaPointerGetAttributes(&attr, pb->dev.kap64);
  if (ge != cudaSuccess) { set_error(std::string("cudaPointerGetAttributes: ") + cudaGetErrorString(ge)); return SGOC_ERR_CUDA; }
  if (attr.type == cudaMemoryTypeDevice && attr.device != dev) {
    set_error("sgoc_apply_chebyshev_noalloc: the problem was uploaded to device " + std::to_string(attr.device) +
              " but device " + std::to_string(dev) + " is current");
    return SGOC_ERR_INVALID_ARG;
  }
  void* base = nullptr;
  SGOC_TRY(noalloc_scratch(&base));
  const size_t half = kNoAllocScratchBytes / 2;      // each iterate buffer starts 256-byte aligned
  ChebArgs<T> c{};
  c.B = static_cast<const T*>(d_R);
  c.X = static_cast<T*>(d_X);
  c.tmpA = reinterpret_cast<T*>(static_cast<unsigned char*>(base));
  c.tmpB = reinterpret_cast<T*>(static_cast<unsigned char*>(base) + half);
  c.ncols = ncols; c.n1 = pb->n1; c.n = pb->n; c.steps = pb->opt.cheb_steps;
  c.mass = T(pb->mass_h2_36);
  c.scale_mode = 0;
  cudaError_t e = launch_cheb<T>(c, st);
  if (e != cudaSuccess) { set_error(std::string("chebyshev launch: ") + cudaGetErrorString(e)); return SGOC_ERR_CUDA; }
  return SGOC_OK;
}

}  // namespace sgoc

using namespace sgoc;

extern "C" sgoc_status sgoc_apply_chebyshev_noalloc(sgoc_problem* pb, int32_t precision, const void* d_R,
                                                    void* d_X, int32_t ncols, void* stream) {
  if (!pb) { set_error("null problem"); return SGOC_ERR_INVALID_ARG; }
  if (!pb->uploaded) { set_error("call sgoc_problem_upload first"); return SGOC_ERR_NOT_UPLOADED; }
  if (!d_R || !d_X || ncols < 1) { set_error("bad arguments"); return SGOC_ERR_INVALID_ARG; }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  pdl_fence(st);                                   // the caller's prior work on st
  if (precision == 0) return cheb_noalloc<double>(pb, d_R, d_X, ncols, st);
  if (precision == 1) return cheb_noalloc<float>(pb, d_R, d_X, ncols, st);
  set_error("precision must be 0 or 1");
  return SGOC_ERR_INVALID_ARG;
}
