// noalloc.cu -- a 2-D uint16 entry point that allocates no device memory.
//
// The plan API (swcorr_plan_create) allocates a small device status block
// with cudaMalloc.  Some callers cannot do that: code that runs under a
// device-memory budget owned entirely by its own pool allocator (a framework
// that has reserved the GPU's memory up front), and latency-critical loops
// that must not call cudaMalloc/cudaFree because those calls can synchronise
// the whole device.  swcorr_run2d_u16_noalloc serves them: it runs the same
// fused 2-D uint16 kernel as a 2-D uint16 plan, with the kernel's scratch (its
// status words: the error bits and the count of windows that took the exact
// per-window path) in a file-scope __device__ array instead of a cudaMalloc'd
// block.  The caller passes only its inputs and output.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>

#include "hostapi.h"
#include "launch.h"

using namespace swc;

// 64 uint32 words (256 bytes): every GPU that loads the library holds this
// array until the process exits.  The kernel uses ST_WORDS of it.
#define SWCORR_NOALLOC_SCRATCH_WORDS 64
static __device__ __align__(256) uint32_t g_noalloc_scratch[SWCORR_NOALLOC_SCRATCH_WORDS];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
uint32_t* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  In host code
// the array's name is only a host-side stand-in, so the address is taken
// once per device with that device current.  The cached address belongs to
// the device's primary context: after cudaDeviceReset() on a device this
// entry point must not be used on that device again in the same process.
swcorr_status scratch_address(int dev, uint32_t** out) {
  if (dev < 0 || dev >= kMaxDevices) return fail(SWCORR_ERR_UNSUPPORTED, "device ordinal %d too large", dev);
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-alloc scratch)");
    g_scratch_addr[dev] = static_cast<uint32_t*>(p);
  }
  *out = g_scratch_addr[dev];
  return SWCORR_OK;
}

}  // namespace

extern "C" swcorr_status swcorr_run2d_u16_noalloc(int64_t rows, int64_t cols, int32_t kh, int32_t kw,
                                                  const void* x, const void* y, int64_t in_pitch, float* c,
                                                  int64_t out_pitch, void* stream) {
  if (rows < 1 || cols < 1) return fail(SWCORR_ERR_INVALID_ARG, "rows and cols must be >= 1");
  if (rows > (1ll << 31) - 1024 || cols > (1ll << 31) - 1024)
    return fail(SWCORR_ERR_UNSUPPORTED, "rows/cols beyond the kernel's 32-bit index range");
  if (kh < 1 || kw < 1) return fail(SWCORR_ERR_INVALID_ARG, "window sizes must be >= 1");
  if (!x || !y || !c) return fail(SWCORR_ERR_INVALID_ARG, "x, y and c must not be NULL");
  const int64_t ip = in_pitch > 0 ? in_pitch : cols;
  const int64_t op = out_pitch > 0 ? out_pitch : cols;
  if (ip < cols || op < cols) return fail(SWCORR_ERR_INVALID_ARG, "pitches must be >= cols");
  if ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y)) & 1)
    return fail(SWCORR_ERR_ALIGNMENT, "x and y must be aligned to their element size");
  if (reinterpret_cast<uintptr_t>(c) & 3) return fail(SWCORR_ERR_ALIGNMENT, "c must be 4-byte aligned");
  if (ST_WORDS > SWCORR_NOALLOC_SCRATCH_WORDS)
    return fail(SWCORR_ERR_UNSUPPORTED, "kernel scratch of %d words exceeds the %d-word static array", (int)ST_WORDS,
                SWCORR_NOALLOC_SCRATCH_WORDS);
  DeviceInfo dev;
  swcorr_status st = device_info(&dev);
  if (st != SWCORR_OK) return st;
  uint32_t* scratch = nullptr;
  if ((st = scratch_address(dev.dev, &scratch)) != SWCORR_OK) return st;

  K2DParams k2{};
  Geo2DInfo g2{};
  size_t smem = 0;
  int grid = 0;
  st = setup_2d_u16(dev, (int)rows, (int)cols, kh, kw, 1, 1, &g2, &k2, &smem, &grid);
  if (st != SWCORR_OK) return st;
  bool use_tma = false;
  st = bind_2d_u16(&k2, g2, x, y, ip, c, op, nullptr, true, &use_tma);
  if (st != SWCORR_OK) return st;
  k2.status = scratch;

  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // the status words start at zero for every call (the array keeps the
  // previous call's contents)
  cudaError_t e = cudaMemsetAsync(scratch, 0, ST_WORDS * sizeof(uint32_t), s);
  if (e != cudaSuccess) return cuda_fail(e, "clear no-alloc scratch");
  e = k2d_u16_launch(kw, k2, grid, smem, s, use_tma);
  if (e != cudaSuccess) return cuda_fail(e, "2-D uint16 kernel launch");
  return SWCORR_OK;
}

// The kernel latches its errors (a bounded wait that gave up) and counts its
// exact per-window recomputations in the static array; nothing else can see
// them, so this call copies the words out (into a host array on the stack:
// no allocation), waits for the stream and clears them for the next call.
extern "C" swcorr_status swcorr_noalloc_status(void* stream, int64_t* fallbacks) {
  if (fallbacks) *fallbacks = -1;
  DeviceInfo dev;
  swcorr_status st = device_info(&dev);
  if (st != SWCORR_OK) return st;
  uint32_t* scratch = nullptr;
  if ((st = scratch_address(dev.dev, &scratch)) != SWCORR_OK) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  uint32_t h[ST_WORDS];
  cudaError_t e = cudaMemcpyAsync(h, scratch, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaMemsetAsync(scratch, 0, sizeof(h), s);
  if (e != cudaSuccess) return cuda_fail(e, "read no-alloc status words");
  if (fallbacks) *fallbacks = h[ST_FALLBACK];
  if (h[ST_ERROR] & ERRBIT_TIMEOUT) return fail(SWCORR_ERR_TIMEOUT, "a kernel's bounded wait gave up");
  if (h[ST_ERROR]) return fail(SWCORR_ERR_CUDA, "device status bits 0x%x", h[ST_ERROR]);
  return SWCORR_OK;
}
