// Allocation-free variant of ff_consistency_filter.
//
// Some callers cannot hand the library a workspace: code that runs inside a
// framework which owns the whole device memory pool and gives plugins no
// allocator, or a real-time frame loop that reserves all memory at start-up and
// must not call cudaMalloc later (it can synchronise the device and stall the
// pipeline). For them this entry point takes its scratch from one file-scope
// device array of fixed size instead of a caller workspace.
//
// The array lives in every GPU that loads the library until the process exits.
// In host code its name is only a stand-in for the device symbol, so the kernels
// get the device address obtained with cudaGetSymbolAddress, once per device.
#include <mutex>

#include "ff_internal.cuh"

namespace ff {

// Largest image handled: 1,048,576 pixels (e.g. 1024 x 1024, 1280 x 720).
constexpr long long STATIC_MAX_PIXELS = 1ll << 20;
// filter_scratch_bytes() is at most 10 B per pixel plus 4 B per 3x3 block and 4 B
// per 256 blocks, plus block alignment: under 12 MiB for 2^20 pixels.
constexpr size_t STATIC_SCRATCH_BYTES = 12u << 20;

static __device__ __align__(256) unsigned char g_filter_scratch[STATIC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
static void *g_scratch_ptr[MAX_DEVICES];
static std::mutex g_scratch_mu;

// Device address of g_filter_scratch on the current device (set-up on first use).
static ff_status static_scratch(void **out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return FF_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_filter_scratch) != cudaSuccess || !p) {
      (void)cudaGetLastError();
      return FF_ERR_CUDA;
    }
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return FF_OK;
}

}  // namespace ff

using namespace ff;

extern "C" ff_status ff_consistency_filter_static(const int16_t *F, const int16_t *Fb1,
                                                  const int16_t *Fb2, int W, int H,
                                                  const ff_params *p, uint8_t *valid,
                                                  int32_t *err_sum, int32_t *sparse,
                                                  int32_t *n_sparse, uint8_t *mask,
                                                  void *stream) {
  // the checks of ff_consistency_filter first, then this entry point's own limits
  FF_TRY(check_shape(W, H));
  FF_TRY(check_params(p));
  if ((long long)W * H > STATIC_MAX_PIXELS) return FF_ERR_SHAPE;
  if (filter_scratch_bytes(W, H) > STATIC_SCRATCH_BYTES) return FF_ERR_SHAPE;
  if (!F || !Fb1 || !Fb2 || !valid || !err_sum || !sparse || !n_sparse || !mask)
    return FF_ERR_INVALID_ARG;
  if (((uintptr_t)F | (uintptr_t)Fb1 | (uintptr_t)Fb2) & 3) return FF_ERR_INVALID_ARG;
  void *scratch = nullptr;
  FF_TRY(static_scratch(&scratch));
  // launch_filter clears the per-region flags it needs zeroed on the stream and
  // writes every other scratch word before reading it.
  return launch_filter((const uint32_t *)F, (const uint32_t *)Fb1, (const uint32_t *)Fb2, W, H,
                       p->eps, p->e, p->s, p->subpel, valid, err_sum, sparse, n_sparse, mask, scratch,
                       (cudaStream_t)stream);
}
