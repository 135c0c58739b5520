// Measurement probes: small kernels whose rates are the roofline denominators of
// the search kernels (not part of the method).
//
// The search evaluates census taps: one xor, one popcount and one add per tap,
// the source word from shared memory and the target word from shared memory (the
// staged window) or through L1/L2 (the census phase planes). So the ceilings that
// bound it are the popcount issue rate, the shared-memory load rate with two words
// per tap, and the L2 read rate for gathered words. Each probe measures one of
// them with enough independent work in flight that latency does not bind; the
// caller times the launch with CUDA events and owns every buffer.
#include "ff_internal.cuh"

namespace ff {

constexpr int PROBE_THREADS = 256;

// Eight independent xor / popcount / add chains per thread on register operands.
// The operands change every round (xor with the round counter), so nothing is
// loop-invariant; the sums are stored so that the work is live.
__global__ void __launch_bounds__(PROBE_THREADS) k_probe_popc(uint32_t *sink, int iters) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t a[8];
  int acc[8];
#pragma unroll
  for (int k = 0; k < 8; k++) {
    a[k] = (t + 1u) * 0x9e3779b1u + (uint32_t)k * 0x85ebca6bu;
    acc[k] = 0;
  }
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int k = 0; k < 8; k++) acc[k] += __popc(a[k] ^ (uint32_t)it);
#pragma unroll
    for (int k = 0; k < 8; k++) acc[k] += __popc(a[k] ^ ~(uint32_t)it);
  }
  int s = 0;
#pragma unroll
  for (int k = 0; k < 8; k++) s += acc[k];
  sink[t] = (uint32_t)s;
}

// Census taps with both words from shared memory: per round every thread
// evaluates 16 taps, lane-consecutive words (no bank conflicts), four
// accumulators; the window moves over four quarters of the buffer. The loads are
// volatile, so that each round issues them again (the buffer does not change,
// and plain loads would be hoisted out of the loop).
constexpr int PROBE_SMEM_WORDS = 2048;
__global__ void __launch_bounds__(PROBE_THREADS) k_probe_smem_taps(uint32_t *sink, int iters) {
  __shared__ uint32_t sa[PROBE_SMEM_WORDS], sb[PROBE_SMEM_WORDS];
  for (int i = threadIdx.x; i < PROBE_SMEM_WORDS; i += blockDim.x) {
    sa[i] = (uint32_t)i * 0x9e3779b1u + blockIdx.x;
    sb[i] = (uint32_t)i * 0x85ebca6bu ^ blockIdx.x;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int a0 = 0, a1 = 0, a2 = 0, a3 = 0;
  for (int it = 0; it < iters; it++) {
    const int off = ((it + warp) & 3) * 512 + lane;
    const volatile uint32_t *pa = sa + off, *pb = sb + off;
#pragma unroll
    for (int k = 0; k < 16; k += 4) {
      a0 += __popc(pa[32 * k] ^ pb[32 * k]);
      a1 += __popc(pa[32 * k + 32] ^ pb[32 * k + 32]);
      a2 += __popc(pa[32 * k + 64] ^ pb[32 * k + 64]);
      a3 += __popc(pa[32 * k + 96] ^ pb[32 * k + 96]);
    }
  }
  sink[blockIdx.x * blockDim.x + threadIdx.x] = (uint32_t)((a0 + a1) + (a2 + a3));
}

// L2 reads from an L2-resident buffer of `words` (a power of two) 32-bit words,
// through ld.global.cg (cached in L2, not L1). Every thread keeps 8 loads in
// flight per round; addresses come from a per-thread linear congruential stream.
//   mode 0: one random 4-byte word per lane
//   mode 1: one random 16-byte line per lane
//   mode 2: 512 contiguous bytes per warp (16 bytes per lane) at a random
//           512-byte aligned position
__global__ void __launch_bounds__(PROBE_THREADS) k_probe_l2(const uint32_t *buf, uint32_t mask,
                                                           int mode, uint32_t *sink, int iters) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  uint32_t x = (t + 1u) * 0x9e3779b1u;
  uint32_t acc = 0;
  if (mode == 0) {
    for (int it = 0; it < iters; it++) {
      uint32_t v[8];
#pragma unroll
      for (int k = 0; k < 8; k++) {
        x = x * 1664525u + 1013904223u;
        v[k] = __ldcg(buf + ((x >> 7) & mask));
      }
#pragma unroll
      for (int k = 0; k < 8; k++) acc ^= v[k];
    }
  } else {
    const uint4 *b4 = (const uint4 *)buf;
    const uint32_t mask4 = mask >> 2;
    uint32_t xw = __shfl_sync(0xffffffffu, x, 0);  // mode 2: one stream per warp
    for (int it = 0; it < iters; it++) {
      uint4 v[8];
#pragma unroll
      for (int k = 0; k < 8; k++) {
        uint32_t i4;
        if (mode == 1) {
          x = x * 1664525u + 1013904223u;
          i4 = (x >> 7) & mask4;
        } else {
          xw = xw * 1664525u + 1013904223u;
          i4 = (((xw >> 7) << 5) + lane) & mask4;
        }
        v[k] = __ldcg(b4 + i4);
      }
#pragma unroll
      for (int k = 0; k < 8; k++) acc ^= v[k].x ^ v[k].y ^ v[k].z ^ v[k].w;
    }
  }
  sink[t] = acc;
}

}  // namespace ff

using namespace ff;

extern "C" {

ff_status ff_probe_popc(uint32_t *sink, int blocks, int iters, void *stream) {
  if (!sink || blocks < 1 || iters < 1) return FF_ERR_INVALID_ARG;
  k_probe_popc<<<blocks, PROBE_THREADS, 0, (cudaStream_t)stream>>>(sink, iters);
  FF_CHECK_LAUNCH();
  return FF_OK;
}

ff_status ff_probe_smem_taps(uint32_t *sink, int blocks, int iters, void *stream) {
  if (!sink || blocks < 1 || iters < 1) return FF_ERR_INVALID_ARG;
  k_probe_smem_taps<<<blocks, PROBE_THREADS, 0, (cudaStream_t)stream>>>(sink, iters);
  FF_CHECK_LAUNCH();
  return FF_OK;
}

ff_status ff_probe_l2_gather(const uint32_t *buf, size_t words, int mode, uint32_t *sink,
                             int blocks, int iters, uint64_t *bytes, void *stream) {
  if (!buf || !sink || blocks < 1 || iters < 1 || mode < 0 || mode > 2) return FF_ERR_INVALID_ARG;
  if (words < 1024 || words > (1ull << 31) || (words & (words - 1)) || ((uintptr_t)buf & 15))
    return FF_ERR_INVALID_ARG;
  k_probe_l2<<<blocks, PROBE_THREADS, 0, (cudaStream_t)stream>>>(buf, (uint32_t)(words - 1), mode,
                                                                sink, iters);
  FF_CHECK_LAUNCH();
  if (bytes) *bytes = (uint64_t)blocks * PROBE_THREADS * iters * 8 * (mode == 0 ? 4 : 16);
  return FF_OK;
}

}  // extern "C"
