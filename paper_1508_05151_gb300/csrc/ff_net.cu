// Learned proposal net (not in the paper): a small convolutional net that reads
// the coarsest pyramid level of both frames and emits K flow candidates per grid
// point of the coarsest search level; they are tried beside the kd-tree
// candidates (Eq. 1/4 rerank), so they can only ever replace the kd result when
// the exact integer data term prefers them.
//
// Layers l = 0..3: 3x3 convolution, dilation dil[l], zero padding dil[l], bias,
// ReLU except after the last layer. Channels cin(=6) -> c1 -> c2 -> c3 -> 2K.
// The public input and output are NCHW FP32. Inside the workspace activations and
// gradients are channels-last (pixel-major, channels padded to a multiple of 8
// with zeros), so the 8 channels of one pixel are 16 contiguous bytes; every
// convolution input is BF16 and accumulates in FP32. The reduction index of the
// convolutions is tap-major, k = tap * Cpad + c.
// Parameters (FP32 master copy) per layer: W [cout][cin][3][3], then b [cout].
//
// All three convolution products are implicit GEMMs on the 5th-generation
// tensor cores (tcgen05.mma kind::f16, BF16 x BF16 -> FP32 accumulator in tensor
// memory):
//   forward   out[m][n]  = sum_k A[m][k] B[k][n],  m = pixel, n = cout, k = (cin, tap)
//   dgrad     din[m][n]  = sum_k G[m][k] Bd[k][n], m = pixel, n = cin,  k = (cout, tap), taps mirrored
//   wgrad     dW[n][k]   = sum_m G[m][n] A[m][k]   (reduction over pixels, split across CTAs)
// where A is the im2col view of the layer input and G the gradient at the
// pre-activation. A CTA of 128 threads computes a 128 x 64 tile: both operands
// are staged in shared memory (the convolutions: 16-byte cp.async copies into a
// four-stage pipeline, 16 deep per stage; the weight gradient: 32 pixels, two
// MMAs, per stage), one thread issues the MMAs, an mbarrier reports their
// completion, and the epilogue reads the accumulator back with tcgen05.ld. Waits
// are bounded; a wait that runs out sets the device status word at the start of
// the workspace.
#include <cuda_bf16.h>

#include "ff_internal.cuh"

namespace ff {

constexpr int NET_LAYERS = 4;

struct NetShape {
  int cin[NET_LAYERS], cout[NET_LAYERS], dil[NET_LAYERS];
  size_t woff[NET_LAYERS], boff[NET_LAYERS];  // offsets into the parameter vector
  size_t nparams;
};

static bool net_shape(const ff_net_desc *d, NetShape &s) {
  if (!d || d->cin != 6 || d->k < 1 || d->k > MAX_K) return false;
  const int ch[5] = {d->cin, d->c1, d->c2, d->c3, 2 * d->k};
  size_t off = 0;
  for (int l = 0; l < NET_LAYERS; l++) {
    if (ch[l + 1] < 1 || ch[l + 1] > 64 || d->dil[l] < 1 || d->dil[l] > 16) return false;
    s.cin[l] = ch[l];
    s.cout[l] = ch[l + 1];
    s.dil[l] = d->dil[l];
    s.woff[l] = off;
    off += (size_t)ch[l + 1] * ch[l] * 9;
    s.boff[l] = off;
    off += ch[l + 1];
  }
  s.nparams = off;
  return true;
}

static int pad64(int v) { return (v + 63) & ~63; }
static int padk(int v);  // K padded to whole stages of the convolution kernel
__host__ __device__ __forceinline__ int cpad8(int c) { return (c + 7) & ~7; }

// ------------------------------------------------------- forward / dgrad -----
// out[m][n] = bias[n] + sum_{tap, c} Bt[n][tap * Ca + c] * act[pixel m + s * off(tap)][c]
// with off(tap) = ((tap/3)-1, (tap%3)-1) * dil and s = +1 (forward) or -1 (dgrad),
// m = (b, y, x). Writes the pre-activation (FP32, channels-last, or NCHW for the
// net's output) and a BF16 channels-last copy: relu(out) in the forward pass, or
// out times the ReLU mask of the lower layer's pre-activation in dgrad.
struct ConvArgs {
  const __nv_bfloat16 *act;  // [B][H][W][Ca] channels-last, Ca = cpad8(C)
  int B, Ca, H, W, dil, sign;
  const __nv_bfloat16 *Bt;   // [Np][Kp] K-major (zero rows and columns up to Np, Kp)
  int K, Kp, N, Np;          // K = 9 * Ca
  const float *bias;         // [N] or null
  float *out;                // [B][H][W][cpad8(N)] fp32, or [B][N][H][W] with out_nchw, or null
  int out_nchw;
  __nv_bfloat16 *out_bf;     // [B][H][W][cpad8(N)] bf16 or null
  const float *mask_pre;     // dgrad: [B][H][W][cpad8(N)] lower pre-activation; grad *= (pre > 0)
  int relu;
  int stall;                 // test hook: > 0 polls of a wait that nothing completes
};

// ------------------------------------------------ forward / dgrad, tcgen05 --
// One CTA (128 threads) computes a 128-pixel x 64-column tile. A stage holds
// CONV_KSTEP of K (CONV_SUB MMAs of 16): thread t copies the 16-byte groups (8
// channels of one tap each) of A row t (pixel m0 + t) and CONV_SUB 16-byte pieces
// of the B^T tile straight into shared memory with cp.async, in the no-swizzle
// K-major core-matrix layout (per 16-deep slice: 8 rows x 16 bytes per core
// matrix, the two core matrices of a row group 128 B apart along K, row groups
// 256 B apart). Taps outside the image are zero-filled by the copy. Six stages
// of 16, filled four ahead: while one thread issues the tcgen05.mma of a stage
// (BF16 x BF16 -> FP32, the accumulator in tensor memory) the next four stages'
// copies are in flight; tcgen05.commit signals a stage's mbarrier when its MMA is
// done, and the stage is refilled, so a refill waits on the MMA of two steps
// before. (Forward pass of 64 pairs: 0.248 ms, against 0.260 with four stages
// filled three ahead, 0.295 with eight filled four ahead, and 0.278 with stages
// of 64 filled two ahead, 96 KB per CTA.) The epilogue reads the accumulator with tcgen05.ld (warp w owns TMEM
// lanes = tile rows 32w..32w+31) and writes 8 channels of a pixel as one vector
// store.
constexpr int UMMA_M = 128, UMMA_N = 64, UMMA_K = 16;
constexpr int UMMA_A_BYTES = UMMA_M * UMMA_K * 2, UMMA_B_BYTES = UMMA_N * UMMA_K * 2;
constexpr int CONV_STAGES = 6, CONV_AHEAD = 4, CONV_SUB = 1;  // stages, fill distance, MMAs per stage
constexpr int CONV_KSTEP = UMMA_K * CONV_SUB;
constexpr int CONV_A_STAGE = UMMA_A_BYTES * CONV_SUB, CONV_B_STAGE = UMMA_B_BYTES * CONV_SUB;
constexpr size_t CONV_SMEM = (size_t)CONV_STAGES * (CONV_A_STAGE + CONV_B_STAGE);
static int padk(int v) { return (v + CONV_KSTEP - 1) / CONV_KSTEP * CONV_KSTEP; }
constexpr unsigned UMMA_WAIT_LIMIT = 1u << 22;  // bounded mbarrier waits (polls)

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: start address, leading (K-direction) and
// stride (row-group) byte offsets, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__device__ __forceinline__ uint32_t umma_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// byte offset of element (row, k) of a K-major tile with 16-element rows
__device__ __forceinline__ int umma_off(int row, int k) {
  return (row >> 3) * 256 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity,
                                          unsigned limit = UMMA_WAIT_LIMIT) {
  for (unsigned it = 0; it < limit; it++) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// 16-byte global -> shared copy; `bytes` = 0 fills the destination with zeros
// (src is then not read).
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__global__ void __launch_bounds__(128) k_conv_umma(ConvArgs a, DeviceStatus *status) {
  extern __shared__ __align__(1024) uint8_t conv_smem[];  // stages: A tiles, then B tiles
  __shared__ __align__(8) uint64_t mbar[CONV_STAGES];
  __shared__ uint32_t tmem_holder;
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int HW = a.H * a.W, M = a.B * HW;
  const int m0 = blockIdx.x * UMMA_M, n0 = blockIdx.y * UMMA_N;

  if (warp == 0) {  // 64 TMEM columns hold the 128 x 64 FP32 accumulator
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(&tmem_holder)),
                 "r"(UMMA_N)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    s_fail = 0;
    for (int i = 0; i < CONV_STAGES; i++)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar[i])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_holder;

  // this thread's A row (pixel m0 + tid) and B^T row tid % 64 (its pieces:
  // (tid / 64) + 2 i, i < CONV_SUB, numbering the stage's 16-k slice halves)
  const int ms = m0 + tid;
  int pb = -1, py = 0, px = 0;
  if (ms < M) {
    pb = ms / HW;
    const int p = ms - pb * HW;
    py = p / a.W;
    px = p - py * a.W;
  }
  const int bn = tid & 63, bq = tid >> 6;
  const __nv_bfloat16 *brow = a.Bt + (size_t)(n0 + bn) * a.Kp;
  const uint32_t sA0 = smem_u32(conv_smem), sB0 = sA0 + CONV_STAGES * CONV_A_STAGE;
  // (tap, channel) of the first 8-channel group of the next stage to issue; stages
  // are issued in order, so it advances by CONV_KSTEP channels per stage (Ca, the
  // padded channel count, is a multiple of 8)
  int nx_tap = 0, nx_c0 = 0;
  auto issue = [&](int s) {  // the copies of stage s (K from s * CONV_KSTEP) into buffer s % CONV_STAGES
    const int buf = s % CONV_STAGES, k0 = s * CONV_KSTEP;
    const uint32_t aS = sA0 + buf * CONV_A_STAGE, bS = sB0 + buf * CONV_B_STAGE;
    int tap = nx_tap, c0 = nx_c0;
#pragma unroll
    for (int g = 0; g < CONV_KSTEP / 8; g++) {
      const int kk = k0 + 8 * g;
      const __nv_bfloat16 *src = a.act;
      int bytes = 0;
      if (pb >= 0 && kk < a.K) {
        const int yy = py + a.sign * ((tap / 3) - 1) * a.dil;
        const int xx = px + a.sign * ((tap % 3) - 1) * a.dil;
        if (yy >= 0 && yy < a.H && xx >= 0 && xx < a.W) {
          src = a.act + (((size_t)pb * a.H + yy) * a.W + xx) * a.Ca + c0;
          bytes = 16;
        }
      }
      cp_async16(aS + (g >> 1) * UMMA_A_BYTES + umma_off(tid, 8 * (g & 1)), src, bytes);
      c0 += 8;
      if (c0 >= a.Ca) {
        c0 -= a.Ca;
        tap++;
      }
    }
    nx_tap = tap;
    nx_c0 = c0;
#pragma unroll
    for (int i = 0; i < CONV_SUB; i++) {  // piece (row bn, 16-k slice, half) of the B^T stage
      const int rest = bq + 2 * i, sub = rest >> 1, e = rest & 1;
      cp_async16(bS + sub * UMMA_B_BYTES + umma_off(bn, 8 * e), brow + k0 + UMMA_K * sub + 8 * e, 16);
    }
  };
  const uint32_t idesc = umma_idesc(UMMA_M, UMMA_N);
  int nsteps = a.Kp / CONV_KSTEP;
  if (a.stall > 0) {  // test hook: stage 0's barrier before any MMA (nothing completes it)
    if (!mbar_wait(smem_u32(&mbar[0]), 0u, (unsigned)a.stall)) s_fail = 1;
    __syncthreads();
    if (s_fail) nsteps = 0;  // no MMA in flight: the accumulator is freed below
  }
  uint32_t phase = 0u;  // bit i: parity of stage i's next mbarrier phase
#pragma unroll
  for (int s = 0; s < CONV_AHEAD; s++) {
    if (s < nsteps) issue(s);
    cp_async_commit();
  }
  // One CTA barrier per step. Before it, every thread's copies of stage `step` have
  // landed, and thread 0 (alone: it tracks the mbarrier phases) has seen the MMA that
  // last read the buffer of stage step + CONV_AHEAD complete; after it, thread 0
  // issues stage `step`'s MMA and every thread the copies of stage step + CONV_AHEAD.
  for (int step = 0; step < nsteps; step++) {
    const int ns = step + CONV_AHEAD;
    cp_async_wait<CONV_AHEAD - 1>();  // this thread's copies of stage `step` landed
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    if (tid == 0 && ns < nsteps && ns >= CONV_STAGES) {  // the MMA of step ns - CONV_STAGES
      const int nb = ns % CONV_STAGES;
      if (!mbar_wait(smem_u32(&mbar[nb]), (phase >> nb) & 1u)) s_fail = 1;
      phase ^= 1u << nb;
    }
    __syncthreads();
    if (tid == 0) {
      const int buf = step % CONV_STAGES;
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll
      for (int sub = 0; sub < CONV_SUB; sub++) {
        const uint64_t adesc = umma_desc(sA0 + buf * CONV_A_STAGE + sub * UMMA_A_BYTES, 128, 256);
        const uint64_t bdesc = umma_desc(sB0 + buf * CONV_B_STAGE + sub * UMMA_B_BYTES, 128, 256);
        const uint32_t acc = (step > 0 || sub > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                       smem_u32(&mbar[buf]))
                   : "memory");
    }
    if (ns < nsteps) issue(ns);
    cp_async_commit();
  }
  cp_async_wait<0>();
  // the last MMAs (commits complete in order, so every earlier MMA is done too)
  if (tid == 0 && nsteps > 0) {
    const int lb = (nsteps - 1) % CONV_STAGES;
    if (!mbar_wait(smem_u32(&mbar[lb]), (phase >> lb) & 1u)) s_fail = 1;
  }
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  __syncthreads();
  const bool ok = s_fail == 0;
  if (!ok && tid == 0) raise_status(status, DEV_ERR_TIMEOUT, blockIdx.x, blockIdx.y);

  // epilogue: row m0 + 32 warp + lane, eight columns per tcgen05.ld
  const int m = m0 + warp * 32 + lane;
  const int b = m / HW, p = m - b * HW, Cs = cpad8(a.N);
#pragma unroll 1
  for (int c0 = 0; c0 < UMMA_N; c0 += 8) {
    uint32_t r[8];
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
    const int nb = n0 + c0;
    if (!ok || m >= M || nb >= Cs) continue;
    float v[8];
#pragma unroll
    for (int j = 0; j < 8; j++) {
      const int n = nb + j;
      v[j] = n < a.N ? __uint_as_float(r[j]) + (a.bias ? a.bias[n] : 0.f) : 0.f;
    }
    if (a.out_nchw) {
#pragma unroll
      for (int j = 0; j < 8; j++)
        if (nb + j < a.N) a.out[((size_t)b * a.N + nb + j) * HW + p] = v[j];
      continue;
    }
    const size_t o = (size_t)m * Cs + nb;  // 8 channels of pixel m: 32 / 16 aligned bytes
    if (a.mask_pre) {
      const float4 q0 = *(const float4 *)(a.mask_pre + o), q1 = *(const float4 *)(a.mask_pre + o + 4);
      const float q[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
#pragma unroll
      for (int j = 0; j < 8; j++)
        if (!(q[j] > 0.f)) v[j] = 0.f;
    }
    if (a.out) {
      *(float4 *)(a.out + o) = make_float4(v[0], v[1], v[2], v[3]);
      *(float4 *)(a.out + o + 4) = make_float4(v[4], v[5], v[6], v[7]);
    }
    if (a.out_bf) {
      uint32_t w[4];
#pragma unroll
      for (int j = 0; j < 4; j++) {
        const float lo = a.relu ? fmaxf(v[2 * j], 0.f) : v[2 * j];
        const float hi = a.relu ? fmaxf(v[2 * j + 1], 0.f) : v[2 * j + 1];
        w[j] = (uint32_t)__bfloat16_as_ushort(__float2bfloat16(lo)) |
               ((uint32_t)__bfloat16_as_ushort(__float2bfloat16(hi)) << 16);
      }
      *(uint4 *)(a.out_bf + o) = make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(UMMA_N)
                 : "memory");
}

// ------------------------------------------------------------------ wgrad ---
struct WgradArgs {
  const __nv_bfloat16 *g;    // [B][H][W][Cg] gradient at the pre-activation (channels-last)
  const __nv_bfloat16 *act;  // [B][H][W][Ca] layer input (channels-last)
  int B, C, Ca, H, W, dil, N, Cg, K;  // K = 9 * Ca rows, k = tap * Ca + c
  float *dW;                 // [N][C][3][3]
  float *db;                 // [N]
  int pix_per_cta;
  int stall;                 // test hook: > 0 polls of a wait that nothing completes
};

// Weight gradient on tcgen05: the transposed product D[k][n] = sum_m A[m][k] G[m][n]
// (k = (tap, c) rows, 128 per CTA; n = cout columns, 64; the reduction runs over
// the CTA's pixel range, WG_PIX pixels per stage = two MMAs of 16). A^T tile row k =
// the layer input at tap(k) of channel c(k) for the stage's pixels; G^T tile row n =
// the gradient of channel n for the same pixels. Lane = pixel when staging: a
// thread loads the 8 channels (16 bytes) of a row group of its pixel and stores
// them down the tile's column. Each 16-pixel half of a tile is K-major in the same
// core-matrix layout as the convolution kernel; the FP32 result is added into dW
// with atomics (the summation order over CTAs is unspecified).
constexpr int WG_PIX = 32;
constexpr int WG_A_HALF = UMMA_M * 16 * 2, WG_B_HALF = UMMA_N * 16 * 2;
__global__ void __launch_bounds__(128, 6) k_wgrad_umma(WgradArgs a, DeviceStatus *status) {
  __shared__ __align__(1024) uint8_t sA[2][2 * WG_A_HALF];
  __shared__ __align__(1024) uint8_t sB[2][2 * WG_B_HALF];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_holder;
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int HW = a.H * a.W, M = a.B * HW;
  const int kt0 = blockIdx.y * UMMA_M;
  const int p0 = blockIdx.x * a.pix_per_cta, p1 = min(p0 + a.pix_per_cta, M);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(&tmem_holder)),
                 "r"(UMMA_N)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    s_fail = 0;
    for (int i = 0; i < 2; i++)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar[i])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  // this thread's A^T row groups rg = warp + 4 q (q = 0..3): tap, first channel,
  // displacement (tap < 0: past K)
  int rtap[4], rc0[4], rdy[4], rdx[4];
#pragma unroll
  for (int q = 0; q < 4; q++) {
    const int k = kt0 + 8 * (warp + 4 * q);
    rtap[q] = k < a.K ? k / a.Ca : -1;
    rc0[q] = k < a.K ? k - rtap[q] * a.Ca : 0;
    rdy[q] = rtap[q] >= 0 ? ((rtap[q] / 3) - 1) * a.dil : 0;
    rdx[q] = rtap[q] >= 0 ? ((rtap[q] % 3) - 1) * a.dil : 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_holder;

  // staging: lane = pixel of the stage; byte offset of the lane's 16-pixel half
  const int a_lane = (lane >> 4) * WG_A_HALF, b_lane = (lane >> 4) * WG_B_HALF, col = lane & 15;
  const uint32_t idesc = umma_idesc(UMMA_M, UMMA_N);
  int nsteps = (p1 - p0 + WG_PIX - 1) / WG_PIX;
  if (a.stall > 0) {  // test hook: stage 0's barrier before any MMA (nothing completes it)
    if (!mbar_wait(smem_u32(&mbar[0]), 0u, (unsigned)a.stall)) s_fail = 1;
    __syncthreads();
    if (s_fail) nsteps = 0;  // no MMA in flight: the accumulator is freed below
  }
  float bsum[2][8];  // this lane's share of the bias gradient of G^T rows 8 (warp + 4 q) + i
#pragma unroll
  for (int q = 0; q < 2; q++)
#pragma unroll
    for (int i = 0; i < 8; i++) bsum[q][i] = 0.f;
  uint32_t phase[2] = {0u, 0u};
  for (int step = 0; step < nsteps; step++) {
    const int st = step & 1;
    if (step >= 2) {
      if (!mbar_wait(smem_u32(&mbar[st]), phase[st])) s_fail = 1;
      phase[st] ^= 1u;
    }
    const int m = p0 + step * WG_PIX + lane;
    const bool pin = m < p1;
    const int b = pin ? m / HW : 0, pp = m - b * HW, y = pp / a.W, x = pp - y * a.W;
    uint4 va[4], vg[2];
#pragma unroll
    for (int q = 0; q < 4; q++) {
      va[q] = make_uint4(0, 0, 0, 0);
      const int yy = y + rdy[q], xx = x + rdx[q];
      if (pin && rtap[q] >= 0 && (unsigned)yy < (unsigned)a.H && (unsigned)xx < (unsigned)a.W)
        va[q] = *(const uint4 *)(a.act + (((size_t)b * a.H + yy) * a.W + xx) * a.Ca + rc0[q]);
    }
#pragma unroll
    for (int q = 0; q < 2; q++) {
      const int n8 = 8 * (warp + 4 * q);
      vg[q] = (pin && n8 < a.Cg) ? *(const uint4 *)(a.g + (size_t)m * a.Cg + n8) : make_uint4(0, 0, 0, 0);
    }
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const uint32_t w[4] = {va[q].x, va[q].y, va[q].z, va[q].w};
      const int r0 = 8 * (warp + 4 * q);
#pragma unroll
      for (int i = 0; i < 8; i++)
        *(unsigned short *)(sA[st] + a_lane + umma_off(r0 + i, col)) =
            (unsigned short)(w[i >> 1] >> (16 * (i & 1)));
    }
#pragma unroll
    for (int q = 0; q < 2; q++) {
      const uint32_t w[4] = {vg[q].x, vg[q].y, vg[q].z, vg[q].w};
      const int r0 = 8 * (warp + 4 * q);
#pragma unroll
      for (int i = 0; i < 8; i++) {
        const unsigned short h = (unsigned short)(w[i >> 1] >> (16 * (i & 1)));
        *(unsigned short *)(sB[st] + b_lane + umma_off(r0 + i, col)) = h;
        bsum[q][i] += __bfloat162float(__ushort_as_bfloat16(h));
      }
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll
      for (int h = 0; h < 2; h++) {
        const uint64_t adesc = umma_desc(smem_u32(sA[st] + h * WG_A_HALF), 128, 256);
        const uint64_t bdesc = umma_desc(smem_u32(sB[st] + h * WG_B_HALF), 128, 256);
        const uint32_t acc = (step > 0 || h > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                       smem_u32(&mbar[st]))
                   : "memory");
    }
  }
  for (int st = 0; st < 2; st++) {
    const int uses = (nsteps - st + 1) / 2;  // MMAs issued on this stage; all but the last waited
    if (uses > 0) {
      if (!mbar_wait(smem_u32(&mbar[st]), phase[st])) s_fail = 1;
      phase[st] ^= 1u;
    }
  }
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  __syncthreads();
  const bool ok = s_fail == 0 && nsteps > 0;
  if (s_fail && tid == 0) raise_status(status, DEV_ERR_TIMEOUT, blockIdx.x, blockIdx.y);
  const int kr = kt0 + warp * 32 + lane;  // this thread's accumulator row: (tap, c)
  const int ktap = kr / a.Ca, kc = kr - ktap * a.Ca;
#pragma unroll 1
  for (int c0 = 0; c0 < UMMA_N; c0 += 8) {
    uint32_t r[8];
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
    if (!ok || kr >= a.K || kc >= a.C) continue;
#pragma unroll
    for (int j = 0; j < 8; j++) {
      const int n = c0 + j;
      if (n < a.N) atomicAdd(&a.dW[((size_t)n * a.C + kc) * 9 + ktap], __uint_as_float(r[j]));
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(UMMA_N)
                 : "memory");
  // bias gradient (first row block only): the sums of the staged G^T values
  if (blockIdx.y == 0 && a.db) {
#pragma unroll
    for (int q = 0; q < 2; q++)
#pragma unroll
      for (int i = 0; i < 8; i++) {
        float v = bsum[q][i];
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        const int n = 8 * (warp + 4 * q) + i;
        if (lane == 0 && n < a.N) atomicAdd(&a.db[n], v);
      }
  }
}

// ------------------------------------------------------------- helpers ------
// Forward weights, K-major: Bf[n][tap * Ca + c] = W[n][c][tap]; dgrad weights:
// Bd[c][tap * Cg + n] = W[n][c][tap] (the taps are applied mirrored). BF16, zero
// outside the layer's channels.
__global__ void k_pack_weights(const float *W, int N, int C, int Ca, int Cg, __nv_bfloat16 *Bf,
                               int Npf, int Kpf, __nv_bfloat16 *Bd, int Npd, int Kpd) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < Npf * Kpf) {
    const int n = i / Kpf, k = i % Kpf, tap = k / Ca, c = k % Ca;
    Bf[i] = __float2bfloat16((n < N && tap < 9 && c < C) ? W[((size_t)n * C + c) * 9 + tap] : 0.f);
  }
  if (Bd && i < Npd * Kpd) {
    const int c = i / Kpd, k = i % Kpd, tap = k / Cg, n = k % Cg;
    Bd[i] = __float2bfloat16((c < C && tap < 9 && n < N) ? W[((size_t)n * C + c) * 9 + tap] : 0.f);
  }
}

// NCHW fp32 [B][C][HW] -> channels-last bf16 [B][HW][Cp], zero channels C..Cp-1.
__global__ void k_to_nhwc_bf16(const float *x, int B, int C, int HW, int Cp, __nv_bfloat16 *y) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)B * HW * Cp) return;
  const int c = (int)(i % Cp);
  const size_t pix = i / Cp;
  const size_t b = pix / HW, p = pix % HW;
  y[i] = __float2bfloat16(c < C ? x[(b * C + c) * HW + p] : 0.f);
}

// Net input: area mean of each 8x8 block (integer, as for I^n) of both frames,
// scaled to [-0.5, 0.5]. x: [B][6][Gy][Gx] fp32.
__global__ void k_net_input(const uint8_t *I1, const uint8_t *I2, int B, int W, int H, int n,
                            float *x) {
  const int Gx = (W + n - 1) / n, Gy = (H + n - 1) / n;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B * 6 * Gx * Gy) return;
  const int gx = i % Gx, gy = (i / Gx) % Gy, ch = (i / (Gx * Gy)) % 6, b = i / (6 * Gx * Gy);
  const uint8_t *img = (ch < 3 ? I1 : I2) + (size_t)b * W * H * 3;
  const int c = ch % 3;
  int s = 0, cnt = 0;
  for (int y = gy * n; y < min(gy * n + n, H); y++)
    for (int xx = gx * n; xx < min(gx * n + n, W); xx++) {
      s += img[((size_t)y * W + xx) * 3 + c];
      cnt++;
    }
  x[i] = (float)((s + cnt / 2) / cnt) / 255.f - 0.5f;
}

// Relaxed winner-takes-all L1 loss over the K hypotheses of each labelled point:
// the hypothesis nearest to the label (L1, ties to the lowest k) gets weight
// 1 - alpha, the others alpha / (K - 1). Flows are compared in units of
// flow_scale pixels. out: [B][2K][Gy][Gx]; label: [B][Gy][Gx][2] int16;
// valid: [B][Gy][Gx]. Writes dout = d(mean loss)/d(out) and accumulates the loss.
__global__ void k_wta_loss(const float *out, const int16_t *label, const uint8_t *valid, int B,
                           int K, int Gx, int Gy, float scale, float alpha, const int32_t *count,
                           float *dout, float *loss) {
  const int G = Gx * Gy;
  const float inv_count = *count > 0 ? 1.f / (float)*count : 0.f;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B * G) return;
  const int b = i / G, p = i % G;
  const float *o = out + (size_t)b * 2 * K * G + p;
  float *d = dout + (size_t)b * 2 * K * G + p;
  if (!valid[i]) {
    for (int k = 0; k < 2 * K; k++) d[(size_t)k * G] = 0.f;
    return;
  }
  const float lx = label[2 * (size_t)i] / scale, ly = label[2 * (size_t)i + 1] / scale;
  int best = 0;
  float bd = 0.f;
  for (int k = 0; k < K; k++) {
    const float e = fabsf(o[(size_t)(2 * k) * G] - lx) + fabsf(o[(size_t)(2 * k + 1) * G] - ly);
    if (k == 0 || e < bd) {
      bd = e;
      best = k;
    }
  }
  float l = 0.f;
  for (int k = 0; k < K; k++) {
    const float w = (K == 1) ? 1.f : (k == best ? 1.f - alpha : alpha / (K - 1));
    const float ex = o[(size_t)(2 * k) * G] - lx, ey = o[(size_t)(2 * k + 1) * G] - ly;
    l += w * (fabsf(ex) + fabsf(ey));
    d[(size_t)(2 * k) * G] = w * inv_count * (ex > 0.f ? 1.f : (ex < 0.f ? -1.f : 0.f));
    d[(size_t)(2 * k + 1) * G] = w * inv_count * (ey > 0.f ? 1.f : (ey < 0.f ? -1.f : 0.f));
  }
  atomicAdd(loss, l * inv_count);
}

__global__ void k_count_valid(const uint8_t *v, int n, int *cnt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  int c = (i < n && v[i]) ? 1 : 0;
  for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(cnt, c);
}

// Adam (Kingma & Ba, 2015) with bias correction.
__global__ void k_adam(size_t n, float *p, const float *g, float *m, float *v, float lr, float b1,
                       float b2, float eps, float c1, float c2) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi, vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// Integer proposals: rint(out * scale), [B][Gy][Gx][K][2] int16.
__global__ void k_proposals(const float *out, int B, int K, int Gx, int Gy, float scale,
                            int16_t *prop) {
  const int G = Gx * Gy;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B * G * K) return;
  const int k = i % K, p = (i / K) % G, b = i / (K * G);
  const float *o = out + (size_t)b * 2 * K * G + p;
  const float fx = rintf(o[(size_t)(2 * k) * G] * scale), fy = rintf(o[(size_t)(2 * k + 1) * G] * scale);
  prop[2 * (size_t)i] = (int16_t)fminf(fmaxf(fx, -16000.f), 16000.f);
  prop[2 * (size_t)i + 1] = (int16_t)fminf(fmaxf(fy, -16000.f), 16000.f);
}

// ------------------------------------------------------------ workspace ----
struct NetWs {
  __nv_bfloat16 *act[NET_LAYERS + 1];  // bf16 input of layer l, [P][Ca[l]]; act[4] unused
  float *pre[NET_LAYERS];              // fp32 pre-activation of layer l, [P][Cg[l]]
  __nv_bfloat16 *Bf[NET_LAYERS], *Bd[NET_LAYERS];
  __nv_bfloat16 *gbf[NET_LAYERS];      // bf16 gradient at the pre-activation of layer l, [P][Cg[l]]
  int Ca[NET_LAYERS], Cg[NET_LAYERS];  // channel strides: cin, cout padded to 8
  int Kpf[NET_LAYERS], Npf[NET_LAYERS], Kpd[NET_LAYERS], Npd[NET_LAYERS];
};

static NetWs net_ws(Arena &a, const NetShape &s, int B, int Gx, int Gy) {
  NetWs w;
  const size_t P = (size_t)B * Gx * Gy;
  for (int l = 0; l < NET_LAYERS; l++) {
    w.Ca[l] = cpad8(s.cin[l]);
    w.Cg[l] = cpad8(s.cout[l]);
    w.act[l] = a.take<__nv_bfloat16>(P * w.Ca[l]);
    w.pre[l] = a.take<float>(P * w.Cg[l]);
    w.gbf[l] = a.take<__nv_bfloat16>(P * w.Cg[l]);
    w.Kpf[l] = padk(9 * w.Ca[l]);
    w.Npf[l] = pad64(s.cout[l]);
    w.Kpd[l] = padk(9 * w.Cg[l]);
    w.Npd[l] = pad64(s.cin[l]);
    w.Bf[l] = a.take<__nv_bfloat16>((size_t)w.Kpf[l] * w.Npf[l]);
    w.Bd[l] = a.take<__nv_bfloat16>((size_t)w.Kpd[l] * w.Npd[l]);
  }
  w.act[NET_LAYERS] = nullptr;
  return w;
}

static ff_status launch_conv(ConvArgs c, int M, DeviceStatus *status, cudaStream_t st) {
  dim3 g((M + UMMA_M - 1) / UMMA_M, c.Np / UMMA_N);
  c.stall = net_stall_polls();
  FF_TRY(smem_opt_in((const void *)k_conv_umma, CONV_SMEM));
  k_conv_umma<<<g, 128, CONV_SMEM, st>>>(c, status);
  FF_CHECK_LAUNCH();
  return FF_OK;
}

}  // namespace ff

using namespace ff;

extern "C" {

ff_status ff_net_param_count(const ff_net_desc *d, size_t *n) {
  NetShape s;
  if (!n || !net_shape(d, s)) return FF_ERR_INVALID_ARG;
  *n = s.nparams;
  return FF_OK;
}

ff_status ff_net_workspace_size(const ff_net_desc *d, int B, int Gx, int Gy, size_t *bytes) {
  NetShape s;
  if (!bytes || !net_shape(d, s) || B < 1 || Gx < 1 || Gy < 1) return FF_ERR_INVALID_ARG;
  Arena a;
  a.take<char>(WS_HEADER);
  net_ws(a, s, B, Gx, Gy);
  *bytes = a.off;
  return FF_OK;
}

ff_status ff_net_input(const uint8_t *I1, const uint8_t *I2, int B, int W, int H, float *x,
                       void *stream) {
  if (!I1 || !I2 || !x || B < 1 || W < 1 || H < 1) return FF_ERR_INVALID_ARG;
  const int n = 8, Gx = (W + n - 1) / n, Gy = (H + n - 1) / n;
  const int tot = B * 6 * Gx * Gy;
  k_net_input<<<(tot + 255) / 256, 256, 0, (cudaStream_t)stream>>>(I1, I2, B, W, H, n, x);
  FF_CHECK_LAUNCH();
  return FF_OK;
}

ff_status ff_net_forward(const ff_net_desc *d, const float *params, const float *x, int B, int Gx,
                         int Gy, float *out, void *ws, size_t ws_bytes, void *stream) {
  NetShape s;
  if (!net_shape(d, s) || !params || !x || !out || B < 1 || Gx < 1 || Gy < 1)
    return FF_ERR_INVALID_ARG;
  size_t need;
  FF_TRY(ff_net_workspace_size(d, B, Gx, Gy, &need));
  if (!ws || ((uintptr_t)ws & 255) || ws_bytes < need) return FF_ERR_WORKSPACE;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemsetAsync(ws, 0, sizeof(DeviceStatus), st) != cudaSuccess) return FF_ERR_CUDA;
  Arena a(ws, ws_bytes);
  a.take<char>(WS_HEADER);
  NetWs w = net_ws(a, s, B, Gx, Gy);
  const size_t P = (size_t)B * Gx * Gy;
  {
    const size_t tot = P * w.Ca[0];
    k_to_nhwc_bf16<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(x, B, s.cin[0], Gx * Gy, w.Ca[0],
                                                                  w.act[0]);
    FF_CHECK_LAUNCH();
  }
  for (int l = 0; l < NET_LAYERS; l++) {
    const int tot = max(w.Kpf[l] * w.Npf[l], w.Kpd[l] * w.Npd[l]);
    k_pack_weights<<<(tot + 255) / 256, 256, 0, st>>>(params + s.woff[l], s.cout[l], s.cin[l],
                                                     w.Ca[l], w.Cg[l], w.Bf[l], w.Npf[l],
                                                     w.Kpf[l], w.Bd[l], w.Npd[l], w.Kpd[l]);
    FF_CHECK_LAUNCH();
    const bool last = l == NET_LAYERS - 1;
    ConvArgs c{};
    c.act = w.act[l];
    c.B = B;
    c.Ca = w.Ca[l];
    c.H = Gy;
    c.W = Gx;
    c.dil = s.dil[l];
    c.sign = 1;
    c.Bt = w.Bf[l];
    c.K = 9 * w.Ca[l];
    c.Kp = w.Kpf[l];
    c.N = s.cout[l];
    c.Np = w.Npf[l];
    c.bias = params + s.boff[l];
    c.out = last ? out : w.pre[l];
    c.out_nchw = last ? 1 : 0;
    c.out_bf = last ? nullptr : w.act[l + 1];
    c.relu = last ? 0 : 1;
    FF_TRY(launch_conv(c, (int)P, (DeviceStatus *)ws, st));
  }
  return FF_OK;
}

ff_status ff_net_backward(const ff_net_desc *d, const float *params, const float *dout, int B,
                          int Gx, int Gy, float *grads, void *ws, size_t ws_bytes, void *stream) {
  NetShape s;
  if (!net_shape(d, s) || !params || !dout || !grads || B < 1 || Gx < 1 || Gy < 1)
    return FF_ERR_INVALID_ARG;
  size_t need;
  FF_TRY(ff_net_workspace_size(d, B, Gx, Gy, &need));
  if (!ws || ((uintptr_t)ws & 255) || ws_bytes < need) return FF_ERR_WORKSPACE;
  cudaStream_t st = (cudaStream_t)stream;
  Arena a(ws, ws_bytes);
  a.take<char>(WS_HEADER);
  NetWs w = net_ws(a, s, B, Gx, Gy);
  const size_t P = (size_t)B * Gx * Gy;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1)
    return FF_ERR_CUDA;
  if (cudaMemsetAsync(grads, 0, sizeof(float) * s.nparams, st) != cudaSuccess) return FF_ERR_CUDA;
  if (cudaMemsetAsync(ws, 0, sizeof(DeviceStatus), st) != cudaSuccess) return FF_ERR_CUDA;
  // gradient at the last pre-activation (the output has no ReLU)
  const int L = NET_LAYERS - 1;
  {
    const size_t tot = P * w.Cg[L];
    k_to_nhwc_bf16<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(dout, B, s.cout[L], Gx * Gy,
                                                                  w.Cg[L], w.gbf[L]);
    FF_CHECK_LAUNCH();
  }
  for (int l = L; l >= 0; l--) {
    WgradArgs wa{};
    wa.g = w.gbf[l];
    wa.act = w.act[l];
    wa.B = B;
    wa.C = s.cin[l];
    wa.Ca = w.Ca[l];
    wa.H = Gy;
    wa.W = Gx;
    wa.dil = s.dil[l];
    wa.N = s.cout[l];
    wa.Cg = w.Cg[l];
    wa.K = 9 * w.Ca[l];
    wa.dW = grads + s.woff[l];
    wa.db = grads + s.boff[l];
    // pixel range per CTA: about six CTAs per SM over the whole grid (the
    // staging is load-latency bound), whole 32-pixel stages, at least 64 pixels
    const int ky = (wa.K + UMMA_M - 1) / UMMA_M;
    const long long want = (long long)nsm * 6;
    long long ppc = ((long long)P * ky + want - 1) / want;
    ppc = ((ppc + WG_PIX - 1) / WG_PIX) * WG_PIX;
    wa.pix_per_cta = (int)(ppc < 64 ? 64 : ppc);
    dim3 gw((unsigned)((P + wa.pix_per_cta - 1) / wa.pix_per_cta), ky);
    wa.stall = net_stall_polls();
    k_wgrad_umma<<<gw, 128, 0, st>>>(wa, (DeviceStatus *)ws);
    FF_CHECK_LAUNCH();
    if (l == 0) break;
    // dgrad: gradient at the input of layer l, masked by the ReLU of layer l-1
    ConvArgs c{};
    c.act = w.gbf[l];
    c.B = B;
    c.Ca = w.Cg[l];
    c.H = Gy;
    c.W = Gx;
    c.dil = s.dil[l];
    c.sign = -1;
    c.Bt = w.Bd[l];
    c.K = 9 * w.Cg[l];
    c.Kp = w.Kpd[l];
    c.N = s.cin[l];
    c.Np = w.Npd[l];
    c.bias = nullptr;
    c.out = nullptr;
    c.out_bf = w.gbf[l - 1];
    c.mask_pre = w.pre[l - 1];
    c.relu = 0;
    FF_TRY(launch_conv(c, (int)P, (DeviceStatus *)ws, st));
  }
  return FF_OK;
}

ff_status ff_net_loss(const ff_net_desc *d, const float *out, const int16_t *label,
                      const uint8_t *valid, int B, int Gx, int Gy, float flow_scale, float alpha,
                      float *loss, float *dout, int32_t *count, void *stream) {
  NetShape s;
  if (!net_shape(d, s) || !out || !label || !valid || !loss || !dout || !count || B < 1 ||
      flow_scale <= 0.f || alpha < 0.f || alpha > 1.f)
    return FF_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const int n = B * Gx * Gy;
  // mean over labelled points (counted on the device)
  if (cudaMemsetAsync(count, 0, sizeof(int32_t), st) != cudaSuccess) return FF_ERR_CUDA;
  k_count_valid<<<(n + 255) / 256, 256, 0, st>>>(valid, n, count);
  FF_CHECK_LAUNCH();
  if (cudaMemsetAsync(loss, 0, sizeof(float), st) != cudaSuccess) return FF_ERR_CUDA;
  k_wta_loss<<<(n + 255) / 256, 256, 0, st>>>(out, label, valid, B, d->k, Gx, Gy, flow_scale,
                                              alpha, count, dout, loss);
  FF_CHECK_LAUNCH();
  return FF_OK;
}

ff_status ff_net_adam(size_t n, float *params, const float *grads, float *m, float *v, int step,
                      float lr, float b1, float b2, float eps, void *stream) {
  if (!params || !grads || !m || !v || step < 1 || n == 0) return FF_ERR_INVALID_ARG;
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  k_adam<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(n, params, grads, m, v, lr,
                                                                       b1, b2, eps, c1, c2);
  FF_CHECK_LAUNCH();
  return FF_OK;
}

ff_status ff_net_proposals(const ff_net_desc *d, const float *out, int B, int Gx, int Gy,
                           float flow_scale, int16_t *proposals, void *stream) {
  NetShape s;
  if (!net_shape(d, s) || !out || !proposals || B < 1 || flow_scale <= 0.f)
    return FF_ERR_INVALID_ARG;
  const int tot = B * Gx * Gy * d->k;
  k_proposals<<<(tot + 255) / 256, 256, 0, (cudaStream_t)stream>>>(out, B, d->k, Gx, Gy, flow_scale,
                                                                  proposals);
  FF_CHECK_LAUNCH();
  return FF_OK;
}

}  // extern "C"
