// Learned proposal net (not in the paper): a small convolutional net that reads
// the coarsest pyramid level of both frames and emits K flow candidates per grid
// point of the coarsest search level; they are tried beside the kd-tree
// candidates (Eq. 1/4 rerank), so they can only ever replace the kd result when
// the exact integer data term prefers them.
//
// Layers l = 0..3: 3x3 convolution, dilation dil[l], zero padding dil[l], bias,
// ReLU except after the last layer. Channels cin(=6) -> c1 -> c2 -> c3 -> 2K.
// Activations are NCHW; every convolution input is BF16 and accumulates in FP32.
// Parameters (FP32 master copy) per layer: W [cout][cin][3][3], then b [cout].
//
// All three convolution products are implicit GEMMs on the tensor cores
// (mma.sync m16n8k16, BF16 x BF16 -> FP32):
//   forward   out[m][n]  = sum_k A[m][k] B[k][n],  m = pixel, n = cout, k = (cin, tap)
//   dgrad     din[m][n]  = sum_k G[m][k] Bd[k][n], m = pixel, n = cin,  k = (cout, tap), taps mirrored
//   wgrad     dW[n][k]   = sum_m G[m][n] A[m][k]   (reduction over pixels, split across CTAs)
// where A is the im2col view of the layer input and G the gradient at the
// pre-activation. One CTA computes a 64 x 64 output tile with 4 warps (16 rows
// each, 8 n-tiles of 8); K is staged in shared memory 16 at a time.
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

static int pad16(int v) { return (v + 15) & ~15; }
static int pad64(int v) { return (v + 63) & ~63; }

// ---------------------------------------------------------------- mma -------
__device__ __forceinline__ void mma_bf16(float *c, const uint32_t *a, const uint32_t *b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// 64x64 tile of out = A B with A[64][16] and B^T[64][16] staged per K step.
// sA: [64][24] bf16 (row = m), sB: [64][24] bf16 (row = n); the pitch 24 keeps
// the 32-bit fragment loads conflict-free.
constexpr int SP = 24;

__device__ __forceinline__ void tile_mma(const __nv_bfloat16 *sA, const __nv_bfloat16 *sB,
                                         float acc[8][4], int warp, int lane) {
  const int g = lane >> 2, t = lane & 3;
  const __nv_bfloat16 *ar = sA + (warp * 16 + g) * SP;
  uint32_t a[4];
  a[0] = *(const uint32_t *)(ar + 2 * t);
  a[1] = *(const uint32_t *)(ar + 8 * SP + 2 * t);
  a[2] = *(const uint32_t *)(ar + 2 * t + 8);
  a[3] = *(const uint32_t *)(ar + 8 * SP + 2 * t + 8);
#pragma unroll
  for (int j = 0; j < 8; j++) {
    const __nv_bfloat16 *br = sB + (8 * j + g) * SP;
    uint32_t b[2];
    b[0] = *(const uint32_t *)(br + 2 * t);
    b[1] = *(const uint32_t *)(br + 2 * t + 8);
    mma_bf16(acc[j], a, b);
  }
}

// ------------------------------------------------------- forward / dgrad -----
// out[b][n][y][x] = bias[n] + sum_{c, tap} Bmat[(c,tap)][n] * act[b][c][y + s*oy][x + s*ox]
// with (oy, ox) = ((tap/3)-1, (tap%3)-1) * dil and s = +1 (forward) or -1 (dgrad).
// Optionally writes the pre-activation (fp32) and relu'd BF16 copy, or, for
// dgrad, multiplies by the ReLU mask of the lower layer's pre-activation.
struct ConvArgs {
  const __nv_bfloat16 *act;  // [B][C][H][W]
  int B, C, H, W, dil, sign;
  const __nv_bfloat16 *Bmat;  // [Kp][Np] row-major, K = C*9 (zero rows up to Kp)
  int K, Kp, N, Np;
  const float *bias;           // [N] or null
  float *out;                  // [B][N][H][W] fp32 or null
  __nv_bfloat16 *out_bf;       // [B][N][H][W] bf16 of relu(out) (or of out*mask) or null
  const float *mask_pre;       // dgrad: lower layer's pre-activation [B][N][H][W]; grad *= (pre > 0)
  int relu;
};

__global__ void __launch_bounds__(128) k_conv_gemm(ConvArgs a) {
  __shared__ __align__(16) __nv_bfloat16 sA[64 * SP];
  __shared__ __align__(16) __nv_bfloat16 sB[64 * SP];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int HW = a.H * a.W, M = a.B * HW;
  const int m0 = blockIdx.x * 64, n0 = blockIdx.y * 64;
  float acc[8][4];
#pragma unroll
  for (int j = 0; j < 8; j++) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
  // Each thread stages column kk = tid % 16 of the A and B^T tiles for rows
  // tid / 16 + 8 j (j = 0..7); the pixel coordinates of its A rows are computed
  // once, and the next k chunk is loaded into registers while the current one
  // is multiplied.
  const int kk = tid & 15, r0 = tid >> 4;
  int rb[8], ry[8], rx[8];
#pragma unroll
  for (int j = 0; j < 8; j++) {
    const int m = m0 + r0 + 8 * j;
    if (m < M) {
      const int b = m / HW, p = m - b * HW;
      rb[j] = b;
      ry[j] = p / a.W;
      rx[j] = p - ry[j] * a.W;
    } else {
      rb[j] = -1;
      ry[j] = rx[j] = 0;
    }
  }
  __nv_bfloat16 va[8], vb[8];
  auto load_chunk = [&](int k0) {
    const int k = k0 + kk;
    const bool kin = k < a.K;
    const int c = kin ? k / 9 : 0, tap = kin ? k - 9 * (k / 9) : 0;
    const int dy = a.sign * ((tap / 3) - 1) * a.dil, dx = a.sign * ((tap % 3) - 1) * a.dil;
#pragma unroll
    for (int j = 0; j < 8; j++) {
      const int yy = ry[j] + dy, xx = rx[j] + dx;
      va[j] = (kin && rb[j] >= 0 && yy >= 0 && yy < a.H && xx >= 0 && xx < a.W)
                  ? a.act[((size_t)rb[j] * a.C + c) * HW + (size_t)yy * a.W + xx]
                  : __float2bfloat16(0.f);
      vb[j] = a.Bmat[(size_t)k * a.Np + n0 + r0 + 8 * j];  // zero rows pad K up to Kp
    }
  };
  load_chunk(0);
  for (int k0 = 0; k0 < a.Kp; k0 += 16) {
#pragma unroll
    for (int j = 0; j < 8; j++) {
      sA[(r0 + 8 * j) * SP + kk] = va[j];
      sB[(r0 + 8 * j) * SP + kk] = vb[j];
    }
    __syncthreads();
    if (k0 + 16 < a.Kp) load_chunk(k0 + 16);
    tile_mma(sA, sB, acc, warp, lane);
    __syncthreads();
  }
  // epilogue: rows g, g+8 of this warp's 16; columns 8j + 2t, +1
  const int g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int j = 0; j < 8; j++)
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const int m = m0 + warp * 16 + g + (q >> 1) * 8, n = n0 + 8 * j + 2 * t + (q & 1);
      if (m >= M || n >= a.N) continue;
      const int b = m / HW, p = m % HW;
      const size_t o = ((size_t)b * a.N + n) * HW + p;
      float v = acc[j][q] + (a.bias ? a.bias[n] : 0.f);
      if (a.mask_pre && !(a.mask_pre[o] > 0.f)) v = 0.f;
      if (a.out) a.out[o] = v;
      if (a.out_bf) a.out_bf[o] = __float2bfloat16(a.relu ? fmaxf(v, 0.f) : v);
    }
}

// ------------------------------------------------------------------ wgrad ---
// dW[n][k] += sum_m G[m][n] A[m][k] over the pixels of this CTA's chunk;
// n = cout (rows of the tile), k = (cin, tap) (columns). Partial sums are added
// into dW with atomics (the FP32 summation order is unspecified).
struct WgradArgs {
  const __nv_bfloat16 *g;    // [B][N][H][W] gradient at the pre-activation
  const __nv_bfloat16 *act;  // [B][C][H][W] layer input
  int B, C, H, W, dil, N, K;
  float *dW;                 // [N][K]
  float *db;                 // [N]
  int pix_per_cta;
};

__global__ void __launch_bounds__(128) k_conv_wgrad(WgradArgs a) {
  __shared__ __align__(16) __nv_bfloat16 sA[64 * SP];  // rows n, cols 16 pixels
  __shared__ __align__(16) __nv_bfloat16 sB[64 * SP];  // rows k, cols 16 pixels
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int HW = a.H * a.W, M = a.B * HW;
  const int kcol0 = blockIdx.y * 64;
  const int p0 = blockIdx.x * a.pix_per_cta, p1 = min(p0 + a.pix_per_cta, M);
  float acc[8][4];
#pragma unroll
  for (int j = 0; j < 8; j++) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
  // Each thread stages pixel column kk = tid % 16 for rows tid / 16 + 8 j: the
  // (channel, tap) of its eight k rows are fixed, its pixel changes per chunk,
  // and the next chunk is loaded into registers while the current one is used.
  const int kk = tid & 15, r0 = tid >> 4;
  int kc[8], kdy[8], kdx[8];
#pragma unroll
  for (int j = 0; j < 8; j++) {
    const int k = kcol0 + r0 + 8 * j;
    const int tap = k % 9;
    kc[j] = k < a.K ? k / 9 : -1;
    kdy[j] = ((tap / 3) - 1) * a.dil;
    kdx[j] = ((tap % 3) - 1) * a.dil;
  }
  __nv_bfloat16 vg[8], va[8];
  auto load_chunk = [&](int q0) {
    const int m = q0 + kk;
    const bool in = m < p1;
    const int b = in ? m / HW : 0, p = in ? m - b * HW : 0;
    const int y = p / a.W, x = p - y * a.W;
#pragma unroll
    for (int j = 0; j < 8; j++) {
      const int r = r0 + 8 * j;
      vg[j] = (in && r < a.N) ? a.g[((size_t)b * a.N + r) * HW + p] : __float2bfloat16(0.f);
      const int yy = y + kdy[j], xx = x + kdx[j];
      va[j] = (in && kc[j] >= 0 && yy >= 0 && yy < a.H && xx >= 0 && xx < a.W)
                  ? a.act[((size_t)b * a.C + kc[j]) * HW + (size_t)yy * a.W + xx]
                  : __float2bfloat16(0.f);
    }
  };
  if (p0 < p1) load_chunk(p0);
  for (int q0 = p0; q0 < p1; q0 += 16) {
#pragma unroll
    for (int j = 0; j < 8; j++) {
      sA[(r0 + 8 * j) * SP + kk] = vg[j];
      sB[(r0 + 8 * j) * SP + kk] = va[j];
    }
    __syncthreads();
    if (q0 + 16 < p1) load_chunk(q0 + 16);
    tile_mma(sA, sB, acc, warp, lane);
    __syncthreads();
  }
  const int g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int j = 0; j < 8; j++)
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const int n = warp * 16 + g + (q >> 1) * 8, k = kcol0 + 8 * j + 2 * t + (q & 1);
      if (n < a.N && k < a.K) atomicAdd(&a.dW[(size_t)n * a.K + k], acc[j][q]);
    }
  // bias gradient from the first column block only
  if (blockIdx.y == 0 && a.db)
    for (int n = warp; n < a.N; n += 4) {
      float s = 0.f;
      for (int m = p0 + lane; m < p1; m += 32) {
        const int b = m / HW, p = m % HW;
        s += __bfloat162float(a.g[((size_t)b * a.N + n) * HW + p]);
      }
      for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) atomicAdd(&a.db[n], s);
    }
}

// ------------------------------------------------------------- helpers ------
// Forward weight matrix: Bf[(c*9 + tap)][n] = W[n][c][tap] (bf16, zero padded).
// Dgrad weight matrix:   Bd[(n*9 + tap)][c] = W[n][c][tap] (taps applied mirrored).
__global__ void k_pack_weights(const float *W, int N, int C, __nv_bfloat16 *Bf, int Npf,
                               __nv_bfloat16 *Bd, int Npd, int Kpf, int Kpd) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int total = max(Kpf * Npf, Kpd * Npd);
  if (i >= total) return;
  if (i < Kpf * Npf) {
    const int k = i / Npf, n = i % Npf, c = k / 9, tap = k % 9;
    Bf[i] = __float2bfloat16((k < C * 9 && n < N) ? W[((size_t)n * C + c) * 9 + tap] : 0.f);
  }
  if (Bd && i < Kpd * Npd) {
    const int k = i / Npd, c = i % Npd, n = k / 9, tap = k % 9;
    Bd[i] = __float2bfloat16((k < N * 9 && c < C) ? W[((size_t)n * C + c) * 9 + tap] : 0.f);
  }
}

__global__ void k_to_bf16(const float *x, size_t n, __nv_bfloat16 *y) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = __float2bfloat16(x[i]);
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
  __nv_bfloat16 *act[NET_LAYERS + 1];  // bf16 input of layer l (act[0] = x); act[4] unused
  float *pre[NET_LAYERS];              // fp32 pre-activation of layer l
  __nv_bfloat16 *Bf[NET_LAYERS], *Bd[NET_LAYERS];
  __nv_bfloat16 *gbf[NET_LAYERS];      // bf16 gradient at the pre-activation of layer l
  int Kpf[NET_LAYERS], Npf[NET_LAYERS], Kpd[NET_LAYERS], Npd[NET_LAYERS];
};

static NetWs net_ws(Arena &a, const NetShape &s, int B, int Gx, int Gy) {
  NetWs w;
  const size_t P = (size_t)B * Gx * Gy;
  for (int l = 0; l < NET_LAYERS; l++) {
    w.act[l] = a.take<__nv_bfloat16>(P * s.cin[l]);
    w.pre[l] = a.take<float>(P * s.cout[l]);
    w.gbf[l] = a.take<__nv_bfloat16>(P * s.cout[l]);
    w.Kpf[l] = pad16(s.cin[l] * 9);
    w.Npf[l] = pad64(s.cout[l]);
    w.Kpd[l] = pad16(s.cout[l] * 9);
    w.Npd[l] = pad64(s.cin[l]);
    w.Bf[l] = a.take<__nv_bfloat16>((size_t)w.Kpf[l] * w.Npf[l]);
    w.Bd[l] = a.take<__nv_bfloat16>((size_t)w.Kpd[l] * w.Npd[l]);
  }
  w.act[NET_LAYERS] = nullptr;
  return w;
}

static ff_status launch_conv(const ConvArgs &c, int M, cudaStream_t st) {
  dim3 g((M + 63) / 64, c.Np / 64);
  k_conv_gemm<<<g, 128, 0, st>>>(c);
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
  Arena a(ws, ws_bytes);
  a.take<char>(WS_HEADER);
  NetWs w = net_ws(a, s, B, Gx, Gy);
  const size_t P = (size_t)B * Gx * Gy;
  k_to_bf16<<<(unsigned)((P * s.cin[0] + 255) / 256), 256, 0, st>>>(x, P * s.cin[0], w.act[0]);
  FF_CHECK_LAUNCH();
  for (int l = 0; l < NET_LAYERS; l++) {
    const int tot = max(w.Kpf[l] * w.Npf[l], w.Kpd[l] * w.Npd[l]);
    k_pack_weights<<<(tot + 255) / 256, 256, 0, st>>>(params + s.woff[l], s.cout[l], s.cin[l],
                                                     w.Bf[l], w.Npf[l], w.Bd[l], w.Npd[l],
                                                     w.Kpf[l], w.Kpd[l]);
    FF_CHECK_LAUNCH();
    const bool last = l == NET_LAYERS - 1;
    ConvArgs c{};
    c.act = w.act[l];
    c.B = B;
    c.C = s.cin[l];
    c.H = Gy;
    c.W = Gx;
    c.dil = s.dil[l];
    c.sign = 1;
    c.Bmat = w.Bf[l];
    c.K = s.cin[l] * 9;
    c.Kp = w.Kpf[l];
    c.N = s.cout[l];
    c.Np = w.Npf[l];
    c.bias = params + s.boff[l];
    c.out = last ? out : w.pre[l];
    c.out_bf = last ? nullptr : w.act[l + 1];
    c.relu = last ? 0 : 1;
    FF_TRY(launch_conv(c, (int)P, st));
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
  if (cudaMemsetAsync(grads, 0, sizeof(float) * s.nparams, st) != cudaSuccess) return FF_ERR_CUDA;
  // gradient at the last pre-activation (the output has no ReLU)
  const int L = NET_LAYERS - 1;
  k_to_bf16<<<(unsigned)((P * s.cout[L] + 255) / 256), 256, 0, st>>>(dout, P * s.cout[L], w.gbf[L]);
  FF_CHECK_LAUNCH();
  for (int l = L; l >= 0; l--) {
    WgradArgs wa{};
    wa.g = w.gbf[l];
    wa.act = w.act[l];
    wa.B = B;
    wa.C = s.cin[l];
    wa.H = Gy;
    wa.W = Gx;
    wa.dil = s.dil[l];
    wa.N = s.cout[l];
    wa.K = s.cin[l] * 9;
    wa.dW = grads + s.woff[l];
    wa.db = grads + s.boff[l];
    wa.pix_per_cta = 512;
    dim3 gw((unsigned)((P + wa.pix_per_cta - 1) / wa.pix_per_cta), (wa.K + 63) / 64);
    k_conv_wgrad<<<gw, 128, 0, st>>>(wa);
    FF_CHECK_LAUNCH();
    if (l == 0) break;
    // dgrad: gradient at the input of layer l, masked by the ReLU of layer l-1
    ConvArgs c{};
    c.act = w.gbf[l];
    c.B = B;
    c.C = s.cout[l];
    c.H = Gy;
    c.W = Gx;
    c.dil = s.dil[l];
    c.sign = -1;
    c.Bmat = w.Bd[l];
    c.K = s.cout[l] * 9;
    c.Kp = w.Kpd[l];
    c.N = s.cin[l];
    c.Np = w.Npd[l];
    c.bias = nullptr;
    c.out = nullptr;
    c.out_bf = w.gbf[l - 1];
    c.mask_pre = w.pre[l - 1];
    c.relu = 0;
    FF_TRY(launch_conv(c, (int)P, st));
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
