// Sec. 3.1: Walsh-Hadamard patch features (27 per pixel: 9 bases x 3 channels).
//
// The (2r+1)-pixel window is split r | r+1 and each half again into two, giving
// 4 blocks per axis (r = 8: 4,4,4,5). The first three Walsh functions in sequency
// order are constant on those blocks with signs (++++), (++--), (+--+), so every
// feature is a signed sum of the 16 block sums of its channel:
//   f(c, i, j) = sum_{a,b} s_i[a] s_j[b] S_c[a][b]   (a = row block, b = column block).
//
// All-pixel kernel: a CTA stages a (32 + 2r) x (16 + 2r) RGB tile (clamped) in
// shared memory, turns it into a 2-D integral image, and every output pixel reads
// the 5 x 5 block corners per channel (75 shared loads) to form its 16 block
// sums. Output rows are 28 int32 (112 B): 27 features + a zero pad.
#include "ff_internal.cuh"

namespace ff {

__host__ __device__ inline void wht_blocks(int L, int *sz) {
  int h0 = L / 2, h1 = L - h0;
  sz[0] = h0 / 2;
  sz[1] = h0 - h0 / 2;
  sz[2] = h1 / 2;
  sz[3] = h1 - h1 / 2;
}

__constant__ int c_wsign[3][4] = {{1, 1, 1, 1}, {1, 1, -1, -1}, {1, -1, -1, 1}};

// Combine the 4x4 block sums of one channel into its 9 features.
__device__ __forceinline__ void combine9(const int S[4][4], int32_t *f) {
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) {
      int acc = 0;
#pragma unroll
      for (int a = 0; a < 4; a++)
#pragma unroll
        for (int b = 0; b < 4; b++) acc += c_wsign[i][a] * c_wsign[j][b] * S[a][b];
      f[3 * i + j] = acc;
    }
}

constexpr int FT_X = 32, FT_Y = 16;

// Integral image layout: [c][row 0..RH][col 0..RW], row/col 0 are zeros.
__global__ void __launch_bounds__(512) k_features_all(const uint8_t *__restrict__ img, int W, int H,
                                                      int r, int32_t *__restrict__ feat, int packed) {
  extern __shared__ int32_t sI[];
  const int L = 2 * r + 1;
  const int RW = FT_X + L - 1, RH = FT_Y + L - 1;
  const int SW = RW + 1, SH = RH + 1;
  const int x0 = blockIdx.x * FT_X, y0 = blockIdx.y * FT_Y;
  const int tid = threadIdx.x;
  // stage clamped pixels at [c][1 + ry][1 + rx]
  for (int t = tid; t < RW * RH; t += blockDim.x) {
    int rx = t % RW, ry = t / RW;
    int x = clampi(x0 - r + rx, 0, W - 1), y = clampi(y0 - r + ry, 0, H - 1);
    const uint8_t *p = img + ((size_t)y * W + x) * 3;
#pragma unroll
    for (int c = 0; c < 3; c++) sI[(c * SH + ry + 1) * SW + rx + 1] = p[c];
  }
  for (int t = tid; t < 3 * SW; t += blockDim.x) sI[((t / SW) * SH) * SW + t % SW] = 0;
  for (int t = tid; t < 3 * SH; t += blockDim.x) sI[((t / SH) * SH + t % SH) * SW] = 0;
  __syncthreads();
  for (int t = tid; t < 3 * RH; t += blockDim.x) {  // row prefix sums
    int32_t *row = sI + ((t / RH) * SH + 1 + t % RH) * SW;
    int32_t acc = 0;
    for (int x = 1; x < SW; x++) row[x] = (acc += row[x]);
  }
  __syncthreads();
  for (int t = tid; t < 3 * RW; t += blockDim.x) {  // column prefix sums
    int32_t *col = sI + (t / RW) * SH * SW + 1 + t % RW;
    int32_t acc = 0;
    for (int y = 1; y < SH; y++) col[y * SW] = (acc += col[y * SW]);
  }
  __syncthreads();
  int sz[4];
  wht_blocks(L, sz);
  const int lx = tid % FT_X, ly = tid / FT_X;
  const int x = x0 + lx, y = y0 + ly;
  if (x >= W || y >= H || ly >= FT_Y) return;
  int ex[5], ey[5];
  ex[0] = lx;
  ey[0] = ly;
#pragma unroll
  for (int a = 0; a < 4; a++) {
    ex[a + 1] = ex[a] + sz[a];
    ey[a + 1] = ey[a] + sz[a];
  }
  int32_t out[FEAT_STRIDE];
#pragma unroll
  for (int c = 0; c < 3; c++) {
    int Cn[5][5];
    const int32_t *Ic = sI + c * SH * SW;
#pragma unroll
    for (int a = 0; a < 5; a++)
#pragma unroll
      for (int b = 0; b < 5; b++) Cn[a][b] = Ic[ey[a] * SW + ex[b]];
    int S[4][4];
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
      for (int b = 0; b < 4; b++) S[a][b] = Cn[a + 1][b + 1] - Cn[a][b + 1] - Cn[a + 1][b] + Cn[a][b];
    combine9(S, out + 9 * c);
  }
  out[27] = 0;
  if (packed) {  // 64-byte rows of 18-bit fields (|value| <= (2r+1)^2 * 255 < 2^17)
    uint32_t w[FEAT_PACKED_WORDS];
    pack_feat_row(out, w);
    uint4 *dst = (uint4 *)(feat + ((size_t)y * W + x) * FEAT_PACKED_WORDS);
#pragma unroll
    for (int q = 0; q < 4; q++) dst[q] = make_uint4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
    return;
  }
  int4 *dst = (int4 *)(feat + ((size_t)y * W + x) * FEAT_STRIDE);
#pragma unroll
  for (int q = 0; q < 7; q++) dst[q] = make_int4(out[4 * q], out[4 * q + 1], out[4 * q + 2], out[4 * q + 3]);
}

// Features at a point list or at the grid of spacing grid_n; direct block sums.
// Point-list kernel: one warp per point. Lanes 0..15 each sum one of the 4 x 4
// blocks (a = lane / 4 rows, b = lane % 4 columns) for the three channels, then
// lanes 0..2 combine their channel's 16 sums into its 9 features.
constexpr int PTS_WARPS = 4;

__global__ void __launch_bounds__(PTS_WARPS * 32) k_features_pts(
    const uint8_t *__restrict__ img, int W, int H, int r, const int32_t *__restrict__ pts, int npts,
    int grid_n, int Gx, int32_t *__restrict__ feat) {
  __shared__ int sS[PTS_WARPS][3][4][4];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int k = blockIdx.x * PTS_WARPS + warp;
  if (k >= npts) return;  // whole warp
  int x, y;
  if (pts) {
    x = pts[2 * k];
    y = pts[2 * k + 1];
  } else {
    x = (k % Gx) * grid_n;
    y = (k / Gx) * grid_n;
  }
  const int L = 2 * r + 1;
  int sz[4], st[5];
  wht_blocks(L, sz);
  st[0] = 0;
  for (int a = 0; a < 4; a++) st[a + 1] = st[a] + sz[a];
  if (lane < 16) {
    const int a = lane >> 2, b = lane & 3;
    int s0 = 0, s1 = 0, s2 = 0;
    for (int v = st[a]; v < st[a + 1]; v++) {
      const int yy = clampi(y - r + v, 0, H - 1);
      for (int u = st[b]; u < st[b + 1]; u++) {
        const uint8_t *q = img + ((size_t)yy * W + clampi(x - r + u, 0, W - 1)) * 3;
        s0 += q[0];
        s1 += q[1];
        s2 += q[2];
      }
    }
    sS[warp][0][a][b] = s0;
    sS[warp][1][a][b] = s1;
    sS[warp][2][a][b] = s2;
  }
  __syncwarp();
  if (lane < 3) {
    int32_t out[9];
    combine9(sS[warp][lane], out);
    for (int q = 0; q < 9; q++) feat[(size_t)k * FEAT_STRIDE + 9 * lane + q] = out[q];
  } else if (lane == 3) {
    feat[(size_t)k * FEAT_STRIDE + 27] = 0;
  }
}

ff_status launch_features(const uint8_t *img, int W, int H, int r, const int32_t *pts, int npts,
                          int grid_n, int32_t *feat, cudaStream_t st, bool packed) {
  if (packed && (pts || grid_n != 1 || r < 1 || r > 8)) return FF_ERR_INVALID_ARG;
  if (!pts && grid_n == 1) {
    const int L = 2 * r + 1;
    size_t smem = sizeof(int32_t) * 3 * (FT_X + L) * (FT_Y + L);
    FF_TRY(smem_opt_in((const void *)k_features_all, smem));
    dim3 g((W + FT_X - 1) / FT_X, (H + FT_Y - 1) / FT_Y);
    k_features_all<<<g, FT_X * FT_Y, smem, st>>>(img, W, H, r, feat, packed ? 1 : 0);
    FF_CHECK_LAUNCH();
    return FF_OK;
  }
  int Gx = (W + grid_n - 1) / grid_n;
  if (!pts) npts = Gx * ((H + grid_n - 1) / grid_n);
  if (npts <= 0) return FF_OK;
  k_features_pts<<<(npts + PTS_WARPS - 1) / PTS_WARPS, PTS_WARPS * 32, 0, st>>>(img, W, H, r, pts,
                                                                                 npts, grid_n, Gx, feat);
  FF_CHECK_LAUNCH();
  return FF_OK;
}

}  // namespace ff
