// Sec. 3.2 smoothed images I^n (area down + Lanczos up) and Sec. 3.3 census.
//
// All three image kernels are HBM/L2-streaming elementwise passes with small
// fixed stencils; one thread per output element, 256-thread blocks.
#include <math.h>

#include "ff_internal.cuh"

namespace ff {

// Lanczos-3 taps for integer upsampling by n. The coarse sample j is centred on
// full-resolution position j*n + (n-1)/2, so pixel x sits at coarse coordinate
// u = (2x - n + 1) / (2n); the six taps j0-2 .. j0+3 around j0 = floor(u) get
// weight L(u - j), normalised, scaled to Q14 and rounded half away from zero;
// the largest-magnitude tap (first on ties) absorbs the rounding residual so a
// phase sums to exactly 16384. Computed on the host in double precision.
static double lanczos_kernel3(double t) {
  if (t == 0.0) return 1.0;
  if (t <= -3.0 || t >= 3.0) return 0.0;
  const double a = M_PI * t;
  return 3.0 * sin(a) * sin(a / 3.0) / (a * a);
}

void lanczos_table(int n, LanczosTable *t) {
  for (int phase = 0; phase < n; phase++) {
    long num = 2L * phase - n + 1, den = 2L * n;
    long j0 = num >= 0 ? num / den : -((-num + den - 1) / den);
    double frac = (double)(num - j0 * den) / (double)den;
    double raw[6], total = 0.0;
    for (int k = 0; k < 6; k++) {
      raw[k] = lanczos_kernel3(frac - (k - 2));
      total += raw[k];
    }
    int sum = 0, arg = 0;
    for (int k = 0; k < 6; k++) {
      double v = raw[k] * 16384.0 / total;
      int q = v < 0 ? -(int)floor(-v + 0.5) : (int)floor(v + 0.5);
      t->w[phase][k] = q;
      sum += q;
    }
    for (int k = 1; k < 6; k++)
      if (abs(t->w[phase][k]) > abs(t->w[phase][arg])) arg = k;
    t->w[phase][arg] += 16384 - sum;
    t->base[phase] = (int32_t)j0;
  }
}

__device__ __forceinline__ void area_down_at(const uint8_t *__restrict__ img, int W, int H, int n,
                                             uint8_t *__restrict__ out, int Wc, int t) {
  int c = t % 3, i = (t / 3) % Wc, j = t / (3 * Wc);
  int x0 = i * n, y0 = j * n, x1 = min(x0 + n, W), y1 = min(y0 + n, H);
  int s = 0;
  for (int y = y0; y < y1; y++)
    for (int x = x0; x < x1; x++) s += img[((size_t)y * W + x) * 3 + c];
  int cnt = (x1 - x0) * (y1 - y0);
  out[t] = (uint8_t)((s + cnt / 2) / cnt);
}
__global__ void k_area_down(const uint8_t *__restrict__ img, int W, int H, int n,
                            uint8_t *__restrict__ out, int Wc, int Hc) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= Wc * Hc * 3) return;
  area_down_at(img, W, H, n, out, Wc, t);
}

// Horizontal pass on the coarse rows: h[yc][x][c] = sum_k w_k(x mod n) D[yc][clamp(j0+k)].
__device__ __forceinline__ void lanczos_h_at(const uint8_t *__restrict__ down, int Wc, int W, int n,
                                             const LanczosTable &tab, int32_t *__restrict__ h,
                                             int t) {
  int c = t % 3, x = (t / 3) % W, yc = t / (3 * W);
  int ph = x % n, j0 = x / n + tab.base[ph];
  int32_t acc = 0;
#pragma unroll
  for (int k = 0; k < 6; k++) {
    int j = clampi(j0 + k - 2, 0, Wc - 1);
    acc += tab.w[ph][k] * (int32_t)down[((size_t)yc * Wc + j) * 3 + c];
  }
  h[t] = acc;
}
__global__ void k_lanczos_h(const uint8_t *__restrict__ down, int Wc, int Hc, int W, int n,
                            LanczosTable tab, int32_t *__restrict__ h) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= Hc * W * 3) return;
  lanczos_h_at(down, Wc, W, n, tab, h, t);
}

// Vertical pass to full resolution, rounded (acc + 2^27) >> 28 and clamped.
__device__ __forceinline__ void lanczos_v_at(const int32_t *__restrict__ h, int Hc, int W, int n,
                                             const LanczosTable &tab, uint8_t *__restrict__ out,
                                             int t) {
  int c = t % 3, x = (t / 3) % W, y = t / (3 * W);
  int ph = y % n, j0 = y / n + tab.base[ph];
  long long acc = 0;
#pragma unroll
  for (int k = 0; k < 6; k++) {
    int j = clampi(j0 + k - 2, 0, Hc - 1);
    acc += (long long)tab.w[ph][k] * h[((size_t)j * W + x) * 3 + c];
  }
  long long v = (acc + (1ll << 27)) >> 28;  // arithmetic shift = floor division
  out[t] = (uint8_t)(v < 0 ? 0 : (v > 255 ? 255 : v));
}
__global__ void k_lanczos_v(const int32_t *__restrict__ h, int Hc, int W, int H, int n,
                            LanczosTable tab, uint8_t *__restrict__ out) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= H * W * 3) return;
  lanczos_v_at(h, Hc, W, n, tab, out, t);
}

size_t smooth_scratch_bytes(int W, int H, int n) {
  if (n <= 1) return 0;
  int Wc = (W + n - 1) / n, Hc = (H + n - 1) / n;
  size_t a = ((size_t)Wc * Hc * 3 + 255) & ~(size_t)255;
  return a + (size_t)Hc * W * 3 * sizeof(int32_t);
}

ff_status launch_smooth(const uint8_t *img, int W, int H, int n, uint8_t *out, void *scratch,
                        cudaStream_t st) {
  if (n == 1) {
    if (cudaMemcpyAsync(out, img, (size_t)W * H * 3, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      return FF_ERR_CUDA;
    return FF_OK;
  }
  int Wc = (W + n - 1) / n, Hc = (H + n - 1) / n;
  uint8_t *down = (uint8_t *)scratch;
  int32_t *h = (int32_t *)((char *)scratch + (((size_t)Wc * Hc * 3 + 255) & ~(size_t)255));
  LanczosTable tab;
  lanczos_table(n, &tab);
  const int B = 256;
  int na = Wc * Hc * 3, nh = Hc * W * 3, nv = H * W * 3;
  k_area_down<<<(na + B - 1) / B, B, 0, st>>>(img, W, H, n, down, Wc, Hc);
  FF_CHECK_LAUNCH();
  k_lanczos_h<<<(nh + B - 1) / B, B, 0, st>>>(down, Wc, Hc, W, n, tab, h);
  FF_CHECK_LAUNCH();
  k_lanczos_v<<<(nv + B - 1) / B, B, 0, st>>>(h, Hc, W, H, n, tab, out);
  FF_CHECK_LAUNCH();
  return FF_OK;
}

// Census: bit 8c + o set when channel c of neighbour o (raster order of the
// 3x3 neighbourhood at spacing n, centre skipped, clamped) is below the centre.
__device__ __forceinline__ void census_at(const uint8_t *__restrict__ img, int W, int H, int n,
                                          uint32_t *__restrict__ out, int x, int y) {
  const uint8_t *ctr = img + ((size_t)y * W + x) * 3;
  int c0 = ctr[0], c1 = ctr[1], c2 = ctr[2];
  uint32_t code = 0;
  int o = 0;
#pragma unroll
  for (int dy = -1; dy <= 1; dy++)
#pragma unroll
    for (int dx = -1; dx <= 1; dx++) {
      if (dx == 0 && dy == 0) continue;
      int xx = clampi(x + n * dx, 0, W - 1), yy = clampi(y + n * dy, 0, H - 1);
      const uint8_t *q = img + ((size_t)yy * W + xx) * 3;
      code |= (uint32_t)(q[0] < c0) << o;
      code |= (uint32_t)(q[1] < c1) << (8 + o);
      code |= (uint32_t)(q[2] < c2) << (16 + o);
      o++;
    }
  out[(size_t)y * W + x] = code;
}
__global__ void k_census(const uint8_t *__restrict__ img, int W, int H, int n,
                         uint32_t *__restrict__ out) {
  int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= W || y >= H) return;
  census_at(img, W, H, n, out, x, y);
}

ff_status launch_census(const uint8_t *imgn, int W, int H, int n, uint32_t *out, cudaStream_t st) {
  dim3 b(32, 8), g((W + 31) / 32, (H + 7) / 8);
  k_census<<<g, b, 0, st>>>(imgn, W, H, n, out);
  FF_CHECK_LAUNCH();
  return FF_OK;
}

// Sec. 3.1, subpixel targets: the census of I^n interpolated at (x + a/q,
// y + b/q). Colours are q^2 times the bilinear value, sum over i, j in {0, 1} of
// (i ? a : q - a) (j ? b : q - b) I^n(clamp(x + i), clamp(y + j)), so every
// comparison is exact; the census compares them as k_census compares pixels.
__device__ __forceinline__ void interp_px(const uint8_t *__restrict__ img, int W, int H, int x,
                                          int y, int q, int a, int b, int *c) {
  const int x1 = min(x + 1, W - 1), y1 = min(y + 1, H - 1);
  const uint8_t *p00 = img + ((size_t)y * W + x) * 3, *p10 = img + ((size_t)y * W + x1) * 3;
  const uint8_t *p01 = img + ((size_t)y1 * W + x) * 3, *p11 = img + ((size_t)y1 * W + x1) * 3;
  const int w00 = (q - a) * (q - b), w10 = a * (q - b), w01 = (q - a) * b, w11 = a * b;
#pragma unroll
  for (int ch = 0; ch < 3; ch++) c[ch] = w00 * p00[ch] + w10 * p10[ch] + w01 * p01[ch] + w11 * p11[ch];
}

__global__ void k_census_subpel(const uint8_t *__restrict__ img, int W, int H, int n, int q, int a,
                                int b, uint32_t *__restrict__ out) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= W || y >= H) return;
  int ctr[3];
  interp_px(img, W, H, x, y, q, a, b, ctr);
  uint32_t code = 0;
  int o = 0;
#pragma unroll
  for (int dy = -1; dy <= 1; dy++)
#pragma unroll
    for (int dx = -1; dx <= 1; dx++) {
      if (dx == 0 && dy == 0) continue;
      int v[3];
      interp_px(img, W, H, clampi(x + n * dx, 0, W - 1), clampi(y + n * dy, 0, H - 1), q, a, b, v);
      code |= (uint32_t)(v[0] < ctr[0]) << o;
      code |= (uint32_t)(v[1] < ctr[1]) << (8 + o);
      code |= (uint32_t)(v[2] < ctr[2]) << (16 + o);
      o++;
    }
  out[(size_t)y * W + x] = code;
}

ff_status launch_census_subpel(const uint8_t *imgn, int W, int H, int n, int q, int a, int b,
                               uint32_t *out, cudaStream_t st) {
  dim3 bl(32, 8), g((W + 31) / 32, (H + 7) / 8);
  k_census_subpel<<<g, bl, 0, st>>>(imgn, W, H, n, q, a, b, out);
  FF_CHECK_LAUNCH();
  return FF_OK;
}

// Relayout of a plain census image into the padded phase planes and their
// transposed copies.
__device__ __forceinline__ void planes_at(const uint32_t *__restrict__ census, const Planes &P,
                                          int i, int j, int pl) {
  const int px = pl % P.n, py = pl / P.n;
  const int x = clampi(px + P.n * (i - PLANE_PAD), 0, P.W - 1);
  const int y = clampi(py + P.n * (j - PLANE_PAD), 0, P.H - 1);
  const uint32_t v = census[(size_t)y * P.W + x];
  P.base[(size_t)pl * P.plane_words + (size_t)j * P.pitch + i] = v;
  if (i < P.NX + 2 * PLANE_PAD) P.baseT[(size_t)pl * P.plane_wordsT + (size_t)i * P.pitchT + j] = v;
}
__global__ void k_planes(const uint32_t *__restrict__ census, Planes P) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= P.pitch || j >= P.rows) return;
  planes_at(census, P, i, j, blockIdx.z);
}

ff_status launch_planes(const uint32_t *census, Planes P, cudaStream_t st) {
  dim3 b(64, 4), g((P.pitch + 63) / 64, (P.rows + 3) / 4, P.n * P.n);
  k_planes<<<g, b, 0, st>>>(census, P);
  FF_CHECK_LAUNCH();
  return FF_OK;
}

// ---------------------------------------------------------- batched form ----
// The same steps over many frames per launch (blockIdx.y, or blockIdx.z for the
// planes, selects the job); blocks past a smaller job's extent return.
__global__ void k_area_down_b(const PyrJob *J, int n) {
  const PyrJob &j = J[blockIdx.y];
  const int Wc = (j.W + n - 1) / n, Hc = (j.H + n - 1) / n;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= Wc * Hc * 3) return;
  area_down_at(j.img, j.W, j.H, n, j.down, Wc, t);
}
__global__ void k_lanczos_h_b(const PyrJob *J, int n, LanczosTable tab) {
  const PyrJob &j = J[blockIdx.y];
  const int Wc = (j.W + n - 1) / n, Hc = (j.H + n - 1) / n;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= Hc * j.W * 3) return;
  lanczos_h_at(j.down, Wc, j.W, n, tab, j.h, t);
}
__global__ void k_lanczos_v_b(const PyrJob *J, int n, LanczosTable tab) {
  const PyrJob &j = J[blockIdx.y];
  const int Hc = (j.H + n - 1) / n;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= j.H * j.W * 3) return;
  lanczos_v_at(j.h, Hc, j.W, n, tab, j.sm, t);
}
__global__ void k_census_b(const PyrJob *J, int n) {
  const PyrJob &j = J[blockIdx.y];
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= j.W * j.H) return;
  census_at(n > 1 ? j.sm : j.img, j.W, j.H, n, j.census, t % j.W, t / j.W);
}
__global__ void k_planes_b(const PyrJob *J, int nn) {
  const PyrJob &j = J[blockIdx.z / nn];
  const int i = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= j.pl.pitch || r >= j.pl.rows) return;
  planes_at(j.census, j.pl, i, r, blockIdx.z % nn);
}

// I^n (n > 1) of every job (img -> down -> h -> sm), three launches; census and
// planes are not touched.
ff_status launch_smooth_batch(const PyrJob *host, PyrJob *dev, int njobs, int n, cudaStream_t st) {
  if (njobs <= 0) return FF_OK;
  if (n < 2 || n > 16 || (n & (n - 1)) || njobs > 65535) return FF_ERR_INVALID_ARG;
  int maxA = 0, maxH = 0, maxV = 0;
  for (int i = 0; i < njobs; i++) {
    const int W = host[i].W, H = host[i].H, Wc = (W + n - 1) / n, Hc = (H + n - 1) / n;
    maxA = max(maxA, Wc * Hc * 3);
    maxH = max(maxH, Hc * W * 3);
    maxV = max(maxV, H * W * 3);
  }
  FF_TRY(upload_desc(host, dev, njobs, st));
  const int B = 256;
  LanczosTable tab;
  lanczos_table(n, &tab);
  k_area_down_b<<<dim3((maxA + B - 1) / B, njobs), B, 0, st>>>(dev, n);
  FF_CHECK_LAUNCH();
  k_lanczos_h_b<<<dim3((maxH + B - 1) / B, njobs), B, 0, st>>>(dev, n, tab);
  FF_CHECK_LAUNCH();
  k_lanczos_v_b<<<dim3((maxV + B - 1) / B, njobs), B, 0, st>>>(dev, n, tab);
  FF_CHECK_LAUNCH();
  return FF_OK;
}

ff_status launch_pyramid_level(const PyrJob *host, PyrJob *dev, int njobs, int n, cudaStream_t st) {
  if (njobs <= 0) return FF_OK;
  if (n < 1 || n > 16 || (n & (n - 1))) return FF_ERR_INVALID_ARG;
  const int chunk = 65535 / (n * n);  // grid.y / grid.z limits
  if (njobs > chunk) {
    for (int i = 0; i < njobs; i += chunk)
      FF_TRY(launch_pyramid_level(host + i, dev + i, min(chunk, njobs - i), n, st));
    return FF_OK;
  }
  int maxA = 0, maxH = 0, maxV = 0, maxP = 0, maxPitch = 0, maxRows = 0;
  for (int i = 0; i < njobs; i++) {
    const int W = host[i].W, H = host[i].H, Wc = (W + n - 1) / n, Hc = (H + n - 1) / n;
    maxA = max(maxA, Wc * Hc * 3);
    maxH = max(maxH, Hc * W * 3);
    maxV = max(maxV, H * W * 3);
    maxP = max(maxP, W * H);
    maxPitch = max(maxPitch, host[i].pl.pitch);
    maxRows = max(maxRows, host[i].pl.rows);
  }
  FF_TRY(upload_desc(host, dev, njobs, st));
  const int B = 256;
  if (n > 1) {
    LanczosTable tab;
    lanczos_table(n, &tab);
    k_area_down_b<<<dim3((maxA + B - 1) / B, njobs), B, 0, st>>>(dev, n);
    FF_CHECK_LAUNCH();
    k_lanczos_h_b<<<dim3((maxH + B - 1) / B, njobs), B, 0, st>>>(dev, n, tab);
    FF_CHECK_LAUNCH();
    k_lanczos_v_b<<<dim3((maxV + B - 1) / B, njobs), B, 0, st>>>(dev, n, tab);
    FF_CHECK_LAUNCH();
  }
  k_census_b<<<dim3((maxP + B - 1) / B, njobs), B, 0, st>>>(dev, n);
  FF_CHECK_LAUNCH();
  const dim3 pb(64, 4), pg((maxPitch + 63) / 64, (maxRows + 3) / 4, njobs * n * n);
  k_planes_b<<<pg, pb, 0, st>>>(dev, n * n);
  FF_CHECK_LAUNCH();
  return FF_OK;
}

}  // namespace ff
