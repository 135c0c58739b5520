// Sec. 4.1 (Table 1, "k=3+median"): the raw forward field filtered by a median
// weighted by the matching error. The paper gives neither window nor weights;
// reading: the matching error of pixel p is E(p) = E_d(P_r(p), P_r(p + F(p))) at
// full resolution (census of both frames with spacing 1, taps clamped), the
// weight w(q) = floor(2^16 / (1 + E(q))), the window the in-image pixels within
// rho (max-norm) of p, and each flow component the weighted lower median: the
// smallest value v whose samples <= v carry at least half of the total weight.
#include "ff_internal.cuh"

namespace ff {

constexpr int MEDIAN_MAX_RHO = 3;  // windows of up to 7 x 7

// E(p) by one thread per pixel, the (2r+1)^2 taps read with clamped coordinates.
__global__ void __launch_bounds__(256) k_match_errors(const uint32_t *__restrict__ C1,
                                                      const uint32_t *__restrict__ C2,
                                                      const uint32_t *__restrict__ F, int W, int H,
                                                      int r, int32_t *__restrict__ E) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= W * H) return;
  const int x = p % W, y = p / W;
  const uint32_t f = F[p];
  const int tx = x + flow_dx(f), ty = y + flow_dy(f);
  int e = 0;
  for (int v = -r; v <= r; v++) {
    const int ys = clampi(y + v, 0, H - 1), yt = clampi(ty + v, 0, H - 1);
    const uint32_t *rs = C1 + (size_t)ys * W, *rt = C2 + (size_t)yt * W;
    for (int u = -r; u <= r; u++)
      e += __popc(__ldg(rs + clampi(x + u, 0, W - 1)) ^ __ldg(rt + clampi(tx + u, 0, W - 1)));
  }
  E[p] = e;
}

// The weighted lower median of n (value, weight) samples: values sorted in
// place (insertion sort, n <= 49), then the first value at which twice the
// running weight reaches the total.
__device__ __forceinline__ int weighted_lower_median(int *v, int *w, int n, long long total) {
  for (int i = 1; i < n; i++) {
    const int a = v[i], b = w[i];
    int j = i;
    for (; j > 0 && v[j - 1] > a; j--) {
      v[j] = v[j - 1];
      w[j] = w[j - 1];
    }
    v[j] = a;
    w[j] = b;
  }
  long long run = 0;
  for (int i = 0; i < n; i++) {
    run += w[i];
    if (2 * run >= total) return v[i];
  }
  return v[n - 1];
}

__global__ void __launch_bounds__(128) k_weighted_median(const uint32_t *__restrict__ F,
                                                         const int32_t *__restrict__ E, int W, int H,
                                                         int rho, uint32_t *__restrict__ out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= W * H) return;
  const int x = p % W, y = p / W;
  constexpr int CAP = (2 * MEDIAN_MAX_RHO + 1) * (2 * MEDIAN_MAX_RHO + 1);
  int vx[CAP], vy[CAP], wx[CAP], wy[CAP];
  int n = 0;
  long long total = 0;
  for (int yy = max(y - rho, 0); yy <= min(y + rho, H - 1); yy++)
    for (int xx = max(x - rho, 0); xx <= min(x + rho, W - 1); xx++) {
      const size_t q = (size_t)yy * W + xx;
      const uint32_t f = F[q];
      const int w = 65536 / (1 + E[q]);
      vx[n] = flow_dx(f);
      vy[n] = flow_dy(f);
      wx[n] = w;
      wy[n] = w;
      total += w;
      n++;
    }
  const int mx = weighted_lower_median(vx, wx, n, total);
  const int my = weighted_lower_median(vy, wy, n, total);
  out[p] = pack_flow(mx, my);
}

size_t median_scratch_bytes(int W, int H) {
  Arena a;
  const size_t N = (size_t)W * H;
  a.take<uint32_t>(N);
  a.take<uint32_t>(N);
  a.take<int32_t>(N);
  return a.off;
}

}  // namespace ff

using namespace ff;

extern "C" {

ff_status ff_median_workspace_size(int W, int H, size_t *bytes) {
  FF_TRY(check_shape(W, H));
  if (!bytes) return FF_ERR_INVALID_ARG;
  *bytes = WS_HEADER + median_scratch_bytes(W, H);
  return FF_OK;
}

ff_status ff_weighted_median(const uint8_t *I1, const uint8_t *I2, const int16_t *flow, int W,
                             int H, int r, int rho, int16_t *out, int32_t *match_err, void *ws,
                             size_t ws_bytes, void *stream) {
  FF_TRY(check_shape(W, H));
  if (!I1 || !I2 || !flow || !out || r < 1 || r > PLANE_PAD || rho < 0 || rho > MEDIAN_MAX_RHO)
    return FF_ERR_INVALID_ARG;
  if (((uintptr_t)flow & 3) || ((uintptr_t)out & 3) || (uintptr_t)ws % 256) return FF_ERR_INVALID_ARG;
  if (!ws || ws_bytes < WS_HEADER + median_scratch_bytes(W, H)) return FF_ERR_WORKSPACE;
  if ((const void *)flow == (const void *)out) return FF_ERR_INVALID_ARG;  // out-of-place
  cudaStream_t st = (cudaStream_t)stream;
  const size_t N = (size_t)W * H;
  Arena a((char *)ws + WS_HEADER, ws_bytes - WS_HEADER);
  uint32_t *C1 = a.take<uint32_t>(N), *C2 = a.take<uint32_t>(N);
  int32_t *E = a.take<int32_t>(N);
  FF_TRY(launch_census(I1, W, H, 1, C1, st));
  FF_TRY(launch_census(I2, W, H, 1, C2, st));
  const int blocks = (int)((N + 255) / 256);
  k_match_errors<<<blocks, 256, 0, st>>>(C1, C2, (const uint32_t *)flow, W, H, r, E);
  FF_CHECK_LAUNCH();
  k_weighted_median<<<(int)((N + 127) / 128), 128, 0, st>>>((const uint32_t *)flow, E, W, H, rho,
                                                            (uint32_t *)out);
  FF_CHECK_LAUNCH();
  if (match_err &&
      cudaMemcpyAsync(match_err, E, N * sizeof(int32_t), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return FF_ERR_CUDA;
  return FF_OK;
}

}  // extern "C"
